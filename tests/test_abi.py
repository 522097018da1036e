"""The C-ABI library builds, loads without a GPU and exports every symbol that
``include/*.h`` declares; argument validation happens before any CUDA call."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(mdwf_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_1206_5214_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["mdwf_create", "mdwf_destroy", "mdwf_load_gauge", "mdwf_apply", "mdwf_apply_dag",
                     "mdwf_cgne", "mdwf_field_import", "mdwf_field_export", "mdwf_strerror"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_has_no_torch_dependency(libpath):
    out = subprocess.run(["ldd", libpath], capture_output=True, text=True).stdout
    assert "torch" not in out and "c10" not in out


def test_argument_validation_without_gpu(libpath):
    import paper_1206_5214_gb300 as m
    lib = m.load()
    h = ctypes.c_void_p()
    bad_dims = (ctypes.c_int * 4)(3, 4, 4, 4)
    assert lib.mdwf_create(ctypes.byref(h), bad_dims, 8, 1.8, 1.5, 0.5, 0.01, None) == 1
    dims = (ctypes.c_int * 4)(4, 4, 4, 4)
    assert lib.mdwf_create(ctypes.byref(h), dims, 7, 1.8, 1.5, 0.5, 0.01, None) == 1  # odd Ls
    assert lib.mdwf_create(ctypes.byref(h), dims, 0, 1.8, 1.5, 0.5, 0.01, None) == 1
    assert lib.mdwf_create(None, dims, 8, 1.8, 1.5, 0.5, 0.01, None) == 1
    assert lib.mdwf_apply(None, None, None, 0, 1, None) == 1
    assert lib.mdwf_cgne(None, None, None, 1, None, 0, None, None) == 1
    assert lib.mdwf_field_bytes(None, 0, 1) == 0
    assert m.mdwf_strerror(0) == "MDWF_OK"
    assert "invalid" in m.mdwf_strerror(1)


def _argtype(decl):
    decl = " ".join(decl.split())
    if "*" in decl or "[" in decl:
        return ctypes.c_void_p
    if decl.startswith("double"):
        return ctypes.c_double
    if decl.startswith("int") or decl.startswith("const int"):
        return ctypes.c_int
    raise AssertionError(f"unexpected parameter type in the header: {decl}")


def declared_signatures():
    """name -> (return type text, [parameter declarations]) from include/*.h."""
    sigs = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^\s*([A-Za-z_][\w\s\*]*?)\b(mdwf_\w+)\s*\(([^)]*)\)\s*;", text, flags=re.M | re.S):
            params = [p.strip() for p in m.group(3).split(",") if p.strip() and p.strip() != "void"]
            sigs[m.group(2)] = (m.group(1).strip(), params)
    return sigs


def test_every_entry_point_refuses_a_null_context(libpath):
    """Every call that takes a context returns MDWF_EINVAL for a NULL one (MDWF_OK for
    mdwf_destroy, 0 bytes for mdwf_field_bytes and mdwf_slab_face_bytes), before any CUDA call: no GPU is needed.
    A separate handle of the library is used, so that the binding's signatures stay as set."""
    lib = ctypes.CDLL(libpath)
    checked = 0
    for name, (ret, params) in declared_signatures().items():
        if not params or not re.match(r"(const )?mdwf_ctx\s*\*\s*\w+$", params[0]):
            continue
        f = getattr(lib, name)
        f.argtypes = [_argtype(p) for p in params]
        f.restype = ctypes.c_size_t if ret == "size_t" else ctypes.c_int
        args = [None if t is ctypes.c_void_p else t(0).value for t in f.argtypes]
        got = f(*args)
        expect = {"mdwf_destroy": 0, "mdwf_field_bytes": 0, "mdwf_slab_face_bytes": 0}.get(name, 1)
        assert got == expect, (name, got)
        checked += 1
    assert checked >= 30


def test_create_refuses_invalid_geometry(libpath):
    import paper_1206_5214_gb300 as m
    lib = m.load()
    h = ctypes.c_void_p()
    for dims, Ls in [((4, 4, 4, 0), 8), ((4, 4, 4, 4), 2 * 64 + 2), ((4, 4, 4, 4), -2), ((4, 4, 5, 4), 8)]:
        d = (ctypes.c_int * 4)(*dims)
        assert lib.mdwf_create(ctypes.byref(h), d, Ls, ctypes.c_double(1.8), ctypes.c_double(1.5),
                               ctypes.c_double(0.5), ctypes.c_double(0.01), None) == 1, (dims, Ls)
        assert not h.value


def test_strerror_names_every_status(libpath):
    import paper_1206_5214_gb300 as m
    names = [m.mdwf_strerror(s) for s in range(0, 9)]
    assert names[0] == "MDWF_OK"
    assert all(n.startswith("MDWF_") for n in names[:8]), names
    assert len(set(names[:8])) == 8
    assert not names[8].startswith("MDWF_")


def test_binding_signatures_match_the_header(libpath):
    """The ctypes binding declares every header function with the header's number of
    parameters, pointers where the header has pointers and doubles where it has doubles."""
    import paper_1206_5214_gb300 as m
    lib = m.load()
    for name, (ret, params) in declared_signatures().items():
        f = getattr(lib, name)
        assert f.argtypes is not None, f"{name} has no argtypes in the binding"
        assert len(f.argtypes) == len(params), (name, f.argtypes, params)
        for t, p in zip(f.argtypes, params):
            kind = _argtype(p)
            if kind is ctypes.c_void_p:
                assert t is ctypes.c_void_p or hasattr(t, "_type_") and t not in (ctypes.c_int, ctypes.c_double), \
                    (name, p, t)
            else:
                assert t is kind, (name, p, t)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without libmdwf.so the binding raises; it never falls back to the CPU."""
    import paper_1206_5214_gb300 as m
    monkeypatch.setattr(m, "_lib", None)
    monkeypatch.setattr(m._build, "LIB", str(tmp_path / "libmdwf.so"))
    with pytest.raises(OSError, match="not found"):
        m.load(build_if_missing=False)


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes structures of the binding have the C layout of the header's structs:
    a C program built against include/mdwf.h prints each struct's size and each field's
    offset, and they equal the ctypes figures (field names in the header's order)."""
    import shutil
    import subprocess
    import paper_1206_5214_gb300 as m
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"mdwf_opts": m._Opts, "mdwf_solve_params": m.SolveParams, "mdwf_solve_info": m.SolveInfo,
               "mdwf_kernel_stat": m.KernelStat}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "mdwf.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
