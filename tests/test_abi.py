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
