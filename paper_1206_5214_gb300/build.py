"""Builds libmdwf.so (CUDA, sm_103a) in-tree under paper_1206_5214_gb300/_build/.

Each translation unit is compiled in parallel with
``nvcc -gencode arch=compute_103a,code=sm_103a -O3 -lineinfo`` and linked into
one shared library with the CUDA runtime linked statically; the library has
no dependency on PyTorch.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmdwf.so")
# the bounds-checked debug build (every field and link index checked on the device)
BUILD_BOUNDS = os.path.join(HERE, "_build_bounds")
LIB_BOUNDS = os.path.join(BUILD_BOUNDS, "libmdwf.so")
SOURCES = ["api.cu", "dslash.cu", "dslash_f64.cu", "dslash_f32.cu", "dslash_f16n.cu", "m5.cu", "layout.cu", "cg.cu", "force.cu", "noalloc.cu", "overlap.cu", "hmc4d.cu", "slab.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: libmdwf needs the CUDA toolkit to build")


def _flags(verbose_ptxas: bool, debug_bounds: bool = False) -> list[str]:
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
                "--expt-relaxed-constexpr"]
    if debug_bounds:
        f += ["-DMDWF_BOUNDS_CHECK=1"]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _inputs_newer(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    deps = [os.path.join(CSRC, s) for s in os.listdir(CSRC)] + [os.path.join(INCLUDE, "mdwf.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose_ptxas: bool = False, jobs: int | None = None,
          debug_bounds: bool = False) -> str:
    """Compile and link libmdwf.so if any source changed; return its path.
    debug_bounds: the bounds-checked debug build, in its own directory."""
    bdir, lib = (BUILD_BOUNDS, LIB_BOUNDS) if debug_bounds else (BUILD, LIB)
    os.makedirs(bdir, exist_ok=True)
    if not force and not verbose_ptxas and not _inputs_newer(lib):
        return lib
    cc = nvcc()

    def compile_one(src: str) -> tuple[str, str]:
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = [cc] + _flags(verbose_ptxas, debug_bounds) + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=jobs or len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose_ptxas:
        for _, log in results:
            sys.stderr.write(log)
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose_ptxas="-v" in sys.argv))
