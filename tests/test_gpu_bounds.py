"""The bounds-checked debug build (every field and link index that a kernel
computes is checked against the extent of its buffer view; an access out of
range is skipped and recorded). It stands in for a device memory checker:
the parity cases of the operator, the fused solve (with and without the t
field), the t-slab stages, the allocation-free entry point and the force run
against the FP64 oracle on small and ragged lattices, in a separate process
that loads the debug library, and no access may have been out of range."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
sys.path.insert(0, ROOT)
sys.path.insert(0, TESTS)
import numpy as np, torch
import paper_1206_5214_gb300 as mdwf
from paper_1206_5214_gb300 import _build, domain
_build.LIB = _build.LIB_BOUNDS
import oracle, synthetic as sy
from _gpu import Ctx, rel_err
checked, bad = mdwf.mdwf_bounds_status(reset=True)
assert checked and not bad, (checked, bad)
F64, F32, F16N = mdwf.MDWF_F64, mdwf.MDWF_F32, mdwf.MDWF_F16N

def check(prec, got, ref):
    emax, el2 = rel_err(got, ref)
    assert (el2 <= 3e-3) if prec == F16N else (emax <= (1e-12 if prec == F64 else 1e-5)), (prec, emax, el2)

# operator and adjoint, three precisions, a ragged lattice and Ls = 16
for dims, Ls in (((4, 4, 4, 4), 8), ((2, 4, 6, 4), 6), ((4, 2, 2, 4), 16)):
    U = sy.gauge_field(dims, 0.3, 1301)
    odd = oracle.split(sy.gaussian_field(dims, Ls, 2301), dims)[1]
    p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, 0.02)
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.02, U) as c:
        for prec in (F64, F32, F16N):
            for dag in (False, True):
                check(prec, c.apply(odd, prec, dag)[0], oracle.m(odd, U, p, dagger=dag))
        fin = c.upload(odd, F32)
        got = c.alloc(F32)
        mdwf.mdwf_apply_noalloc(c.h, got, fin, F32, 1, [0.02])
        torch.cuda.synchronize()
        check(F32, c.download(got, F32)[0], oracle.m(odd, U, p))

# mixed solves: Ls = 16 (no t field) and Ls = 8, two right-hand sides
for Ls in (16, 8):
    dims = (4, 4, 4, 4)
    U = sy.gauge_field(dims, 0.3, 1302)
    b = sy.gaussian_field(dims, Ls, 2302, nrhs=2)
    h = mdwf.mdwf_create(dims, Ls, 1.8, 1.5, 0.5, 0.01)
    try:
        mdwf.mdwf_load_gauge(h, torch.from_numpy(U).cuda())
        bd = torch.from_numpy(b).cuda()
        x = torch.zeros_like(bd)
        st, info = mdwf.mdwf_cgne(h, x, bd, nrhs=2, mf_per_rhs=[0.01, 0.05], tol=1e-10, inner_prec=F32)
        assert st == 0 and all(i.true_res <= 1e-10 for i in info), [i.as_dict() for i in info]
        phi = torch.from_numpy(np.ascontiguousarray(oracle.split(b[0], dims)[1])).cuda()
        G = torch.empty(U.shape, dtype=torch.complex128, device="cuda")
        S, db5, dc5, st, finfo = mdwf.mdwf_force(h, G, phi, tol=1e-11)
        assert st == 0
    finally:
        mdwf.mdwf_destroy(h)
    xs = x.cpu().numpy()
    for r, m in enumerate((0.01, 0.05)):
        p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, m)
        res = b[r] - oracle.ddw(xs[r], U, p)
        assert np.linalg.norm(res) / np.linalg.norm(b[r]) <= 1e-7, (Ls, r)

# t-slab stages, two slabs
dims, Ls = (4, 4, 4, 8), 8
part = domain.SlabPartition(dims, 2)
U = sy.gauge_field(dims, 0.3, 1303)
odd = oracle.split(sy.gaussian_field(dims, Ls, 2303), dims)[1][None]
for prec in (F64, F32):
    ctxs, ins, outs = [], [], []
    try:
        for r in range(2):
            h = mdwf.mdwf_create_slab(part.local_dims, Ls, 1.8, 1.5, 0.5, 0.02)
            ctxs.append(h)
            mdwf.mdwf_load_gauge(h, torch.from_numpy(part.gauge(U, r)).cuda())
            fi = torch.empty(mdwf.mdwf_field_bytes(h, prec, 1), dtype=torch.uint8, device="cuda")
            mdwf.mdwf_field_import(h, fi, torch.from_numpy(np.ascontiguousarray(part.odd(odd, r))).cuda(), prec, 1)
            ins.append(fi)
            outs.append(torch.empty_like(fi))
        domain.apply_local(mdwf, ctxs, outs, ins, prec, 1)
        got = []
        for r in range(2):
            o = torch.empty((1, Ls, part.vh_local, 4, 3), dtype=torch.complex128, device="cuda")
            mdwf.mdwf_field_export(ctxs[r], o, outs[r], prec, 1)
            got.append(o.cpu().numpy())
    finally:
        for h in ctxs:
            mdwf.mdwf_destroy(h)
    check(prec, part.join_odd(got)[0], oracle.m(odd[0], U, oracle.Params(dims, Ls, 1.8, 1.5, 0.5, 0.02)))

checked, bad = mdwf.mdwf_bounds_status()
assert checked and not bad, "an index was out of range"
print("BOUNDS-CLEAN")
'''


def test_bounds_checked_build_runs_the_parity_cases_clean():
    from paper_1206_5214_gb300 import build
    build.build(debug_bounds=True)
    code = CHILD.replace("ROOT", repr(ROOT)).replace("TESTS", repr(os.path.join(ROOT, "tests")))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0 and "BOUNDS-CLEAN" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]


def test_release_build_reports_no_checks():
    import paper_1206_5214_gb300 as mdwf
    assert mdwf.mdwf_bounds_status() == (False, False)
