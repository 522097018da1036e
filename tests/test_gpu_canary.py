"""NaN canaries (MDWF_CANARY=1): every allocation of the library starts as 0xFF
bytes, a NaN in every precision, so a kernel that reads memory nothing has
written spreads NaN into its result. In that mode a child process applies M and
M^dag in every precision (Ls = 8 and 16, constant and per-slice coefficients),
runs mixed and FP64 solves, the force and the overlap operator, and compares
them with the oracle at the usual tolerances."""
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
import os, sys
sys.path.insert(0, os.path.join(os.environ["MDWF_ROOT"], "tests"))
sys.path.insert(0, os.environ["MDWF_ROOT"])
import numpy as np, torch
import oracle, synthetic as sy
import paper_1206_5214_gb300 as mdwf
from _gpu import Ctx, rel_err
F64, F32, F16N = mdwf.MDWF_F64, mdwf.MDWF_F32, mdwf.MDWF_F16N
TOL = {F64: 1e-12, F32: 1e-5}

def check(got, ref, prec):
    emax, el2 = rel_err(got, ref)
    assert (el2 <= 3e-3) if prec == F16N else (emax <= TOL[prec]), (prec, emax, el2)

for dims, Ls, prof in (((4, 4, 4, 4), 8, None), ((4, 4, 2, 4), 16, None),
                       ((4, 4, 2, 4), 8, ([1.2, 1.9, 1.4, 2.3, 1.1, 1.7, 1.3, 2.0],
                                          [0.1, 0.8, 0.2, 1.0, 0.3, 0.6, 0.4, 0.9]))):
    U = sy.gauge_field(dims, 0.3, 1101)
    _, odd = oracle.split(sy.gaussian_field(dims, Ls, 2101), dims)
    p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, 0.02)
    if prof:
        p = p.with_(b5s=tuple(prof[0]), c5s=tuple(prof[1]))
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.02, U) as c:
        if prof:
            mdwf.mdwf_set_s_coefficients(c.h, *prof)
        for prec in (F64, F32, F16N):
            for dagger in (False, True):
                check(c.apply(odd, prec, dagger)[0], oracle.m(odd, U, p, dagger=dagger), prec)
    b = sy.gaussian_field(dims, Ls, 2102)
    h = mdwf.mdwf_create(dims, Ls, 1.8, 1.5, 0.5, 0.02)
    try:
        mdwf.mdwf_load_gauge(h, torch.from_numpy(U).cuda())
        if prof:
            mdwf.mdwf_set_s_coefficients(h, *prof)
        for inner in (F64, F32, F16N):
            bb = torch.from_numpy(b).cuda()
            x = torch.zeros_like(bb)
            st, info = mdwf.mdwf_cgne(h, x, bb, tol=1e-10, inner_prec=inner)
            assert st == 0 and info[0].true_res <= 1e-10, (inner, info[0].as_dict())
            r = b - oracle.ddw(x.cpu().numpy(), U, p)
            assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-7, inner
        G = torch.empty(U.shape, dtype=torch.complex128, device="cuda")
        S, db, dc, st, info = mdwf.mdwf_force(h, G, torch.from_numpy(odd).cuda(), tol=1e-12)
        assert st == 0 and np.isfinite(S) and bool(torch.isfinite(G).all()) and np.all(np.isfinite(db))
        psi = sy.gaussian_field(dims, 1, 2103)[0]
        out = torch.empty(psi.shape, dtype=torch.complex128, device="cuda")
        st, info = mdwf.mdwf_overlap_apply(h, out, torch.from_numpy(psi).cuda(), tol=1e-12)
        assert st == 0 and bool(torch.isfinite(out).all())
    finally:
        mdwf.mdwf_destroy(h)
print("canary ok")
'''


def test_no_kernel_reads_unwritten_memory():
    env = dict(os.environ, MDWF_CANARY="1", MDWF_ROOT=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], capture_output=True, text=True, cwd=ROOT, env=env,
                       timeout=900)
    assert r.returncode == 0 and "canary ok" in r.stdout, (r.stdout[-2000:], r.stderr[-4000:])
