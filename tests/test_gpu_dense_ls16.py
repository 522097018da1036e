"""The dense Ls x Ls s-operators at Ls = 16, the length whose epilogue is
compiled with its column length fixed: the operator with dense tables on two
lattice shapes, with per-slice (Zolotarev-type) coefficients and with several
right-hand sides at different masses, and the fused solve whose epilogues
apply A and A^dag as dense tables, all against the FP64 oracle at the bars of
the operator tests (FP32 1e-5 of the largest element, FP16+norm 3e-3 in the
2-norm)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle
import paper_1206_5214_gb300 as mdwf
import synthetic as sy
from paper_1206_5214_gb300 import zolotarev
from _gpu import Ctx, rel_err

pytestmark = pytest.mark.gpu

F32, F16N = mdwf.MDWF_F32, mdwf.MDWF_F16N
LS = 16


def check(got, ref, prec):
    emax, el2 = rel_err(got, ref)
    if prec == F16N:
        assert el2 <= 3e-3, (emax, el2)
    else:
        assert emax <= 1e-5, (emax, el2)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 2, 2, 4)], ids=["Vh128", "Vh48"])
@pytest.mark.parametrize("b5,c5", [(1.5, 0.5), (1.0, 0.0)], ids=["moebius", "shamir"])
@pytest.mark.parametrize("dagger", [False, True])
def test_dense_tables_ls16(dims, b5, c5, dagger):
    U = sy.gauge_field(dims, 0.3, 1401)
    odd = oracle.split(sy.gaussian_field(dims, LS, 2401), dims)[1]
    ref = oracle.m(odd, U, oracle.Params(dims, LS, 1.8, b5, c5, 0.03), dagger=dagger)
    with Ctx(dims, LS, 1.8, b5, c5, 0.03, U, dense_s=True) as c:
        for prec in (F32, F16N):
            check(c.apply(odd, prec, dagger)[0], ref, prec)


@pytest.mark.parametrize("dagger", [False, True])
def test_per_slice_coefficients_ls16(dagger):
    dims = (4, 4, 2, 4)
    b5s, c5s = zolotarev.zolotarev_coefficients(LS, 0.05, 0.756)
    U = sy.gauge_field(dims, 0.3, 1402)
    odd = oracle.split(sy.gaussian_field(dims, LS, 2402), dims)[1]
    p = oracle.Params(dims, LS, 1.8, 1.5, 0.5, 0.02, b5s=tuple(b5s), c5s=tuple(c5s))
    ref = oracle.m(odd, U, p, dagger=dagger)
    with Ctx(dims, LS, 1.8, 1.5, 0.5, 0.02, U) as c:
        mdwf.mdwf_set_s_coefficients(c.h, list(b5s), list(c5s))
        check(c.apply(odd, F32, dagger)[0], ref, F32)


def test_multi_mass_dense_tables_ls16():
    """Three right-hand sides at three masses: each block multiplies by its own
    right-hand side's tables."""
    dims, masses = (4, 4, 2, 4), [0.01, 0.1, 0.4]
    U = sy.gauge_field(dims, 0.3, 1403)
    b = sy.gaussian_field(dims, LS, 2403, nrhs=3)
    odd = np.stack([oracle.split(b[r], dims)[1] for r in range(3)])
    with Ctx(dims, LS, 1.8, 1.5, 0.5, 0.01, U, dense_s=True) as c:
        got = c.apply(odd, F32, False, nrhs=3, masses=masses)
    for r, m in enumerate(masses):
        check(got[r], oracle.m(odd[r], U, oracle.Params(dims, LS, 1.8, 1.5, 0.5, m)), F32)


@pytest.mark.parametrize("inner", [F32, F16N], ids=["mixed-f32", "mixed-f16n"])
def test_fused_solve_with_dense_tables_ls16(inner):
    """The fused iteration applies A (and A^dag for v) as dense tables in its
    epilogues; the mixed solve reaches 1e-10 and the oracle confirms it."""
    dims = (4, 4, 4, 4)
    U = sy.gauge_field(dims, 0.3, 1404)
    b = sy.gaussian_field(dims, LS, 2404)
    p = oracle.Params(dims, LS, 1.8, 1.5, 0.5, 0.01)
    h = mdwf.mdwf_create(dims, LS, 1.8, 1.5, 0.5, 0.01, dense_s=True)
    try:
        mdwf.mdwf_load_gauge(h, torch.from_numpy(U).cuda())
        bd = torch.from_numpy(b).cuda()
        x = torch.zeros_like(bd)
        st, info = mdwf.mdwf_cgne(h, x, bd, tol=1e-10, inner_prec=inner)
        xs = x.cpu().numpy()
    finally:
        mdwf.mdwf_destroy(h)
    assert st == 0 and info[0].true_res <= 1e-10
    bp = oracle.prepare(b, U, p)
    src = oracle.m(bp, U, p, dagger=True)
    _, xo = oracle.split(xs, dims)
    assert np.linalg.norm(src - oracle.mdagm(xo, U, p)) / np.linalg.norm(src) <= 1.05e-10
