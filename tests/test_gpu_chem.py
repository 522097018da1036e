"""GPU operator with a chemical potential on the time links (Sec. 6.6) against
the FP64 oracle with the same mu: M and M^dag in every precision (tolerances
of the operator tests), the adjoint identity, a mixed-precision solve, the
overlap operator with its non-Hermitian kernel, and the force's refusal."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle
import paper_1206_5214_gb300 as mdwf
import synthetic as sy
from _gpu import Ctx, rel_err
from _pins import dense_of

pytestmark = pytest.mark.gpu

F64, F32, F16N = mdwf.MDWF_F64, mdwf.MDWF_F32, mdwf.MDWF_F16N
MU = 0.3


def check(gpu, ref, prec):
    emax, el2 = rel_err(gpu, ref)
    if prec == F16N:
        assert el2 <= 3e-3, (emax, el2)
    else:
        assert emax <= {F64: 1e-12, F32: 1e-5}[prec], (emax, el2)


@pytest.mark.parametrize("prec", [F64, F32, F16N])
@pytest.mark.parametrize("dagger", [False, True])
def test_apply_with_chemical_potential(prec, dagger):
    dims, Ls = (4, 4, 4, 4), 8
    U = sy.gauge_field(dims, 0.3, 1081)
    _, odd = oracle.split(sy.gaussian_field(dims, Ls, 2081), dims)
    p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, 0.02, mu=MU)
    ref = oracle.m(odd, U, p, dagger=dagger)
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.02, U) as c:
        mdwf.mdwf_set_chemical_potential(c.h, MU)
        check(c.apply(odd, prec, dagger)[0], ref, prec)
        # and back to mu = 0
        mdwf.mdwf_set_chemical_potential(c.h, 0.0)
        check(c.apply(odd, prec, dagger)[0], oracle.m(odd, U, p.with_(mu=0.0), dagger=dagger), prec)


def test_adjoint_identity_with_chemical_potential():
    dims, Ls = (4, 4, 2, 4), 6
    U = sy.gauge_field(dims, 0.3, 1082)
    _, x = oracle.split(sy.gaussian_field(dims, Ls, 2082), dims)
    _, y = oracle.split(sy.gaussian_field(dims, Ls, 2083), dims)
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.02, U) as c:
        mdwf.mdwf_set_chemical_potential(c.h, MU)
        my = c.apply(y, F64)[0]
        mdx = c.apply(x, F64, dagger=True)[0]
    lhs, rhs = np.vdot(x, my), np.vdot(mdx, y)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_cgne_with_chemical_potential():
    dims, Ls, mf = (4, 4, 4, 4), 8, 0.02
    U = sy.gauge_field(dims, 0.3, 1084)
    b = sy.gaussian_field(dims, Ls, 2084)
    p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, mf, mu=MU)
    h = mdwf.mdwf_create(dims, Ls, 1.8, 1.5, 0.5, mf)
    try:
        mdwf.mdwf_load_gauge(h, torch.from_numpy(U).cuda())
        mdwf.mdwf_set_chemical_potential(h, MU)
        bb = torch.from_numpy(b).cuda()
        x = torch.zeros_like(bb)
        st, info = mdwf.mdwf_cgne(h, x, bb, tol=1e-10, inner_prec=F32)
        assert st == 0
        xs = x.cpu().numpy()
        G = torch.empty(U.shape, dtype=torch.complex128, device="cuda")
        _, _, _, fst, _ = mdwf.mdwf_force(h, G, torch.from_numpy(oracle.split(b, dims)[1]).cuda(),
                                          raise_on_error=False)
        assert fst == 1
    finally:
        mdwf.mdwf_destroy(h)
    r = b - oracle.ddw(xs, U, p)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-7


def test_overlap_with_nonhermitian_kernel():
    """2^4, Ls = 4: D_ov(m) with A = gamma5 (b5+c5) D_W(mu) / (2 + (b5-c5) D_W(mu))."""
    dims, Ls, M5, m, b5, c5 = (2, 2, 2, 2), 4, 1.8, 0.1, 1.5, 0.5
    U = sy.gauge_field(dims, 0.3, 1085)
    V, n = 16, 192
    DW = dense_of(lambda v: oracle.dw(v, U, dims, M5, mu=MU), n, (2, 2, 2, 2, 4, 3))
    g5 = np.kron(np.eye(V), np.kron(np.diag([1, 1, -1, -1]), np.eye(3))).astype(complex)
    one = np.eye(n)
    A = g5 @ ((b5 + c5) * DW) @ np.linalg.inv(2 * one + (b5 - c5) * DW)
    Pl, Mi = np.linalg.matrix_power(one + A, Ls), np.linalg.matrix_power(one - A, Ls)
    Dov = 0.5 * (1 + m) * one + 0.5 * (1 - m) * g5 @ (Pl - Mi) @ np.linalg.inv(Pl + Mi)
    rng = np.random.default_rng(3)
    psi = rng.standard_normal((2, 2, 2, 2, 4, 3)) + 1j * rng.standard_normal((2, 2, 2, 2, 4, 3))
    h = mdwf.mdwf_create(dims, Ls, M5, b5, c5, m)
    try:
        mdwf.mdwf_load_gauge(h, torch.from_numpy(U).cuda())
        mdwf.mdwf_set_chemical_potential(h, MU)
        out = np.empty_like(psi)
        st, info = mdwf.mdwf_overlap_apply(h, out, psi, tol=1e-13)
    finally:
        mdwf.mdwf_destroy(h)
    assert st == 0
    ref = (Dov @ psi.reshape(-1)).reshape(psi.shape)
    assert np.abs(out - ref).max() <= 1e-9 * np.abs(ref).max()
