"""GPU operator with a chemical potential on the time links (Sec. 6.6) against
the FP64 oracle with the same mu: M and M^dag in every precision (tolerances
of the operator tests), the adjoint identity, a mixed-precision solve, the
overlap operator with its non-Hermitian kernel, and both forces against central
differences of the oracle's actions."""
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


def su3_direction(shape, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(shape + (3, 3)) + 1j * rng.standard_normal(shape + (3, 3))
    h = 0.5 * (a - np.conj(np.swapaxes(a, -1, -2)))
    return h - np.trace(h, axis1=-2, axis2=-1)[..., None, None] / 3.0 * np.eye(3)


def expm_ah(w):
    lam, v = np.linalg.eigh(1j * w)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(-1j * lam), np.conj(v))


def oracle_action(phi, U, p):
    """S = phi^dag (M^dag M)^-1 phi with the oracle's M^dag M (chemical potential included) dense."""
    A = dense_of(lambda v: oracle.mdagm(v, U, p), phi.size, phi.shape)
    return float(np.real(np.vdot(phi.reshape(-1), np.linalg.solve(A, phi.reshape(-1)))))


def test_force_with_chemical_potential():
    """4x2x2x2, Ls = 4, mu = 0.3: S, dS/dU along a random su(3) direction, dS/db5 and
    dS/dc5 against central differences (h = 1e-5) of the oracle's action."""
    dims, Ls, mf = (4, 2, 2, 2), 4, 0.05
    U = sy.gauge_field(dims, 0.3, 1086)
    _, phi = oracle.split(sy.gaussian_field(dims, Ls, 2086), dims)
    p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, mf, mu=MU)
    h = mdwf.mdwf_create(dims, Ls, 1.8, 1.5, 0.5, mf)
    try:
        mdwf.mdwf_load_gauge(h, torch.from_numpy(U).cuda())
        mdwf.mdwf_set_chemical_potential(h, MU)
        G = torch.empty(U.shape, dtype=torch.complex128, device="cuda")
        S, db5, dc5, st, info = mdwf.mdwf_force(h, G, torch.from_numpy(phi).cuda(), tol=1e-13)
        G = G.cpu().numpy()
    finally:
        mdwf.mdwf_destroy(h)
    assert st == 0
    assert S == pytest.approx(oracle_action(phi, U, p), rel=1e-10)
    eps = 1e-5
    w = su3_direction(U.shape[:-2], 86)
    fd = (oracle_action(phi, expm_ah(eps * w) @ U, p) - oracle_action(phi, expm_ah(-eps * w) @ U, p)) / (2 * eps)
    an = float(np.sum(np.real(np.conj(G) * (w @ U))))
    assert an == pytest.approx(fd, rel=1e-6)
    for name, got in (("b5", db5), ("c5", dc5)):
        v = getattr(p, name)
        fd = (oracle_action(phi, U, p.with_(**{name: v + eps})) -
              oracle_action(phi, U, p.with_(**{name: v - eps}))) / (2 * eps)
        assert got == pytest.approx(fd, rel=1e-6, abs=1e-9 * abs(S)), name


def oracle_wall_action(phi4, U, p):
    """S = |D(1)^dag D(m)^-dag P phi|^2 (Sec. 2.4) with the oracle's D_DW as dense matrices
    (exact solves: at mu != 0 an iterative solve to 1e-14 is not reachable in FP64)."""
    Ls = p.Ls
    shape = (Ls,) + phi4.shape
    n = int(np.prod(shape))
    D = dense_of(lambda v: oracle.ddw(v, U, p), n, shape)
    D1 = dense_of(lambda v: oracle.ddw(v, U, p.with_(mf=1.0)), n, shape)
    b = np.zeros(shape, complex)
    b[0, ..., 2:, :] = phi4[..., 2:, :]
    b[Ls - 1, ..., :2, :] = phi4[..., :2, :]
    chi = np.linalg.solve(D.conj().T, b.reshape(-1))
    eta = D1.conj().T @ chi
    return float(np.vdot(eta, eta).real)


def test_force4d_with_chemical_potential():
    """The wall-pseudofermion action with mu = 0.3 (4x2x2x2, Ls = 4): S against the oracle
    and dS/dU against central differences of the oracle's action (Richardson-extrapolated
    from h = 1e-4 and 5e-5)."""
    dims, Ls, mf = (4, 2, 2, 2), 4, 0.05
    U = sy.gauge_field(dims, 0.3, 1087)
    phi = sy.gaussian_field(dims, 1, 2087)[0]
    p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, mf, mu=MU)
    h = mdwf.mdwf_create(dims, Ls, 1.8, 1.5, 0.5, mf)
    try:
        mdwf.mdwf_load_gauge(h, torch.from_numpy(U).cuda())
        mdwf.mdwf_set_chemical_potential(h, MU)
        G = torch.empty(U.shape, dtype=torch.complex128, device="cuda")
        S, st, info = mdwf.mdwf_force4d(h, G, torch.from_numpy(phi).cuda(), tol=1e-12)
        G = G.cpu().numpy()
    finally:
        mdwf.mdwf_destroy(h)
    assert st == 0
    assert S == pytest.approx(oracle_wall_action(phi, U, p), rel=1e-9)
    w = su3_direction(U.shape[:-2], 87)

    def central(eps):
        return (oracle_wall_action(phi, expm_ah(eps * w) @ U, p) -
                oracle_wall_action(phi, expm_ah(-eps * w) @ U, p)) / (2 * eps)

    # Richardson: the O(h^2) error of the central differences cancels
    fd = (4.0 * central(5e-5) - central(1e-4)) / 3.0
    an = float(np.sum(np.real(np.conj(G) * (w @ U))))
    assert an == pytest.approx(fd, rel=1e-6)
