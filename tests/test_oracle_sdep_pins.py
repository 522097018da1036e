"""Pins of the oracle with per-slice Moebius coefficients b5(s), c5(s).

Row s of Eq. (MoebiusOp) then uses D+^(s) = b5(s) D_W + 1 and
D-^(s) = c5(s) D_W - 1 (Eq. DWaction). What fixes the oracle here:

* constant arrays give the constant-coefficient operator (closed-form I_rr^-1
  against the general elimination);
* App. A: with T_s^-1 = (1 + H_s)/(1 - H_s),
  H_s = gamma5 (b5(s) + c5(s)) D_W / (2 + (b5(s) - c5(s)) D_W) and the ordered
  product T^-Ls = T_1^-1 T_2^-1 ... T_Ls^-1, the first column of
  P^dag D_DW(1)^-1 D_DW(m) P is D_ov(m) = (1+m)/2 + (1-m)/2 gamma5 (T^-Ls - 1)/(T^-Ls + 1),
  the other columns are the identity and the determinants agree; checked by
  dense algebra with random links, for the Zolotarev-type profile of Sec. 4.3
  (b5(s) - c5(s) fixed, commuting T_s) and for a generic profile;
* Sec. 2.1: with a reflection-symmetric profile gamma5 R D_-^-1 D_DW is Hermitian,
  and it is not for a profile without that symmetry;
* the red/black blocks, I_rr^-1, the Schur complement and the solve against
  dense algebra, as for constant coefficients.
"""
import numpy as np
import pytest

import synthetic as sy
from _pins import dense_of

GENERIC = ((1.2, 1.9, 1.4, 2.3), (0.1, 0.8, 0.2, 1.0))          # b5(s) - c5(s) varies, no symmetry
ZOLO = ((1.1, 1.6, 2.4, 1.3), (0.1, 0.6, 1.4, 0.3))             # b5(s) - c5(s) = 1 (Sec. 4.3)
SYMM = ((1.3, 2.0, 2.0, 1.3), (0.2, 1.1, 1.1, 0.2))             # b5(s) = b5(Ls+1-s), c5 likewise


@pytest.fixture(scope="module")
def orc(oracle_lib):
    return oracle_lib


@pytest.fixture(scope="module")
def tiny():
    dims = (4, 2, 2, 2)
    return dims, sy.gauge_field(dims, 0.3, 21)


def _params(orc, dims, prof, mf=0.1, Ls=4):
    b, c = prof
    return orc.Params(dims, Ls, 1.8, 1.5, 0.5, mf, b5s=tuple(b), c5s=tuple(c))


def _dense_ddw(orc, U, p, dagger=False):
    x, y, z, t = p.dims
    shape = (p.Ls, t, z, y, x, 4, 3)
    return dense_of(lambda v: orc.ddw(v, U, p, dagger), int(np.prod(shape)), shape)


def _dense_dw(orc, U, dims, M5):
    x, y, z, t = dims
    shape = (t, z, y, x, 4, 3)
    return dense_of(lambda v: orc.dw(v, U, dims, M5), int(np.prod(shape)), shape)


def _g5(V):
    return np.kron(np.eye(V), np.kron(np.diag([1, 1, -1, -1]), np.eye(3))).astype(complex)


def _wall_perm(Ls, V):
    Pp = np.kron(np.eye(V), np.kron(np.diag([1, 1, 0, 0]), np.eye(3)))
    Pm = np.kron(np.eye(V), np.kron(np.diag([0, 0, 1, 1]), np.eye(3)))
    n = 12 * V
    P = np.zeros((Ls * n, Ls * n), complex)
    for s in range(Ls):
        P[s * n:(s + 1) * n, s * n:(s + 1) * n] += Pm
        sp = (s + 1) % Ls
        P[s * n:(s + 1) * n, sp * n:(sp + 1) * n] += Pp
    return P


def _eo_index(dims, Ls):
    import oracle
    mask = np.broadcast_to(oracle.parity_mask(dims)[None, ..., None, None],
                           (Ls,) + tuple(reversed(dims)) + (4, 3)).reshape(-1)
    return np.nonzero(~mask)[0], np.nonzero(mask)[0]


def test_constant_arrays_equal_constant_operator(orc, tiny):
    """b5(s) = b5, c5(s) = c5 for all s: the general Ls x Ls elimination and the
    closed form of Sec. 3 give the same I_rr^-1 and the same M, M^dag."""
    dims, U = tiny
    Ls = 6
    p0 = orc.Params(dims, Ls, 1.8, 1.5, 0.5, 0.07)
    p1 = p0.with_(b5s=(1.5,) * Ls, c5s=(0.5,) * Ls)
    _, v = orc.split(sy.gaussian_field(dims, Ls, 31), dims)
    for dag in (False, True):
        a, b = orc.m(v, U, p0, dagger=dag), orc.m(v, U, p1, dagger=dag)
        assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()
        a, b = orc.mee_inv(v, p0, dagger=dag), orc.mee_inv(v, p1, dagger=dag)
        assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()


@pytest.mark.parametrize("prof", [ZOLO, GENERIC], ids=["zolotarev-type", "generic"])
def test_transfer_matrix_overlap_identity(orc, tiny, prof):
    """App. A with per-slice coefficients, random links (see module docstring)."""
    dims, U = tiny
    Ls, M5, m = 4, 1.8, 0.1
    V = int(np.prod(dims))
    n = 12 * V
    p = _params(orc, dims, prof, m)
    Dm = _dense_ddw(orc, U, p)
    D1 = _dense_ddw(orc, U, p.with_(mf=1.0))
    P = _wall_perm(Ls, V)
    K = P.conj().T @ np.linalg.solve(D1, Dm) @ P
    A = P.conj().T @ np.linalg.solve(Dm, D1) @ P
    DW = _dense_dw(orc, U, dims, M5)
    g5, one = _g5(V), np.eye(n, dtype=complex)
    Tinv = one.copy()
    for b, c in zip(*prof):                           # T_1^-1 T_2^-1 ... T_Ls^-1
        Hs = g5 @ ((b + c) * DW) @ np.linalg.inv(2 * one + (b - c) * DW)
        Tinv = Tinv @ ((one + Hs) @ np.linalg.inv(one - Hs))
    eps = (Tinv - one) @ np.linalg.inv(Tinv + one)
    Dov = 0.5 * (1 + m) * one + 0.5 * (1 - m) * g5 @ eps
    assert np.allclose(K[:n, :n], Dov, atol=1e-11)
    assert np.allclose(K[:, n:], np.eye(Ls * n)[:, n:], atol=1e-11)
    assert np.allclose(A[:n, :n], np.linalg.inv(Dov), atol=1e-11)
    _, l1 = np.linalg.slogdet(np.linalg.solve(D1, Dm))
    _, l2 = np.linalg.slogdet(Dov)
    assert l1 == pytest.approx(l2, abs=1e-10)


def test_zolotarev_type_profile_order_free(orc, tiny):
    """With b5(s) - c5(s) fixed the T_s commute (Sec. 4.3): permuting the slices
    leaves the first column of K^DW unchanged."""
    dims, U = tiny
    V = int(np.prod(dims))
    n = 12 * V
    P = _wall_perm(4, V)
    outs = []
    for perm in ((0, 1, 2, 3), (2, 0, 3, 1)):
        prof = tuple(tuple(x[i] for i in perm) for x in ZOLO)
        p = _params(orc, dims, prof)
        K = P.conj().T @ np.linalg.solve(_dense_ddw(orc, U, p.with_(mf=1.0)), _dense_ddw(orc, U, p)) @ P
        outs.append(K[:n, :n])
    assert np.allclose(outs[0], outs[1], atol=1e-11)


def test_reflection_hermiticity(orc, tiny):
    """gamma5 R D_-^-1 D_DW(m) is Hermitian for b5(s), c5(s) symmetric under
    s -> Ls+1-s (Eq. Rsym), and not for the generic profile."""
    dims, U = tiny
    Ls, V = 4, int(np.prod(dims))
    n = 12 * V
    DW = _dense_dw(orc, U, dims, 1.8)
    g5 = _g5(V)
    herm = {}
    for name, prof in (("symm", SYMM), ("generic", GENERIC)):
        p = _params(orc, dims, prof)
        D = _dense_ddw(orc, U, p)
        H = np.zeros_like(D)
        for s in range(Ls):
            r = Ls - 1 - s
            Dm_inv = np.linalg.inv(prof[1][r] * DW - np.eye(n))
            H[s * n:(s + 1) * n] = g5 @ Dm_inv @ D[r * n:(r + 1) * n]
        herm[name] = np.abs(H - H.conj().T).max() / np.abs(H).max()
    assert herm["symm"] <= 1e-13
    assert herm["generic"] >= 1e-2


@pytest.mark.parametrize("prof", [GENERIC, SYMM], ids=["generic", "symmetric"])
def test_dagger_is_adjoint(orc, tiny, prof):
    dims, U = tiny
    p = _params(orc, dims, prof)
    assert np.allclose(_dense_ddw(orc, U, p, True), _dense_ddw(orc, U, p).conj().T, atol=1e-14)


def test_blocks_schur_complement_and_solve(orc, tiny):
    """Red/black blocks, I_rr^-1, M, M^dag and the full solve against dense
    algebra for the generic profile."""
    dims, U = tiny
    Ls = 4
    p = _params(orc, dims, GENERIC, mf=0.05)
    D = _dense_ddw(orc, U, p)
    ie, io = _eo_index(dims, Ls)
    Dee, Deo, Doe, Doo = D[np.ix_(ie, ie)], D[np.ix_(ie, io)], D[np.ix_(io, ie)], D[np.ix_(io, io)]
    Vh = int(np.prod(dims)) // 2
    hshape = (Ls, Vh, 4, 3)
    nh = int(np.prod(hshape))
    rng = np.random.default_rng(8)
    v = rng.standard_normal(nh) + 1j * rng.standard_normal(nh)
    vh = v.reshape(hshape)
    assert np.allclose(orc.mee(vh, p).reshape(-1), Dee @ v, atol=1e-13)
    assert np.allclose(orc.mee(vh, p, dagger=True).reshape(-1), Doo.conj().T @ v, atol=1e-13)
    assert np.allclose(orc.dhop(vh, U, p, 0).reshape(-1), Deo @ v, atol=1e-13)
    assert np.allclose(orc.dhop(vh, U, p, 1).reshape(-1), Doe @ v, atol=1e-13)
    assert np.allclose(orc.dhop(vh, U, p, 0, dagger=True).reshape(-1), Doe.conj().T @ v, atol=1e-13)
    assert np.allclose(orc.mee_inv(vh, p).reshape(-1), np.linalg.solve(Dee, v), atol=1e-12)
    assert np.allclose(orc.mee_inv(vh, p, dagger=True).reshape(-1), np.linalg.solve(Dee.conj().T, v), atol=1e-12)
    M = np.eye(nh) - np.linalg.solve(Doo, Doe @ np.linalg.solve(Dee, Deo))
    assert np.allclose(orc.m(vh, U, p).reshape(-1), M @ v, atol=1e-12)
    assert np.allclose(orc.m(vh, U, p, dagger=True).reshape(-1), M.conj().T @ v, atol=1e-12)
    b = sy.gaussian_field(dims, Ls, 2031)
    x, st, it, rel = orc.solve(b, U, p, tol=1e-13, maxiter=5000)
    assert st == 0
    xd = np.linalg.solve(D, b.reshape(-1)).reshape(b.shape)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-10


def test_force_per_slice_outputs(orc, tiny):
    """With per-slice coefficients the force returns Ls values of dS/db5(s) and
    dS/dc5(s) (their values are pinned in test_oracle_force_ext_pins.py)."""
    dims, U = tiny
    p = _params(orc, dims, GENERIC)
    _, phi = orc.split(sy.gaussian_field(dims, 4, 1), dims)
    S, G, db5, dc5, st, _ = orc.force(phi, U, p)
    assert st == 0 and G.shape == U.shape
    assert np.shape(db5) == (4,) and np.shape(dc5) == (4,)
    assert np.all(np.isfinite(db5)) and np.all(np.isfinite(dc5))
