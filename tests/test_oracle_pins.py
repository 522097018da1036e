"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle (``oracle/``) against something other than
itself: printed scalars, closed forms at U = 1, exact identities of the paper
checked by dense linear algebra on tiny lattices, invariances, and special
cases that reduce to textbook operators. A dropped term, a wrong sign of M5,
a swapped projector, a transposed I_rr or a wrong corner fails at least one.
"""
import json
import os

import numpy as np
import pytest

import synthetic as sy
from _pins import (dense_of, eps_polar, free_wilson_momentum, gauge_rotate, momenta,
                   momentum_blocks_5d, overlap_operator, pauli_gammas, rotate_field,
                   wall_permutation)

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
PAR = [(1.0, 0.0), (1.5, 0.5), (1.0, 1.0), (2.5, 1.5)]


@pytest.fixture(scope="module")
def orc(oracle_lib):
    return oracle_lib


# ----------------------------------------------------------------- gammas

def test_gamma_basis(orc):
    g, g5 = orc.gammas()
    ref = pauli_gammas()
    for mu in range(4):
        assert np.allclose(g[mu], ref[mu], atol=0)
        assert np.allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            ac = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(ac, 2.0 * (mu == nu) * np.eye(4), atol=1e-15)
    assert np.allclose(g5, np.diag([1, 1, -1, -1]), atol=1e-15)
    assert np.allclose(g5, g[0] @ g[1] @ g[2] @ g[3], atol=1e-15)


# ------------------------------------------------------- polar sign function

def test_eps_scaling_rule_printed_bound():
    v = GOLDEN["eps_scaling_rule"]
    lam = np.linspace(*v["lambda_range"], 4001)
    d = np.abs(eps_polar(lam, v["Ls_shamir"]) - eps_polar(v["alpha"] * lam, v["Ls_moebius"]))
    assert d.max() < v["bound"]
    # below the printed window the bound fails (max ~1.34e-3 near lambda = 0.034):
    lam_lo = np.linspace(0.01, 0.06, 2001)
    d_lo = np.abs(eps_polar(lam_lo, 48) - eps_polar(4 * lam_lo, 12))
    assert 1.2e-3 < d_lo.max() < 1.5e-3


def test_eps_polar_symmetries():
    v = GOLDEN["eps_polar_symmetries"]
    Ls = v["Ls"]
    lam = np.geomspace(*v["lambda_range"], 501)
    e = eps_polar(lam, Ls)
    assert np.allclose(eps_polar(np.array([1.0, -1.0]), Ls), [1.0, -1.0], atol=0)
    assert np.allclose(eps_polar(-lam, Ls), -e, atol=1e-15)
    assert np.all(1.0 - e >= -1e-15)
    assert np.allclose(1 - eps_polar(1.0 / lam, Ls), 1 - e, atol=1e-13)
    # closed form: tanh(Ls artanh(lambda)) for |lambda| < 1
    sub = lam[lam < 1]
    assert np.allclose(eps_polar(sub, Ls), np.tanh(Ls * np.arctanh(sub)), atol=1e-14)
    # odd Ls breaks the inversion symmetry
    assert abs(eps_polar(0.3, 15) - eps_polar(1 / 0.3, 15)) > 1e-4


# --------------------------------------------------------------- free field

def test_free_wilson_plane_waves(orc):
    """oracle D_W at U = 1 equals the plane-wave closed form at every momentum."""
    dims = (4, 4, 2, 2)
    M5 = 1.8
    U = sy.unit_gauge(dims)

    def apply(src5):
        return orc.dw(src5[0], U, dims, M5)[None]

    blocks = momentum_blocks_5d(apply, dims, 1)
    for k, p in momenta(dims):
        assert np.allclose(blocks[k], free_wilson_momentum(p, M5), atol=1e-13)


def test_lambda_max_shamir(orc):
    """The Shamir H5 at U = 1 (a5 = 1) takes the value (8 - M5)/(10 - M5) ~ 3/4
    that the paper quotes as lambda_max at the doubler corner p = (pi, pi, pi, pi);
    the physical mode at p = 0 sits at M5/(2 - M5) > 1, which the polar
    approximation treats like its inverse. A Wilson mass of +M5 would give
    (8 + M5)/(10 + M5) at the corner instead."""
    v = GOLDEN["lambda_max_shamir"]
    M5 = v["M5"]
    dims = (4, 2, 2, 2)
    U = sy.unit_gauge(dims)
    blocks = momentum_blocks_5d(lambda s: orc.dw(s[0], U, dims, M5)[None], dims, 1)
    g5 = np.diag([1, 1, -1, -1]).astype(complex)
    corner = None
    for k, p in momenta(dims):
        if all(abs(pm - np.pi) < 1e-12 for pm in p[1:]) and abs(p[0] - np.pi) < 1e-12:
            DW = blocks[k]
            H = g5 @ DW @ np.linalg.inv(2 * np.eye(4) + DW)
            corner = np.abs(np.linalg.eigvalsh(0.5 * (H + H.conj().T)))
    target = (8 - M5) / (10 - M5)
    assert np.allclose(corner, target, atol=1e-13)
    assert abs(target - v["approx"]) < v["approx_tol"]
    assert np.abs(np.linalg.eigvals(g5 @ blocks[0, 0, 0, 0] @ np.linalg.inv(2 * np.eye(4) + blocks[0, 0, 0, 0]))).max() == pytest.approx(M5 / (2 - M5), rel=1e-12)


@pytest.mark.parametrize("b5,c5", PAR)
def test_free_field_overlap_identity(orc, b5, c5):
    """At U = 1, per momentum: [P^dag D_DW(m)^-1 D_DW(1) P]_11 = D_ov(m)^-1 with
    the polar eps_Ls of H_M (Eq. inverseDWFmatrix with Eq. GWapprox / ApproxEPS),
    and the other columns of K^DW = P^dag D(1)^-1 D(m) P are the identity (Eq. DWFmatrix)."""
    dims, Ls, M5, m = (4, 4, 4, 4), 8, 1.8, 0.05
    p = orc.Params(dims, Ls, M5, b5, c5, m)
    U = sy.unit_gauge(dims)
    Dm = momentum_blocks_5d(lambda s: orc.ddw(s, U, p), dims, Ls)
    D1 = momentum_blocks_5d(lambda s: orc.ddw(s, U, p.with_(mf=1.0)), dims, Ls)
    Pw = wall_permutation(Ls)
    g5 = np.diag([1, 1, -1, -1]).astype(complex)
    worst = 0.0
    for k, mom in list(momenta(dims))[::3]:
        A = Pw.conj().T @ np.linalg.solve(Dm[k], D1[k]) @ Pw
        K = Pw.conj().T @ np.linalg.solve(D1[k], Dm[k]) @ Pw
        Dov = overlap_operator(free_wilson_momentum(mom, M5), g5, Ls, b5, c5, m)
        worst = max(worst, np.abs(A[:4, :4] - np.linalg.inv(Dov)).max(), np.abs(K[:4, :4] - Dov).max())
        assert np.allclose(K[:, 4:], np.eye(4 * Ls)[:, 4:], atol=1e-11)
    assert worst < 1e-11


def test_overlap_identity_fails_for_wrong_m5_sign(orc):
    """Control: with the Wilson mass taken as +M5 the identity breaks."""
    dims, Ls, M5, m = (4, 4, 4, 4), 8, 1.8, 0.05
    p = orc.Params(dims, Ls, M5, 1.5, 0.5, m)
    U = sy.unit_gauge(dims)
    Dm = momentum_blocks_5d(lambda s: orc.ddw(s, U, p), dims, Ls)
    D1 = momentum_blocks_5d(lambda s: orc.ddw(s, U, p.with_(mf=1.0)), dims, Ls)
    Pw = wall_permutation(Ls)
    g5 = np.diag([1, 1, -1, -1]).astype(complex)
    k, mom = (1, 0, 2, 1), (2 * np.pi / 4, np.pi, 0.0, np.pi / 2)
    A = Pw.conj().T @ np.linalg.solve(Dm[k], D1[k]) @ Pw
    wrong = overlap_operator(free_wilson_momentum(mom, -M5), g5, Ls, 1.5, 0.5, m)
    assert np.abs(A[:4, :4] - np.linalg.inv(wrong)).max() > 1e-2


# -------------------------------------------------- dense, random gauge field

def _dense_ddw(orc, U, p, dagger=False):
    x, y, z, t = p.dims
    shape = (p.Ls, t, z, y, x, 4, 3)
    n = int(np.prod(shape))
    return dense_of(lambda v: orc.ddw(v, U, p, dagger), n, shape)


def _dense_dw(orc, U, dims, M5):
    x, y, z, t = dims
    shape = (t, z, y, x, 4, 3)
    return dense_of(lambda v: orc.dw(v, U, dims, M5), int(np.prod(shape)), shape)


def _g5_4d(V):
    return np.kron(np.eye(V), np.kron(np.diag([1, 1, -1, -1]), np.eye(3))).astype(complex)


def _wall_perm_full(Ls, V):
    """P of Eq. (Pmatrix) on [s][site][spin][colour]."""
    Pp = np.kron(np.eye(V), np.kron(np.diag([1, 1, 0, 0]), np.eye(3)))
    Pm = np.kron(np.eye(V), np.kron(np.diag([0, 0, 1, 1]), np.eye(3)))
    n = 12 * V
    P = np.zeros((Ls * n, Ls * n), complex)
    for s in range(Ls):
        P[s * n:(s + 1) * n, s * n:(s + 1) * n] += Pm
        sp = (s + 1) % Ls
        P[s * n:(s + 1) * n, sp * n:(sp + 1) * n] += Pp
    return P


@pytest.fixture(scope="module", params=[(4, 2, 2, 2), (2, 2, 2, 2)], ids=["4x2x2x2", "2^4"])
def tiny(request):
    dims = request.param
    U = sy.gauge_field(dims, 0.3, 11)
    return dims, U


@pytest.mark.parametrize("b5,c5", [(1.5, 0.5), (1.0, 0.0)])
def test_ddw_dagger_is_adjoint(orc, tiny, b5, c5):
    dims, U = tiny
    p = orc.Params(dims, 4, 1.8, b5, c5, 0.1)
    D = _dense_ddw(orc, U, p)
    Dd = _dense_ddw(orc, U, p, dagger=True)
    assert np.allclose(Dd, D.conj().T, atol=1e-14)


def test_dw_gamma5_hermitian(orc, tiny):
    dims, U = tiny
    V = int(np.prod(dims))
    DW = _dense_dw(orc, U, dims, 1.8)
    g5 = _g5_4d(V)
    assert np.allclose(g5 @ DW @ g5, DW.conj().T, atol=1e-14)


@pytest.mark.parametrize("b5,c5", [(1.5, 0.5), (1.0, 0.0)])
def test_gamma5_reflection_hermiticity(orc, tiny, b5, c5):
    """gamma5 R D_-^-1 D_DW(m) is Hermitian (Eq. Rsym and the Gamma5 relation of Sec. 2.1)."""
    dims, U = tiny
    Ls, V = 4, int(np.prod(dims))
    p = orc.Params(dims, Ls, 1.8, b5, c5, 0.1)
    D = _dense_ddw(orc, U, p)
    DW = _dense_dw(orc, U, dims, 1.8)
    Dminus_inv = np.linalg.inv(c5 * DW - np.eye(12 * V))
    n = 12 * V
    H = np.zeros_like(D)
    g5 = _g5_4d(V)
    for s in range(Ls):
        r = Ls - 1 - s
        H[s * n:(s + 1) * n] = g5 @ Dminus_inv @ D[r * n:(r + 1) * n]
    assert np.allclose(H, H.conj().T, atol=1e-12)


@pytest.mark.parametrize("b5,c5", [(1.5, 0.5), (1.0, 0.0), (1.0, 1.0)])
def test_overlap_identity_random_links(orc, tiny, b5, c5):
    """Random links: [A^DW]_11 = D_ov(m)^-1, K^DW = identity off the first
    column, and Det[D_DW(1)^-1 D_DW(m)] = Det[D_ov(m)] (Sec. 2.2, App. A)."""
    dims, U = tiny
    Ls, M5, m = 4, 1.8, 0.1
    V = int(np.prod(dims))
    n = 12 * V
    p = orc.Params(dims, Ls, M5, b5, c5, m)
    Dm = _dense_ddw(orc, U, p)
    D1 = _dense_ddw(orc, U, p.with_(mf=1.0))
    P = _wall_perm_full(Ls, V)
    A = P.conj().T @ np.linalg.solve(Dm, D1) @ P
    K = P.conj().T @ np.linalg.solve(D1, Dm) @ P
    DW = _dense_dw(orc, U, dims, M5)
    Dov = overlap_operator(DW, _g5_4d(V), Ls, b5, c5, m)
    assert np.allclose(A[:n, :n], np.linalg.inv(Dov), atol=1e-11)
    assert np.allclose(K[:n, :n], Dov, atol=1e-11)
    assert np.allclose(K[:, n:], np.eye(Ls * n)[:, n:], atol=1e-11)
    s1, l1 = np.linalg.slogdet(np.linalg.solve(D1, Dm))
    s2, l2 = np.linalg.slogdet(Dov)
    assert l1 == pytest.approx(l2, abs=1e-10)
    assert abs(s1 - s2) < 1e-9


def test_shamir_limit_textbook(orc, tiny):
    """b5 = 1, c5 = 0 is the textbook Shamir operator: D_W + 1 on the diagonal,
    -P- (s, s+1), -P+ (s, s-1), +m P+ (1, Ls), +m P- (Ls, 1)."""
    dims, U = tiny
    Ls, m = 4, 0.1
    V = int(np.prod(dims))
    n = 12 * V
    p = orc.Params(dims, Ls, 1.8, 1.0, 0.0, m)
    D = _dense_ddw(orc, U, p)
    DW = _dense_dw(orc, U, dims, 1.8)
    Pp = np.kron(np.eye(V), np.kron(np.diag([1, 1, 0, 0]), np.eye(3)))
    Pm = np.kron(np.eye(V), np.kron(np.diag([0, 0, 1, 1]), np.eye(3)))
    S = np.zeros_like(D)
    for s in range(Ls):
        S[s * n:(s + 1) * n, s * n:(s + 1) * n] = DW + np.eye(n)
        if s + 1 < Ls:
            S[s * n:(s + 1) * n, (s + 1) * n:(s + 2) * n] = -Pm
        if s > 0:
            S[s * n:(s + 1) * n, (s - 1) * n:s * n] = -Pp
    S[0:n, (Ls - 1) * n:] = m * Pp
    S[(Ls - 1) * n:, 0:n] = m * Pm
    assert np.allclose(D, S, atol=1e-14)


def test_gauge_covariance(orc, tiny):
    dims, U = tiny
    Om = sy.gauge_transform(dims, 3001)
    UO = gauge_rotate(U, Om)
    p = orc.Params(dims, 4, 1.8, 1.5, 0.5, 0.05)
    psi = sy.gaussian_field(dims, 4, 2001)
    lhs = orc.ddw(rotate_field(psi, Om), UO, p)
    rhs = rotate_field(orc.ddw(psi, U, p), Om)
    assert np.allclose(lhs, rhs, atol=1e-12)
    # and the preconditioned operator on odd sites
    _, po = orc.split(psi, dims)
    _, pO = orc.split(rotate_field(psi, Om), dims)
    e, o = orc.split(rotate_field(orc.join(np.zeros_like(po), orc.m(po, U, p), dims), Om), dims)
    assert np.allclose(orc.m(pO, UO, p), o, atol=1e-12)


def _eo_perm(dims, Ls):
    """Index arrays of the even and odd entries of a flattened full 5d field."""
    mask = np.broadcast_to(np.asarray(__import__("oracle").parity_mask(dims))[None, ..., None, None],
                           (Ls,) + tuple(reversed(dims)) + (4, 3)).reshape(-1)
    return np.nonzero(~mask)[0], np.nonzero(mask)[0]


@pytest.mark.parametrize("b5,c5", [(1.5, 0.5), (1.0, 0.0)])
def test_blocks_and_schur_complement(orc, tiny, b5, c5):
    """I_rr, D_rb, D_br are the red/black blocks of the dense D_DW; I_rr^-1 by
    the closed form inverts I_rr; M equals the Schur complement
    1 - I_bb^-1 D_br I_rr^-1 D_rb computed by dense algebra (Sec. 3)."""
    dims, U = tiny
    Ls = 4
    p = orc.Params(dims, Ls, 1.8, b5, c5, 0.1)
    D = _dense_ddw(orc, U, p)
    ie, io = _eo_perm(dims, Ls)
    Dee, Deo, Doe, Doo = D[np.ix_(ie, ie)], D[np.ix_(ie, io)], D[np.ix_(io, ie)], D[np.ix_(io, io)]
    Vh = int(np.prod(dims)) // 2
    hshape = (Ls, Vh, 4, 3)
    nh = int(np.prod(hshape))
    rng = np.random.default_rng(5)
    v = (rng.standard_normal(nh) + 1j * rng.standard_normal(nh))
    vh = v.reshape(hshape)
    assert np.allclose(orc.mee(vh, p).reshape(-1), Dee @ v, atol=1e-13)
    assert np.allclose(orc.mee(vh, p).reshape(-1), Doo @ v, atol=1e-13)
    assert np.allclose(orc.dhop(vh, U, p, 0).reshape(-1), Deo @ v, atol=1e-13)
    assert np.allclose(orc.dhop(vh, U, p, 1).reshape(-1), Doe @ v, atol=1e-13)
    assert np.allclose(orc.mee_inv(vh, p).reshape(-1), np.linalg.solve(Dee, v), atol=1e-12)
    assert np.allclose(orc.mee_inv(vh, p, dagger=True).reshape(-1), np.linalg.solve(Dee.conj().T, v), atol=1e-12)
    Mdense = np.eye(nh) - np.linalg.solve(Doo, Doe @ np.linalg.solve(Dee, Deo))
    assert np.allclose(orc.m(vh, U, p).reshape(-1), Mdense @ v, atol=1e-12)
    assert np.allclose(orc.m(vh, U, p, dagger=True).reshape(-1), Mdense.conj().T @ v, atol=1e-12)


def test_adjoint_consistency(orc):
    """<x, M y> = <M^dag x, y> for the independently written M and M^dag."""
    dims = (4, 4, 2, 2)
    U = sy.gauge_field(dims, 0.3, 12)
    p = orc.Params(dims, 6, 1.8, 1.5, 0.5, 0.02)
    _, x = orc.split(sy.gaussian_field(dims, 6, 1), dims)
    _, y = orc.split(sy.gaussian_field(dims, 6, 2), dims)
    lhs = np.vdot(x, orc.m(y, U, p))
    rhs = np.vdot(orc.m(x, U, p, dagger=True), y)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("b5,c5", [(1.5, 0.5), (1.0, 0.0)])
def test_solve_matches_dense_inverse(orc, tiny, b5, c5):
    """prepare -> CGNE -> reconstruct reproduces the dense solve of D_DW x = b."""
    dims, U = tiny
    Ls = 4
    p = orc.Params(dims, Ls, 1.8, b5, c5, 0.05)
    D = _dense_ddw(orc, U, p)
    b = sy.gaussian_field(dims, Ls, 2003)
    x, st, it, rel = orc.solve(b, U, p, tol=1e-13, maxiter=5000)
    assert st == 0 and rel <= 1e-13
    xd = np.linalg.solve(D, b.reshape(-1)).reshape(b.shape)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-10


# -------------------------------------------------------------------- force

def _su3_direction(shape, seed):
    """Random traceless anti-Hermitian omega per link, shape (..., 3, 3)."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(shape + (3, 3)) + 1j * rng.standard_normal(shape + (3, 3))
    h = 0.5 * (a - np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1) / 3.0
    return h - tr[..., None, None] * np.eye(3)


def _expm_su3(w):
    """exp of anti-Hermitian 3x3 matrices via eigh of i w."""
    lam, v = np.linalg.eigh(1j * w)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(-1j * lam), np.conj(v))


def test_force_finite_differences(orc):
    """dS/dU along U(t) = exp(t omega) U and dS/db5, dS/dc5 match central differences."""
    dims, Ls = (4, 2, 2, 2), 4
    U = sy.gauge_field(dims, 0.3, 13)
    p = orc.Params(dims, Ls, 1.8, 1.5, 0.5, 0.1)
    _, phi = orc.split(sy.gaussian_field(dims, Ls, 2013), dims)
    S, G, db5, dc5, st, _ = orc.force(phi, U, p, tol=1e-14)
    assert st == 0
    w = _su3_direction(U.shape[:-2], 7)
    h = 1e-5

    def S_of(UU, pp):
        return orc.force(phi, UU, pp, tol=1e-14)[0]

    Up = _expm_su3(h * w) @ U
    Um = _expm_su3(-h * w) @ U
    fd = (S_of(Up, p) - S_of(Um, p)) / (2 * h)
    an = np.sum(np.real(np.conj(G) * (w @ U)))
    assert an == pytest.approx(fd, rel=1e-6)
    fd_b5 = (S_of(U, p.with_(b5=p.b5 + h)) - S_of(U, p.with_(b5=p.b5 - h))) / (2 * h)
    fd_c5 = (S_of(U, p.with_(c5=p.c5 + h)) - S_of(U, p.with_(c5=p.c5 - h))) / (2 * h)
    assert db5 == pytest.approx(fd_b5, rel=1e-6)
    assert dc5 == pytest.approx(fd_c5, rel=1e-6)
    # the action itself: S = phi^dag (M^dag M)^-1 phi against a dense solve
    x, y, z, t = dims
    hshape = (Ls, x * y * z * t // 2, 4, 3)
    Md = dense_of(lambda v: orc.m(v, U, p), int(np.prod(hshape)), hshape)
    Sd = np.real(np.vdot(phi.reshape(-1), np.linalg.solve(Md.conj().T @ Md, phi.reshape(-1))))
    assert S == pytest.approx(Sd, rel=1e-11)


def test_adjoint_solve_inverts_the_adjoint(orc, tiny):
    """solve_dag(b) x satisfies D^dag x = b, equals the dense (D^dag)^-1 b and, for the
    adjoint pairing, <D^-dag b, c> = <b, D^-1 c> with the red/black solve."""
    dims, U = tiny
    Ls = 4
    p = orc.Params(dims, Ls, 1.8, 1.5, 0.5, 0.05)
    b = sy.gaussian_field(dims, Ls, 2061)
    c = sy.gaussian_field(dims, Ls, 2062)
    x, st, it, rel = orc.solve_dag(b, U, p, tol=1e-13)
    assert st == 0 and rel < 1e-11
    D = _dense_ddw(orc, U, p)
    xd = np.linalg.solve(D.conj().T, b.reshape(-1)).reshape(b.shape)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-10
    y, st2, _, _ = orc.solve(c, U, p, tol=1e-13)
    assert abs(np.vdot(x, c) - np.vdot(b, y)) < 1e-10 * abs(np.vdot(b, y))
