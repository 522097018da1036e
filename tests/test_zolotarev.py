"""Pins of the Zolotarev coefficients (Sec. 4.3) against what fixes them:
the alternation theorem (the best uniform approximation's error equioscillates
at N + 1 points), the rational form they are built from, the polar form they
must beat at equal Ls, and App. A's effective operator computed by the oracle
with the resulting per-slice b5(s), c5(s)."""
import numpy as np
import pytest

import synthetic as sy
from _pins import dense_of, hermitian_function
from paper_1206_5214_gb300 import zolotarev as z

CASES = [(6, 0.05, 1.0), (8, 0.02, 1.5), (10, 0.01, 1.0), (12, 0.05, 2.0)]


def extrema(e):
    d = np.diff(e)
    idx = np.where(np.sign(d[1:]) != np.sign(d[:-1]))[0] + 1
    return np.concatenate([[e[0]], e[idx], [e[-1]]])


@pytest.mark.parametrize("Ls,lmin,lmax", CASES)
def test_error_equioscillates(Ls, lmin, lmax):
    """1 - eps has Ls + 1 alternating extrema of one magnitude on [lmin, lmax]."""
    w = z.zolotarev_omegas(Ls, lmin, lmax)
    x = np.geomspace(lmin, lmax, 400001)
    ext = extrema(1.0 - z.eps_of_omegas(x, w))
    assert len(ext) == Ls + 1
    assert np.all(np.sign(ext[1:]) == -np.sign(ext[:-1]))
    assert np.abs(ext).max() / np.abs(ext).min() - 1 < 1e-5
    # odd: eps(-x) = -eps(x)
    assert np.allclose(z.eps_of_omegas(-x[::997], w), -z.eps_of_omegas(x[::997], w), atol=1e-14)


@pytest.mark.parametrize("Ls,lmin,lmax", CASES)
def test_beats_polar(Ls, lmin, lmax):
    """Smaller max error than the polar form at every scale alpha (scanned)."""
    x = np.geomspace(lmin, lmax, 20001)
    ez = np.abs(1.0 - z.eps_of_omegas(x, z.zolotarev_omegas(Ls, lmin, lmax))).max()
    best_polar = min(np.abs(1.0 - z.eps_of_omegas(x, np.full(Ls, a))).max()
                     for a in np.geomspace(0.2 / lmax, 5.0 / lmin, 400))
    assert ez < best_polar


def test_omegas_reproduce_the_rational_form():
    """eps from the omegas equals D x prod(x^2 + c_even) / prod(x^2 + c_odd)."""
    Ls, k = 8, 0.03
    w = z.zolotarev_omegas(Ls, k, 1.0)
    c = z._c_coefficients(Ls, k)
    x = np.geomspace(k, 1.0, 2001)
    r = z._unscaled(x, c)
    D = z.eps_of_omegas(x, w)[0] / r[0]
    assert np.allclose(z.eps_of_omegas(x, w), D * r, rtol=1e-10, atol=0)


def test_coefficients_split():
    b, c = z.zolotarev_coefficients(8, 0.05, 1.0, a5=1.5)
    assert np.allclose(np.array(b) - np.array(c), 1.5)
    assert np.allclose((np.array(b) + np.array(c)) / 1.5, z.zolotarev_omegas(8, 0.05, 1.0))
    pb, pc = z.polar_coefficients(4, 2.0)
    assert pb == [1.5] * 4 and pc == [0.5] * 4


def test_effective_operator_with_zolotarev_slices(oracle_lib):
    """The oracle's 5d operator with the Zolotarev b5(s), c5(s) reduces (App. A)
    to (1+m)/2 + (1-m)/2 gamma5 eps(H_T), eps the Zolotarev function of
    H_T = gamma5 D_W / (2 + D_W) (a5 = 1), random links, 2^4, Ls = 4."""
    orc = oracle_lib
    dims, Ls, M5, m = (2, 2, 2, 2), 4, 1.8, 0.1
    U = sy.gauge_field(dims, 0.3, 23)
    V = 16
    n = 12 * V
    b5s, c5s = z.zolotarev_coefficients(Ls, 0.1, 1.0)
    p = orc.Params(dims, Ls, M5, 1.5, 0.5, m, b5s=tuple(b5s), c5s=tuple(c5s))
    shape = (Ls, 2, 2, 2, 2, 4, 3)
    Dm = dense_of(lambda v: orc.ddw(v, U, p), Ls * n, shape)
    D1 = dense_of(lambda v: orc.ddw(v, U, p.with_(mf=1.0)), Ls * n, shape)
    Pp = np.kron(np.eye(V), np.kron(np.diag([1, 1, 0, 0]), np.eye(3)))
    Pm = np.kron(np.eye(V), np.kron(np.diag([0, 0, 1, 1]), np.eye(3)))
    P = np.zeros((Ls * n, Ls * n), complex)
    for s in range(Ls):
        P[s * n:(s + 1) * n, s * n:(s + 1) * n] += Pm
        sp = (s + 1) % Ls
        P[s * n:(s + 1) * n, sp * n:(sp + 1) * n] += Pp
    K = P.conj().T @ np.linalg.solve(D1, Dm) @ P
    DW = dense_of(lambda v: orc.dw(v, U, dims, M5), n, (2, 2, 2, 2, 4, 3))
    g5 = np.kron(np.eye(V), np.kron(np.diag([1, 1, -1, -1]), np.eye(3))).astype(complex)
    HT = g5 @ DW @ np.linalg.inv(2 * np.eye(n) + DW)
    w = z.zolotarev_omegas(Ls, 0.1, 1.0)
    eps = hermitian_function(HT, lambda lam: z.eps_of_omegas(lam, w))
    Dov = 0.5 * (1 + m) * np.eye(n) + 0.5 * (1 - m) * g5 @ eps
    assert np.allclose(K[:n, :n], Dov, atol=1e-11)
