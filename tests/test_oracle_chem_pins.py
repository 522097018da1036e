"""Pins of the oracle's chemical potential (Sec. 6.6): the time links carry
e^{+mu} forward and e^{-mu} backward.

* U = 1: D_W(mu) is the plane-wave form with p_4 -> p_4 - i mu;
* D_W(mu)^dag = gamma5 D_W(-mu) gamma5 (gamma5-Hermiticity is lost for mu != 0);
* random links: the first column of P^dag D_DW(1)^-1 D_DW(m) P is
  (1+m)/2 + (1-m)/2 gamma5 [(1+A)^Ls - (1-A)^Ls] [(1+A)^Ls + (1-A)^Ls]^-1 with the
  non-Hermitian kernel A = gamma5 (b5+c5) D_W(mu) (2 + (b5-c5) D_W(mu))^-1
  (the finite-Ls form of Sec. 6.6), and the adjoint of D_DW is the conjugate transpose.
"""
import numpy as np
import pytest

import synthetic as sy
from _pins import dense_of, free_wilson_momentum, momenta, momentum_blocks_5d


@pytest.fixture(scope="module")
def orc(oracle_lib):
    return oracle_lib


def test_free_field_shifted_momentum(orc):
    dims, M5, mu = (4, 4, 2, 4), 1.8, 0.37
    U = sy.unit_gauge(dims)
    blocks = momentum_blocks_5d(lambda s5: orc.dw(s5[0], U, dims, M5, mu=mu)[None], dims, 1)
    for k, p in momenta(dims):
        ref = free_wilson_momentum((p[0], p[1], p[2], p[3] - 1j * mu), M5)
        assert np.allclose(blocks[k], ref, atol=1e-13)
    # the adjoint is the conjugate transpose at every momentum
    blocks_d = momentum_blocks_5d(lambda s5: orc.dw(s5[0], U, dims, M5, dagger=True, mu=mu)[None], dims, 1)
    for k, p in momenta(dims):
        ref = free_wilson_momentum((p[0], p[1], p[2], p[3] - 1j * mu), M5)
        assert np.allclose(blocks_d[k], ref.conj().T, atol=1e-13)


def _dense_dw(orc, U, dims, M5, mu, dagger=False):
    x, y, z, t = dims
    shape = (t, z, y, x, 4, 3)
    return dense_of(lambda v: orc.dw(v, U, dims, M5, dagger=dagger, mu=mu), int(np.prod(shape)), shape)


def test_gamma5_relation(orc):
    dims, M5, mu = (4, 2, 2, 2), 1.8, 0.25
    U = sy.gauge_field(dims, 0.3, 31)
    V = int(np.prod(dims))
    g5 = np.kron(np.eye(V), np.kron(np.diag([1, 1, -1, -1]), np.eye(3))).astype(complex)
    Dp = _dense_dw(orc, U, dims, M5, mu)
    Dm = _dense_dw(orc, U, dims, M5, -mu)
    assert np.allclose(_dense_dw(orc, U, dims, M5, mu, dagger=True), Dp.conj().T, atol=1e-14)
    assert np.allclose(Dp.conj().T, g5 @ Dm @ g5, atol=1e-14)
    assert not np.allclose(Dp.conj().T, g5 @ Dp @ g5, atol=1e-6)


@pytest.mark.parametrize("b5,c5", [(1.5, 0.5), (1.0, 0.0)])
def test_nonhermitian_kernel_overlap_identity(orc, b5, c5):
    dims, Ls, M5, m, mu = (2, 2, 2, 2), 4, 1.8, 0.1, 0.3
    U = sy.gauge_field(dims, 0.3, 32)
    V = 16
    n = 12 * V
    p = orc.Params(dims, Ls, M5, b5, c5, m, mu=mu)
    shape = (Ls, 2, 2, 2, 2, 4, 3)
    Dm = dense_of(lambda v: orc.ddw(v, U, p), Ls * n, shape)
    D1 = dense_of(lambda v: orc.ddw(v, U, p.with_(mf=1.0)), Ls * n, shape)
    assert np.allclose(dense_of(lambda v: orc.ddw(v, U, p, dagger=True), Ls * n, shape), Dm.conj().T, atol=1e-13)
    Pp = np.kron(np.eye(V), np.kron(np.diag([1, 1, 0, 0]), np.eye(3)))
    Pm = np.kron(np.eye(V), np.kron(np.diag([0, 0, 1, 1]), np.eye(3)))
    P = np.zeros((Ls * n, Ls * n), complex)
    for s in range(Ls):
        P[s * n:(s + 1) * n, s * n:(s + 1) * n] += Pm
        sp = (s + 1) % Ls
        P[s * n:(s + 1) * n, sp * n:(sp + 1) * n] += Pp
    K = P.conj().T @ np.linalg.solve(D1, Dm) @ P
    DW = _dense_dw(orc, U, dims, M5, mu)
    g5 = np.kron(np.eye(V), np.kron(np.diag([1, 1, -1, -1]), np.eye(3))).astype(complex)
    one = np.eye(n)
    A = g5 @ ((b5 + c5) * DW) @ np.linalg.inv(2 * one + (b5 - c5) * DW)
    Pl = np.linalg.matrix_power(one + A, Ls)
    Mi = np.linalg.matrix_power(one - A, Ls)
    eps = (Pl - Mi) @ np.linalg.inv(Pl + Mi)
    Dov = 0.5 * (1 + m) * one + 0.5 * (1 - m) * g5 @ eps
    assert np.allclose(K[:n, :n], Dov, atol=1e-11)
    assert np.allclose(K[:, n:], np.eye(Ls * n)[:, n:], atol=1e-11)


def test_per_slice_profile_with_chemical_potential(orc):
    """Per-slice b5(s), c5(s) together with mu = 0.3 (2^4, Ls = 4): the first column of
    P^dag D(1)^-1 D(m) P is (1+m)/2 + (1-m)/2 gamma5 (T^-Ls - 1)(T^-Ls + 1)^-1 with
    T^-Ls = T_1^-1 ... T_Ls^-1, T_s^-1 = (1 + H_s)(1 - H_s)^-1 and the non-Hermitian
    H_s = gamma5 (b5(s) + c5(s)) D_W(mu) (2 + (b5(s) - c5(s)) D_W(mu))^-1 (App. A with the
    links of Sec. 6.6); the other columns are the identity and D^dag is the conjugate transpose."""
    dims, Ls, M5, m, mu = (2, 2, 2, 2), 4, 1.8, 0.1, 0.3
    b5s, c5s = (1.2, 1.9, 1.4, 2.3), (0.1, 0.8, 0.2, 1.0)
    U = sy.gauge_field(dims, 0.3, 33)
    V = 16
    n = 12 * V
    p = orc.Params(dims, Ls, M5, 1.5, 0.5, m, b5s=b5s, c5s=c5s, mu=mu)
    shape = (Ls, 2, 2, 2, 2, 4, 3)
    Dm = dense_of(lambda v: orc.ddw(v, U, p), Ls * n, shape)
    D1 = dense_of(lambda v: orc.ddw(v, U, p.with_(mf=1.0)), Ls * n, shape)
    assert np.allclose(dense_of(lambda v: orc.ddw(v, U, p, dagger=True), Ls * n, shape), Dm.conj().T, atol=1e-13)
    Pp = np.kron(np.eye(V), np.kron(np.diag([1, 1, 0, 0]), np.eye(3)))
    Pm = np.kron(np.eye(V), np.kron(np.diag([0, 0, 1, 1]), np.eye(3)))
    P = np.zeros((Ls * n, Ls * n), complex)
    for s in range(Ls):
        P[s * n:(s + 1) * n, s * n:(s + 1) * n] += Pm
        sp = (s + 1) % Ls
        P[s * n:(s + 1) * n, sp * n:(sp + 1) * n] += Pp
    K = P.conj().T @ np.linalg.solve(D1, Dm) @ P
    DW = _dense_dw(orc, U, dims, M5, mu)
    g5 = np.kron(np.eye(V), np.kron(np.diag([1, 1, -1, -1]), np.eye(3))).astype(complex)
    one = np.eye(n)
    Tinv = one.astype(complex)
    for b, c in zip(b5s, c5s):
        Hs = g5 @ ((b + c) * DW) @ np.linalg.inv(2 * one + (b - c) * DW)
        Tinv = Tinv @ ((one + Hs) @ np.linalg.inv(one - Hs))
    eps = (Tinv - one) @ np.linalg.inv(Tinv + one)
    Dov = 0.5 * (1 + m) * one + 0.5 * (1 - m) * g5 @ eps
    assert np.allclose(K[:n, :n], Dov, atol=1e-11)
    assert np.allclose(K[:, n:], np.eye(Ls * n)[:, n:], atol=1e-11)
    # and the same identity fails if the links carry no mu (the pin sees the phases)
    DW0 = _dense_dw(orc, U, dims, M5, 0.0)
    T0 = one.astype(complex)
    for b, c in zip(b5s, c5s):
        Hs = g5 @ ((b + c) * DW0) @ np.linalg.inv(2 * one + (b - c) * DW0)
        T0 = T0 @ ((one + Hs) @ np.linalg.inv(one - Hs))
    Dov0 = 0.5 * (1 + m) * one + 0.5 * (1 - m) * g5 @ ((T0 - one) @ np.linalg.inv(T0 + one))
    assert not np.allclose(K[:n, :n], Dov0, atol=1e-6)
