"""Independent helpers for the oracle pins: dense matrices, free-field momentum
blocks, the polar sign function and the effective overlap operator.

Nothing here reuses the oracle's arithmetic; the oracle is only *applied* to
unit vectors to read off its matrix.
"""
from __future__ import annotations

import numpy as np


def dense_of(apply, n: int, shape) -> np.ndarray:
    """Dense matrix of a linear map given as ``apply(array of shape) -> array``."""
    cols = []
    e = np.zeros(n, dtype=np.complex128)
    for k in range(n):
        e[:] = 0
        e[k] = 1.0
        cols.append(np.asarray(apply(e.reshape(shape))).reshape(-1))
    return np.stack(cols, axis=1)


def eps_polar(lam, Ls: int):
    """Polar approximation of the sign function, Eq. (ApproxEPS)."""
    lam = np.asarray(lam, dtype=np.float64)
    a, b = (1.0 + lam) ** Ls, (1.0 - lam) ** Ls
    return (a - b) / (a + b)


def hermitian_function(H: np.ndarray, f) -> np.ndarray:
    w, v = np.linalg.eigh(0.5 * (H + H.conj().T))
    return (v * f(w)) @ v.conj().T


def pauli_gammas():
    """Chiral basis built directly from its definition: g_mu = [[0, A], [A^dag, 0]],
    A_k = -i sigma_k (k = 1, 2, 3), A_4 = 1."""
    s = [np.array([[0, 1], [1, 0]], complex), np.array([[0, -1j], [1j, 0]]),
         np.array([[1, 0], [0, -1]], complex)]
    A = [-1j * s[0], -1j * s[1], -1j * s[2], np.eye(2, dtype=complex)]
    g = []
    for a in A:
        m = np.zeros((4, 4), complex)
        m[:2, 2:] = a
        m[2:, :2] = a.conj().T
        g.append(m)
    return g


def wall_permutation(Ls: int) -> np.ndarray:
    """The permutation of Sec. 2.2 / Eq. (Pmatrix): P_{ss'} = delta_{ss'} P- + delta_{s',s+1 mod Ls} P+,
    as a (4 Ls) x (4 Ls) matrix in the [s][spin] ordering (colour left out)."""
    Pp = np.diag([1, 1, 0, 0]).astype(complex)
    Pm = np.diag([0, 0, 1, 1]).astype(complex)
    P = np.zeros((4 * Ls, 4 * Ls), complex)
    for s in range(Ls):
        P[4 * s:4 * s + 4, 4 * s:4 * s + 4] += Pm
        sp = (s + 1) % Ls
        P[4 * s:4 * s + 4, 4 * sp:4 * sp + 4] += Pp
    return P


def free_wilson_momentum(p, M5: float) -> np.ndarray:
    """Plane-wave form of D_W at U = 1: M5_f + sum(1 - cos p) + i sum gamma sin p, M5_f = -M5."""
    g = pauli_gammas()
    d = (-M5 + sum(1.0 - np.cos(pm) for pm in p)) * np.eye(4, dtype=complex)
    for mu in range(4):
        d = d + 1j * np.sin(p[mu]) * g[mu]
    return d


def momentum_blocks_5d(apply_full, dims, Ls: int) -> np.ndarray:
    """For a translation-invariant, colour-diagonal 5d operator (U = 1), the
    (4 Ls) x (4 Ls) block at every momentum. Returns array (T, Z, Y, X, 4Ls, 4Ls)
    indexed by the FFT momentum k (p_mu = 2 pi k_mu / L_mu)."""
    x, y, z, t = dims
    out = np.zeros((t, z, y, x, 4 * Ls, 4 * Ls), complex)
    for s0 in range(Ls):
        for a0 in range(4):
            src = np.zeros((Ls, t, z, y, x, 4, 3), complex)
            src[s0, 0, 0, 0, 0, a0, 0] = 1.0
            r = apply_full(src)[..., 0]                  # colour 0 only (U = 1)
            rk = np.fft.fftn(r, axes=(1, 2, 3, 4))        # (Ls, T, Z, Y, X, 4)
            col = np.moveaxis(rk, 0, -2).reshape(t, z, y, x, 4 * Ls)
            out[..., :, 4 * s0 + a0] = col
    return out


def momenta(dims):
    x, y, z, t = dims
    for kt in range(t):
        for kz in range(z):
            for ky in range(y):
                for kx in range(x):
                    p = (2 * np.pi * kx / x, 2 * np.pi * ky / y, 2 * np.pi * kz / z, 2 * np.pi * kt / t)
                    yield (kt, kz, ky, kx), p


def overlap_operator(DW: np.ndarray, g5: np.ndarray, Ls: int, b5: float, c5: float, m: float) -> np.ndarray:
    """D_ov(m) = (1+m)/2 + (1-m)/2 g5 eps_Ls(H_M), H_M = g5 (b5+c5) D_W (2 + (b5-c5) D_W)^-1
    (Eq. GWapprox with the Moebius kernel of Eq. Moebius)."""
    n = DW.shape[0]
    one = np.eye(n, dtype=complex)
    HM = g5 @ ((b5 + c5) * DW) @ np.linalg.inv(2 * one + (b5 - c5) * DW)
    eps = hermitian_function(HM, lambda w: eps_polar(w, Ls))
    return 0.5 * (1 + m) * one + 0.5 * (1 - m) * g5 @ eps


def gauge_rotate(U: np.ndarray, Om: np.ndarray) -> np.ndarray:
    """U^Omega_mu(x) = Omega(x) U_mu(x) Omega(x + mu)^dag; arrays (T,Z,Y,X,4,3,3), (T,Z,Y,X,3,3)."""
    out = np.empty_like(U)
    axes = {0: 3, 1: 2, 2: 1, 3: 0}                      # mu -> array axis of (T, Z, Y, X)
    for mu in range(4):
        Om_fw = np.roll(Om, -1, axis=axes[mu])           # Omega(x + mu)
        out[..., mu, :, :] = Om @ U[..., mu, :, :] @ np.conj(np.swapaxes(Om_fw, -1, -2))
    return out


def rotate_field(psi: np.ndarray, Om: np.ndarray) -> np.ndarray:
    """(Omega psi)(x) on a field (..., T, Z, Y, X, 4, 3)."""
    return np.einsum("tzyxab,...tzyxsb->...tzyxsa", Om, psi)
