"""Per-slice Moebius coefficients b5(s), c5(s) for the Zolotarev form (Sec. 4.3).

With b5(s) - c5(s) = a5 fixed, each slice's kernel is a multiple of one
Shamir-type kernel, H_s = omega_s H_T with H_T = gamma5 a5 D_W / (2 + a5 D_W),
and the transfer matrices of App. A commute. The 4d operator then carries

    eps(x) = [prod_s (1 + omega_s x) - prod_s (1 - omega_s x)]
             / [prod_s (1 + omega_s x) + prod_s (1 - omega_s x)]

of the eigenvalues x of H_T: constant omega_s = alpha gives the polar form
eps_Ls (Eq. ApproxEPS); the omega_s below make eps the best uniform rational
approximation of sign(x) on lam_min <= |x| <= lam_max (Zolotarev's solution,
as used for domain-wall fermions by Chiu). Writing P(x) = prod_s (1 + omega_s x),
eps = x O(x^2) / E(x^2) with E, x O the even and odd parts of P. The optimal
odd rational function of that type on [k, 1], k = lam_min / lam_max, is

    r(x) = D x prod_{j = 2, 4, .., N-2} (x^2 + c_j) / prod_{j = 1, 3, .., N-1} (x^2 + c_j),
    c_j = k^2 sn^2(j K' / N; k') / cn^2(j K' / N; k'),  k' = sqrt(1 - k^2), K' = K(k'),

(N = Ls even), with D fixed by making the error 1 - r equioscillate about 0.
Then P(x) = E(x^2) + x O(x^2) is the polynomial prod_odd (x^2 + c_j) + D x prod_even (x^2 + c_j),
whose roots are -1 / omega_s. Host-side set-up only: the GPU path receives the
resulting b5(s), c5(s) through mdwf_set_s_coefficients.
"""
from __future__ import annotations

import numpy as np
from scipy import special

__all__ = ["zolotarev_omegas", "eps_of_omegas", "coefficients_from_omegas", "zolotarev_coefficients",
           "polar_coefficients"]


def _c_coefficients(N: int, k: float) -> np.ndarray:
    kp2 = 1.0 - k * k                      # k'^2, scipy's parameter m
    Kp = special.ellipk(kp2)
    j = np.arange(1, N)
    sn, cn, _, _ = special.ellipj(j * Kp / N, kp2)
    return k * k * sn ** 2 / cn ** 2       # c_1 .. c_{N-1}


def _unscaled(x: np.ndarray, c: np.ndarray) -> np.ndarray:
    num = np.ones_like(x)
    den = np.ones_like(x)
    for j, cj in enumerate(c, start=1):
        if j % 2 == 0:
            num = num * (x * x + cj)
        else:
            den = den * (x * x + cj)
    return x * num / den


def zolotarev_omegas(Ls: int, lam_min: float, lam_max: float, grid: int = 20001) -> np.ndarray:
    """The Ls values omega_s (ascending) of the optimal eps on lam_min <= |x| <= lam_max."""
    if Ls < 2 or Ls % 2:
        raise ValueError("Ls must be even and >= 2")
    if not 0 < lam_min < lam_max:
        raise ValueError("need 0 < lam_min < lam_max")
    k = lam_min / lam_max
    c = _c_coefficients(Ls, k)
    # D from the extreme values of the unscaled function on a log-spaced grid of [k, 1]
    x = np.geomspace(k, 1.0, grid)
    r = _unscaled(x, c)
    D = 2.0 / (r.max() + r.min())
    # P(x) = prod_odd (x^2 + c_j) + D x prod_even (x^2 + c_j)
    even = np.poly1d([1.0])
    odd = np.poly1d([1.0])
    for j, cj in enumerate(c, start=1):
        if j % 2 == 0:
            even = even * np.poly1d([1.0, 0.0, cj])
        else:
            odd = odd * np.poly1d([1.0, 0.0, cj])
    P = odd + np.poly1d([float(D), 0.0]) * even
    roots = P.roots
    if np.max(np.abs(roots.imag)) > 1e-8 * np.max(np.abs(roots)) or np.any(roots.real >= 0):
        raise ArithmeticError("Zolotarev polynomial without the expected negative real roots")
    omegas = np.sort(-1.0 / roots.real)      # in units of 1 / lam_max
    return omegas / lam_max


def eps_of_omegas(x, omegas) -> np.ndarray:
    """eps(x) = [prod(1 + w x) - prod(1 - w x)] / [prod(1 + w x) + prod(1 - w x)]."""
    x = np.asarray(x, dtype=np.float64)
    p = np.ones_like(x)
    q = np.ones_like(x)
    for w in omegas:
        p = p * (1.0 + w * x)
        q = q * (1.0 - w * x)
    return (p - q) / (p + q)


def coefficients_from_omegas(omegas, a5: float = 1.0):
    """b5(s), c5(s) with b5 - c5 = a5 and b5 + c5 = a5 omega_s (H_s = omega_s H_T)."""
    w = np.asarray(omegas, dtype=np.float64)
    return list(0.5 * a5 * (w + 1.0)), list(0.5 * a5 * (w - 1.0))


def zolotarev_coefficients(Ls: int, lam_min: float, lam_max: float, a5: float = 1.0):
    """(b5s, c5s) of the Zolotarev form for H_T = gamma5 a5 D_W / (2 + a5 D_W) with
    spectrum magnitudes in [lam_min, lam_max]."""
    return coefficients_from_omegas(zolotarev_omegas(Ls, lam_min, lam_max), a5)


def polar_coefficients(Ls: int, alpha: float, a5: float = 1.0):
    """Constant b5, c5 of the polar form with scale alpha (b5 + c5 = alpha a5)."""
    return coefficients_from_omegas(np.full(Ls, float(alpha)), a5)
