"""Pins of the oracle's force beyond constant coefficients: per-slice b5(s), c5(s)
(Sec. 2.1, Eq. DWaction) and a chemical potential on the time links (Sec. 6.6).
Each derivative is checked against central differences of the oracle's own
action S = phi^dag (M^dag M)^-1 phi, formed exactly from its M^dag M as a dense
matrix, and the per-slice derivatives of a constant profile against the
constant-coefficient ones. The force's CG runs to 1e-12 (at mu != 0 FP64 CG on
M^dag M does not reach 1e-14)."""
import numpy as np
import pytest

import synthetic as sy
from _pins import dense_of


@pytest.fixture(scope="module")
def orc(oracle_lib):
    return oracle_lib


def su3_direction(shape, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(shape + (3, 3)) + 1j * rng.standard_normal(shape + (3, 3))
    h = 0.5 * (a - np.conj(np.swapaxes(a, -1, -2)))
    return h - np.trace(h, axis1=-2, axis2=-1)[..., None, None] / 3.0 * np.eye(3)


def expm_ah(w):
    lam, v = np.linalg.eigh(1j * w)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(-1j * lam), np.conj(v))


def action(orc, phi, U, p):
    """S = phi^dag (M^dag M)^-1 phi from the oracle's M^dag M as a dense matrix (exact)."""
    A = dense_of(lambda v: orc.mdagm(v, U, p), phi.size, phi.shape)
    return float(np.real(np.vdot(phi.reshape(-1), np.linalg.solve(A, phi.reshape(-1)))))


PROF = ([1.2, 1.9, 1.4, 2.3], [0.1, 0.8, 0.2, 1.0])
H = 1e-5


@pytest.mark.parametrize("mu", [0.0, 0.3], ids=["mu0", "mu0.3"])
def test_per_slice_force_against_differences(orc, mu):
    dims, Ls, mf = (4, 2, 2, 2), 4, 0.05
    U = sy.gauge_field(dims, 0.3, 61)
    _, phi = orc.split(sy.gaussian_field(dims, Ls, 62), dims)
    p = orc.Params(dims, Ls, 1.8, 1.5, 0.5, mf, b5s=tuple(PROF[0]), c5s=tuple(PROF[1]), mu=mu)
    S, G, db, dc, st, _ = orc.force(phi, U, p, tol=1e-12, maxiter=200000)
    assert st == 0 and db.shape == (Ls,) and dc.shape == (Ls,)
    assert S == pytest.approx(action(orc, phi, U, p), rel=1e-10)
    w = su3_direction(U.shape[:-2], 63)
    fd = (action(orc, phi, expm_ah(H * w) @ U, p) - action(orc, phi, expm_ah(-H * w) @ U, p)) / (2 * H)
    assert float(np.sum(np.real(np.conj(G) * (w @ U)))) == pytest.approx(fd, rel=1e-6)
    for name, got in (("b5s", db), ("c5s", dc)):
        for s in range(Ls):
            up, dn = list(getattr(p, name)), list(getattr(p, name))
            up[s] += H
            dn[s] -= H
            fd = (action(orc, phi, U, p.with_(**{name: tuple(up)})) -
                  action(orc, phi, U, p.with_(**{name: tuple(dn)}))) / (2 * H)
            assert abs(got[s] - fd) <= 1e-6 * np.abs(got).max(), (name, s, got[s], fd)


def test_constant_profile_per_slice_sums(orc):
    dims, Ls, mf = (4, 2, 2, 2), 6, 0.05
    U = sy.gauge_field(dims, 0.3, 64)
    _, phi = orc.split(sy.gaussian_field(dims, Ls, 65), dims)
    p0 = orc.Params(dims, Ls, 1.8, 1.5, 0.5, mf)
    p1 = p0.with_(b5s=(1.5,) * Ls, c5s=(0.5,) * Ls)
    S0, G0, db0, dc0, _, _ = orc.force(phi, U, p0, tol=1e-14, maxiter=200000)
    S1, G1, db1, dc1, _, _ = orc.force(phi, U, p1, tol=1e-14, maxiter=200000)
    assert S1 == pytest.approx(S0, rel=1e-11)
    assert np.abs(G1 - G0).max() <= 1e-10 * np.abs(G0).max()
    assert float(np.sum(db1)) == pytest.approx(db0, rel=1e-10)
    assert float(np.sum(dc1)) == pytest.approx(dc0, rel=1e-10)


def test_chemical_potential_force_against_differences(orc):
    dims, Ls, mf, mu = (4, 2, 2, 2), 4, 0.05, 0.3
    U = sy.gauge_field(dims, 0.3, 66)
    _, phi = orc.split(sy.gaussian_field(dims, Ls, 67), dims)
    p = orc.Params(dims, Ls, 1.8, 1.5, 0.5, mf, mu=mu)
    S, G, db5, dc5, st, _ = orc.force(phi, U, p, tol=1e-12, maxiter=200000)
    assert st == 0
    assert S == pytest.approx(action(orc, phi, U, p), rel=1e-10)
    w = su3_direction(U.shape[:-2], 68)
    fd = (action(orc, phi, expm_ah(H * w) @ U, p) - action(orc, phi, expm_ah(-H * w) @ U, p)) / (2 * H)
    assert float(np.sum(np.real(np.conj(G) * (w @ U)))) == pytest.approx(fd, rel=1e-6)
    for name, got in (("b5", db5), ("c5", dc5)):
        v = getattr(p, name)
        fd = (action(orc, phi, U, p.with_(**{name: v + H})) - action(orc, phi, U, p.with_(**{name: v - H}))) / (2 * H)
        assert got == pytest.approx(fd, rel=1e-6), name
