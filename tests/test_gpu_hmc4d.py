"""The wall-pseudofermion action of Sec. 2.4 on the GPU,
S = |D(1)^dag D(m)^-dag P phi|^2, and its link force (two inversions): S against
the oracle (its adjoint solve is plain CG on D D^dag, not the red/black route of
the GPU), and dS/dU against central differences of S along exp(h omega) U, with
the oracle's S and with the GPU's own, for constant and per-slice coefficients."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle
import paper_1206_5214_gb300 as mdwf
import synthetic as sy

pytestmark = pytest.mark.gpu


def su3_direction(shape, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(shape + (3, 3)) + 1j * rng.standard_normal(shape + (3, 3))
    h = 0.5 * (a - np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1) / 3.0
    return h - tr[..., None, None] * np.eye(3)


def expm_ah(w):
    lam, v = np.linalg.eigh(1j * w)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(-1j * lam), np.conj(v))


def oracle_action(phi, U, p):
    Ls = p.Ls
    tilde = np.zeros((Ls,) + phi.shape, complex)
    tilde[0] = phi
    b = np.empty_like(tilde)  # P phi~: P- phi on s = 0, P+ phi on s = Ls - 1
    b[:] = 0
    b[0, ..., 2:, :] = phi[..., 2:, :]
    b[Ls - 1, ..., :2, :] = phi[..., :2, :]
    chi, st, _, rel = oracle.solve_dag(b, U, p, tol=1e-14, maxiter=100000)
    assert st == 0, rel
    eta = oracle.ddw(chi, U, p.with_(mf=1.0), dagger=True)
    return float(np.vdot(eta, eta).real)


def gpu_action(dims, Ls, b5, c5, mf, U, phi, prof=None, derivs=True):
    h = mdwf.mdwf_create(dims, Ls, 1.8, b5, c5, mf)
    try:
        mdwf.mdwf_load_gauge(h, torch.from_numpy(np.ascontiguousarray(U)).cuda())
        if prof is not None:
            mdwf.mdwf_set_s_coefficients(h, *prof)
        G = torch.empty(U.shape, dtype=torch.complex128, device="cuda") if derivs else None
        S, st, info = mdwf.mdwf_force4d(h, G, torch.from_numpy(phi).cuda(), tol=1e-13)
        return S, (G.cpu().numpy() if derivs else None), st, info
    finally:
        mdwf.mdwf_destroy(h)


PROF4 = ([1.2, 1.9, 1.4, 2.3], [0.1, 0.8, 0.2, 1.0])


@pytest.mark.parametrize("per_slice", [False, True], ids=["constant", "per-slice"])
def test_action_and_force_against_oracle(per_slice):
    """4x4x2x2, Ls = 4: S equals the oracle's; dS/dU matches central differences
    of the oracle's S along a random su(3) direction."""
    dims, Ls, mf = (4, 4, 2, 2), 4, 0.05
    U = sy.gauge_field(dims, 0.3, 1071)
    phi = sy.gaussian_field(dims, 1, 2071)[0]
    prof = PROF4 if per_slice else None
    p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, mf)
    if prof:
        p = p.with_(b5s=tuple(prof[0]), c5s=tuple(prof[1]))
    S0 = oracle_action(phi, U, p)
    S, G, st, info = gpu_action(dims, Ls, 1.5, 0.5, mf, U, phi, prof)
    assert st == 0
    assert S == pytest.approx(S0, rel=1e-10)
    w = su3_direction(U.shape[:-2], 71)
    h = 1e-5
    fd = (oracle_action(phi, expm_ah(h * w) @ U, p) - oracle_action(phi, expm_ah(-h * w) @ U, p)) / (2 * h)
    an = float(np.sum(np.real(np.conj(G) * (w @ U))))
    assert an == pytest.approx(fd, rel=1e-6)


def test_force_finite_differences_4x4x4x4_Ls8():
    """4^4, Ls = 8, Moebius: GPU dS/dU against GPU central differences at h = 1e-5."""
    dims, Ls, mf = (4, 4, 4, 4), 8, 0.02
    U = sy.gauge_field(dims, 0.3, 1072)
    phi = sy.gaussian_field(dims, 1, 2072)[0]
    S, G, st, info = gpu_action(dims, Ls, 1.5, 0.5, mf, U, phi)
    assert st == 0 and info.true_res <= 1e-12
    w = su3_direction(U.shape[:-2], 72)
    h = 1e-5
    Sp = gpu_action(dims, Ls, 1.5, 0.5, mf, expm_ah(h * w) @ U, phi, derivs=False)[0]
    Sm = gpu_action(dims, Ls, 1.5, 0.5, mf, expm_ah(-h * w) @ U, phi, derivs=False)[0]
    an = float(np.sum(np.real(np.conj(G) * (w @ U))))
    assert an == pytest.approx((Sp - Sm) / (2 * h), rel=1e-5)
