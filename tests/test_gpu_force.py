"""GPU force dS/dU, dS/db5, dS/dc5 of S = phi^dag (M^dag M)^-1 phi: against the
FP64 oracle's force on a small lattice, by central finite differences at the
full 16^3 x 32 x 16 size, and through torch.autograd (gradcheck)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle
import paper_1206_5214_gb300 as mdwf
import synthetic as sy
from paper_1206_5214_gb300.autograd import mobius_action

pytestmark = pytest.mark.gpu


def su3_direction(shape, seed):
    """Random traceless anti-Hermitian omega per link, shape (..., 3, 3)."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(shape + (3, 3)) + 1j * rng.standard_normal(shape + (3, 3))
    h = 0.5 * (a - np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1) / 3.0
    return h - tr[..., None, None] * np.eye(3)


def expm_ah(w):
    lam, v = np.linalg.eigh(1j * w)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(-1j * lam), np.conj(v))


def gpu_force(dims, Ls, b5, c5, mf, U, phi, tol=1e-13, inner=mdwf.MDWF_F64, derivs=True):
    h = mdwf.mdwf_create(dims, Ls, 1.8, b5, c5, mf)
    try:
        mdwf.mdwf_load_gauge(h, torch.from_numpy(U).cuda())
        G = torch.empty(U.shape, dtype=torch.complex128, device="cuda") if derivs else None
        S, db5, dc5, st, info = mdwf.mdwf_force(h, G, torch.from_numpy(np.ascontiguousarray(phi)).cuda(), tol=tol,
                                                inner_prec=inner)
        return S, (G.cpu().numpy() if derivs else None), db5, dc5, st, info
    finally:
        mdwf.mdwf_destroy(h)


@pytest.mark.parametrize("b5,c5", [(1.5, 0.5), (1.0, 0.0)])
def test_force_matches_oracle(b5, c5):
    dims, Ls, mf = (4, 4, 2, 4), 8, 0.05
    U = sy.gauge_field(dims, 0.3, 1013)
    _, phi = oracle.split(sy.gaussian_field(dims, Ls, 2013), dims)
    p = oracle.Params(dims, Ls, 1.8, b5, c5, mf)
    S0, G0, db0, dc0, st0, _ = oracle.force(phi, U, p, tol=1e-14)
    assert st0 == 0
    S, G, db, dc, st, info = gpu_force(dims, Ls, b5, c5, mf, U, phi, tol=1e-13)
    assert st == 0
    assert S == pytest.approx(S0, rel=1e-11)
    assert np.abs(G - G0).max() <= 1e-9 * np.abs(G0).max()
    assert db == pytest.approx(db0, rel=1e-9)
    assert dc == pytest.approx(dc0, rel=1e-9, abs=1e-9 * abs(db0))


def test_force_mixed_precision_solve_matches_fp64():
    """The force with X from the mixed FP32/FP64 solve equals the FP64 one to the solve tolerance."""
    dims, Ls, mf = (4, 4, 4, 4), 8, 0.02
    U = sy.gauge_field(dims, 0.3, 1014)
    _, phi = oracle.split(sy.gaussian_field(dims, Ls, 2014), dims)
    S1, G1, db1, dc1, _, _ = gpu_force(dims, Ls, 1.5, 0.5, mf, U, phi, tol=1e-12, inner=mdwf.MDWF_F64)
    S2, G2, db2, dc2, _, info = gpu_force(dims, Ls, 1.5, 0.5, mf, U, phi, tol=1e-12, inner=mdwf.MDWF_F32)
    assert info.reliable_updates >= 1
    assert S2 == pytest.approx(S1, rel=1e-9)
    assert np.abs(G2 - G1).max() <= 1e-7 * np.abs(G1).max()
    assert db2 == pytest.approx(db1, rel=1e-7)


def test_force_finite_differences_full_16x16x16x32():
    """16^3 x 32, Ls = 16, b5 = 1.5, c5 = 0.5, mf = 0.02, eps = 0.2: central differences at h = 1e-6."""
    dims, Ls, b5, c5, mf = (16, 16, 16, 32), 16, 1.5, 0.5, 0.02
    U = sy.gauge_field(dims, 0.2, 1004)
    _, phi = oracle.split(sy.gaussian_field(dims, Ls, 2004), dims)
    inner = mdwf.MDWF_F32
    S, G, db, dc, st, info = gpu_force(dims, Ls, b5, c5, mf, U, phi, tol=1e-13, inner=inner)
    assert st == 0
    h = 1e-6
    w = su3_direction(U.shape[:-2], 17)
    Sp = gpu_force(dims, Ls, b5, c5, mf, expm_ah(h * w) @ U, phi, inner=inner, derivs=False)[0]
    Sm = gpu_force(dims, Ls, b5, c5, mf, expm_ah(-h * w) @ U, phi, inner=inner, derivs=False)[0]
    fd = (Sp - Sm) / (2 * h)
    an = float(np.sum(np.real(np.conj(G) * (w @ U))))
    assert an == pytest.approx(fd, rel=1e-5)
    fdb = (gpu_force(dims, Ls, b5 + h, c5, mf, U, phi, inner=inner, derivs=False)[0]
           - gpu_force(dims, Ls, b5 - h, c5, mf, U, phi, inner=inner, derivs=False)[0]) / (2 * h)
    fdc = (gpu_force(dims, Ls, b5, c5 + h, mf, U, phi, inner=inner, derivs=False)[0]
           - gpu_force(dims, Ls, b5, c5 - h, mf, U, phi, inner=inner, derivs=False)[0]) / (2 * h)
    assert db == pytest.approx(fdb, rel=1e-5)
    assert dc == pytest.approx(fdc, rel=1e-5, abs=1e-5 * abs(db))


def test_autograd_gradcheck_tiny():
    """torch.autograd.gradcheck of S(U, (b5, c5)) on a 2^4 lattice, Ls = 4 (complex U entries
    and the two Moebius parameters perturbed one at a time)."""
    dims, Ls = (2, 2, 2, 2), 4
    U = torch.from_numpy(sy.gauge_field(dims, 0.3, 1015)).cuda().requires_grad_(True)
    _, phi_np = oracle.split(sy.gaussian_field(dims, Ls, 2015), dims)
    phi = torch.from_numpy(phi_np).cuda()
    b5c5 = torch.tensor([1.5, 0.5], dtype=torch.float64, device="cuda", requires_grad=True)
    f = lambda u, bc: mobius_action(u, bc, phi, dims, Ls, 1.8, 0.1, 1e-13)
    assert torch.autograd.gradcheck(f, (U, b5c5), eps=1e-6, atol=1e-6, rtol=1e-5, fast_mode=True)


def test_autograd_backward_matches_force():
    dims, Ls = (4, 4, 2, 2), 4
    U = torch.from_numpy(sy.gauge_field(dims, 0.3, 1016)).cuda().requires_grad_(True)
    _, phi_np = oracle.split(sy.gaussian_field(dims, Ls, 2016), dims)
    phi = torch.from_numpy(phi_np).cuda()
    b5c5 = torch.tensor([1.5, 0.5], dtype=torch.float64, device="cuda", requires_grad=True)
    S = mobius_action(U, b5c5, phi, dims, Ls, 1.8, 0.05)
    S.backward()
    p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, 0.05)
    S0, G0, db0, dc0, _, _ = oracle.force(phi_np, U.detach().cpu().numpy(), p, tol=1e-14)
    assert float(S.detach()) == pytest.approx(S0, rel=1e-10)
    assert np.abs(U.grad.cpu().numpy() - G0).max() <= 1e-8 * np.abs(G0).max()
    assert b5c5.grad.cpu().numpy() == pytest.approx([db0, dc0], rel=1e-8)


def test_autograd_per_slice_and_mu_match_oracle_force():
    """mobius_action with per-slice b5(s), c5(s) (b5c5 of shape (2, Ls)) and mu = 0.3 on
    4x2x2x2, Ls = 4: S, dS/dU and the (2, Ls) coefficient gradient against the oracle's force
    with the same parameters (both solves to 1e-12)."""
    dims, Ls, mf, mu = (4, 2, 2, 2), 4, 0.05, 0.3
    prof = ([1.2, 1.9, 1.4, 2.3], [0.1, 0.8, 0.2, 1.0])
    U = torch.from_numpy(sy.gauge_field(dims, 0.3, 1017)).cuda().requires_grad_(True)
    _, phi_np = oracle.split(sy.gaussian_field(dims, Ls, 2017), dims)
    phi = torch.from_numpy(phi_np).cuda()
    bc = torch.tensor(prof, dtype=torch.float64, device="cuda", requires_grad=True)
    S = mobius_action(U, bc, phi, dims, Ls, 1.8, mf, 1e-12, mu=mu)
    S.backward()
    p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, mf, b5s=tuple(prof[0]), c5s=tuple(prof[1]), mu=mu)
    S0, G0, db0, dc0, st, _ = oracle.force(phi_np, U.detach().cpu().numpy(), p, tol=1e-12, maxiter=200000)
    assert st == 0
    assert float(S.detach()) == pytest.approx(S0, rel=1e-9)
    assert np.abs(U.grad.cpu().numpy() - G0).max() <= 1e-7 * np.abs(G0).max()
    g = bc.grad.cpu().numpy()
    assert g.shape == (2, Ls)
    ref = np.stack([db0, dc0])
    assert np.abs(g - ref).max() <= 1e-7 * np.abs(ref).max()
