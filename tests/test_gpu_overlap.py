"""The full operator D_DW(m), the effective overlap operator of Sec. 2.2 and the
bulk reconstruction of Sec. 2.3 on the GPU, against the FP64 oracle:

* mdwf_apply_full against the oracle's row-by-row D_DW (and its adjoint),
  constant and per-slice coefficients, 1e-12 of max |oracle|;
* mdwf_overlap_apply against D_ov(m) = (1+m)/2 + (1-m)/2 gamma5 eps_Ls(H_M)
  built densely from the oracle's D_W on a 2^4 lattice (random links), and
  against the oracle's own Pauli-Villars route on 4^4;
* mdwf_pv_reconstruct: from psi = D_ov^-1 b (the first slice of the oracle's
  direct 5d solve of D_DW(m) X = D_DW(1) P B), the reconstruction reproduces
  every slice of Psi = P^dag X (Sec. 2.3).
The Pauli-Villars solves run to 1e-12, so those comparisons use 1e-9.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle
import paper_1206_5214_gb300 as mdwf
import synthetic as sy
from _pins import dense_of, overlap_operator

pytestmark = pytest.mark.gpu


def wall_P(x):
    """(P x)_s = P- x_s + P+ x_{s+1}; x: (Ls, T, Z, Y, X, 4, 3)."""
    out = np.empty_like(x)
    out[..., 2:, :] = x[..., 2:, :]
    out[..., :2, :] = np.roll(x[..., :2, :], -1, axis=0)
    return out


def wall_Pdag(x):
    """(P^dag x)_s = P- x_s + P+ x_{s-1}."""
    out = np.empty_like(x)
    out[..., 2:, :] = x[..., 2:, :]
    out[..., :2, :] = np.roll(x[..., :2, :], 1, axis=0)
    return out


def ctx(dims, Ls, b5, c5, mf, U, prof=None):
    h = mdwf.mdwf_create(dims, Ls, 1.8, b5, c5, mf)
    mdwf.mdwf_load_gauge(h, torch.from_numpy(U).cuda())
    if prof is not None:
        mdwf.mdwf_set_s_coefficients(h, *prof)
    return h


@pytest.mark.parametrize("per_slice", [False, True], ids=["constant", "per-slice"])
@pytest.mark.parametrize("dagger", [False, True])
def test_apply_full_matches_oracle(per_slice, dagger):
    dims, Ls, mf = (4, 4, 2, 4), 6, 0.03
    U = sy.gauge_field(dims, 0.3, 1051)
    x = sy.gaussian_field(dims, Ls, 2051)
    prof = ([1.2, 1.9, 1.4, 2.3, 1.1, 1.7], [0.1, 0.8, 0.2, 1.0, 0.3, 0.4]) if per_slice else None
    p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, mf)
    if prof:
        p = p.with_(b5s=tuple(prof[0]), c5s=tuple(prof[1]))
    ref = oracle.ddw(x, U, p, dagger=dagger)
    h = ctx(dims, Ls, 1.5, 0.5, mf, U, prof)
    try:
        out = torch.empty(x.shape, dtype=torch.complex128, device="cuda")
        mdwf.mdwf_apply_full(h, out, torch.from_numpy(x).cuda(), dagger=dagger)
        got = out.cpu().numpy()
        # host buffers give the same result
        outh = np.empty_like(x)
        mdwf.mdwf_apply_full(h, outh, x, dagger=dagger)
    finally:
        mdwf.mdwf_destroy(h)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.array_equal(got, outh)


@pytest.mark.parametrize("b5,c5", [(1.5, 0.5), (1.0, 0.0)])
def test_overlap_apply_matches_dense_overlap(b5, c5):
    """2^4, Ls = 4, random links: D_ov(m) psi against the dense polar formula."""
    dims, Ls, M5, m = (2, 2, 2, 2), 4, 1.8, 0.1
    U = sy.gauge_field(dims, 0.3, 1052)
    V = 16
    DW = dense_of(lambda v: oracle.dw(v, U, dims, M5), 12 * V, (2, 2, 2, 2, 4, 3))
    g5 = np.kron(np.eye(V), np.kron(np.diag([1, 1, -1, -1]), np.eye(3))).astype(complex)
    Dov = overlap_operator(DW, g5, Ls, b5, c5, m)
    rng = np.random.default_rng(7)
    psi = (rng.standard_normal((2, 2, 2, 2, 2, 4, 3)) + 1j * rng.standard_normal((2, 2, 2, 2, 2, 4, 3)))
    h = ctx(dims, Ls, b5, c5, m, U)
    try:
        out = np.empty_like(psi)
        st, info = mdwf.mdwf_overlap_apply(h, out, psi, nrhs=2, tol=1e-13)
    finally:
        mdwf.mdwf_destroy(h)
    assert st == 0
    for r in range(2):
        ref = (Dov @ psi[r].reshape(-1)).reshape(psi[r].shape)
        assert np.abs(out[r] - ref).max() <= 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("inner,tol,bound", [(mdwf.MDWF_F64, 1e-12, 1e-9), (mdwf.MDWF_F32, 1e-10, 1e-8),
                                             (mdwf.MDWF_F16N, 1e-10, 1e-8)], ids=["f64", "mixed-f32", "mixed-f16n"])
def test_overlap_apply_matches_oracle_route(inner, tol, bound):
    """4^4, Ls = 8, Moebius: [P^dag D(1)^-1 D(m) P psi~]_1 with the oracle's solve; the
    Pauli-Villars solve in FP64, or mixed with FP32 or FP16+norm inner iterations."""
    dims, Ls, mf = (4, 4, 4, 4), 8, 0.02
    U = sy.gauge_field(dims, 0.3, 1053)
    psi = sy.gaussian_field(dims, 1, 2053)[0]
    p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, mf)
    tilde = np.zeros((Ls,) + psi.shape, complex)
    tilde[0] = psi
    y = oracle.ddw(wall_P(tilde), U, p)
    x, st0, _, _ = oracle.solve(y, U, p.with_(mf=1.0), tol=1e-13)
    assert st0 == 0
    ref = wall_Pdag(x)[0]
    h = ctx(dims, Ls, 1.5, 0.5, mf, U)
    try:
        out = torch.empty(psi.shape, dtype=torch.complex128, device="cuda")
        st, info = mdwf.mdwf_overlap_apply(h, out, torch.from_numpy(psi).cuda(), tol=tol, inner_prec=inner)
    finally:
        mdwf.mdwf_destroy(h)
    assert st == 0
    assert info[0].iters < 200  # the Pauli-Villars solve is cheap (Sec. 2.3)
    assert np.abs(out.cpu().numpy() - ref).max() <= bound * np.abs(ref).max()


def test_pv_reconstruct_reproduces_bulk_solution():
    """Psi from the reconstruction equals P^dag D(m)^-1 D(1) P B of a direct 5d solve."""
    dims, Ls, mf = (4, 4, 4, 4), 8, 0.05
    U = sy.gauge_field(dims, 0.3, 1054)
    b = sy.gaussian_field(dims, 1, 2054)[0]
    p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, mf)
    B = np.zeros((Ls,) + b.shape, complex)
    B[0] = b
    X, st0, _, _ = oracle.solve(oracle.ddw(wall_P(B), U, p.with_(mf=1.0)), U, p, tol=1e-13)
    assert st0 == 0
    Psi_ref = wall_Pdag(X)
    psi = np.ascontiguousarray(Psi_ref[0])  # = D_ov(m)^-1 b (App. A)
    h = ctx(dims, Ls, 1.5, 0.5, mf, U)
    try:
        Psi = np.empty_like(Psi_ref)
        st, info = mdwf.mdwf_pv_reconstruct(h, Psi, psi, tol=1e-13)
    finally:
        mdwf.mdwf_destroy(h)
    assert st == 0
    assert np.abs(Psi - Psi_ref).max() <= 1e-9 * np.abs(Psi_ref).max()


def test_gw_violation_matches_dense():
    """Delta_Ls psi = (1 - eps_Ls(H_M)^2) psi / 4 (Eq. Delta_Ls) on 2^4, Ls = 4."""
    dims, Ls, M5, m = (2, 2, 2, 2), 4, 1.8, 0.05
    b5, c5 = 1.5, 0.5
    U = sy.gauge_field(dims, 0.3, 1055)
    V = 16
    DW = dense_of(lambda v: oracle.dw(v, U, dims, M5), 12 * V, (2, 2, 2, 2, 4, 3))
    g5 = np.kron(np.eye(V), np.kron(np.diag([1, 1, -1, -1]), np.eye(3))).astype(complex)
    # eps from the dense overlap operator: gamma5 (2 D_ov - (1 + m)) / (1 - m)
    eps = g5 @ (2 * overlap_operator(DW, g5, Ls, b5, c5, m) - (1 + m) * np.eye(12 * V)) / (1 - m)
    delta = 0.25 * (np.eye(12 * V) - eps @ eps)
    rng = np.random.default_rng(11)
    psi = rng.standard_normal((2, 2, 2, 2, 4, 3)) + 1j * rng.standard_normal((2, 2, 2, 2, 4, 3))
    h = ctx(dims, Ls, b5, c5, m, U)
    try:
        out = np.empty_like(psi)
        st, info = mdwf.mdwf_gw_violation(h, out, psi, tol=1e-13)
    finally:
        mdwf.mdwf_destroy(h)
    assert st == 0
    ref = (delta @ psi.reshape(-1)).reshape(psi.shape)
    assert np.abs(out - ref).max() <= 1e-8 * np.abs(psi).max()
