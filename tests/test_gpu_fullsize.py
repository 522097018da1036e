"""Parity at the full sizes of the batched workloads, in the launch
configuration the solver uses (one launch over all right-hand sides):

* 24^3 x 64, Ls = 12, mf = 0.005, b5 = 1.5, c5 = 0.5, links eps = 0.2: a
  12-right-hand-side FP32 apply, and the mixed FP32/FP64 CGNE of the 12
  spin-colour point sources at the origin;
* 32^3 x 64, Ls = 16, b5 = 1.5, c5 = 0.5, links eps = 0.15: an 8-mass FP16+norm
  apply (masses 0.001 .. 0.05 in one launch), and the 8-source, 8-mass mixed
  FP16+norm CGNE with FP64 reliable updates and autotuned tiles (about a minute
  on the GPU and two on the host cores for the oracle's residuals).

* 16^3 x 32, Ls = 16 (the bench lattice): the mixed solve with per-slice
  Zolotarev coefficients, and the force at mf = 0.02 against central
  differences of its action.

The oracle checks sampled right-hand sides element by element (tolerances of
the operator tests: F32 1e-5 of max |oracle|, F16N 3e-3 in the 2-norm) and the
solves through its own FP64 residuals.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle
import paper_1206_5214_gb300 as mdwf
import synthetic as sy
from _gpu import Ctx, rel_err

pytestmark = pytest.mark.gpu

F32, F16N = mdwf.MDWF_F32, mdwf.MDWF_F16N
C5_MASSES = [0.001, 0.002, 0.005, 0.01, 0.02, 0.03, 0.04, 0.05]


def batch_of_copies(odd, n):
    """n right-hand sides e^{i r} (r + 1) psi: one Gaussian draw, distinct per slot."""
    out = np.empty((n,) + odd.shape, np.complex128)
    for r in range(n):
        out[r] = np.exp(1j * r) * (r + 1) * odd
    return out


def oracle_residuals(x_full, b_full, U, p):
    """(|M^dag b' - M^dag M x_o| / |M^dag b'|, |b' - M x_o| / |b'|) from the oracle."""
    bp = oracle.prepare(b_full, U, p)
    _, xo = oracle.split(x_full, p.dims)
    mx = oracle.m(xo, U, p)
    src = oracle.m(bp, U, p, dagger=True)
    normal = np.linalg.norm(src - oracle.m(mx, U, p, dagger=True)) / np.linalg.norm(src)
    first = np.linalg.norm(bp - mx) / np.linalg.norm(bp)
    return normal, first


@pytest.fixture(scope="module")
def c3_links():
    dims = (24, 24, 24, 64)
    return dims, sy.gauge_field(dims, 0.2, sy.config_seed("gauge", 3))


def test_apply_24x24x24x64_Ls12_twelve_rhs_f32(c3_links):
    dims, U = c3_links
    Ls = 12
    p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, 0.005)
    _, odd = oracle.split(sy.gaussian_field(dims, Ls, sy.config_seed("source", 3)), dims)
    batch = batch_of_copies(odd, 12)
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.005, U) as c:
        for dagger in (False, True):
            got = c.apply(batch, F32, dagger, nrhs=12)
            ref = oracle.m(odd, U, p, dagger=dagger)
            for r in (0, 7, 11):
                emax, _ = rel_err(got[r], np.exp(1j * r) * (r + 1) * ref)
                assert emax <= 1e-5, (dagger, r, emax)


def test_cgne_24x24x24x64_Ls12_point_sources_mixed_f32(c3_links):
    """12 point sources in one batched mixed solve (host buffers) to 1e-10."""
    dims, U = c3_links
    Ls = 12
    p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, 0.005)
    b = sy.point_sources(dims, Ls)
    x = np.zeros_like(b)
    h = mdwf.mdwf_create(dims, Ls, 1.8, 1.5, 0.5, 0.005)
    try:
        mdwf.mdwf_load_gauge(h, U)
        st, info = mdwf.mdwf_cgne(h, x, b, nrhs=12, tol=1e-10, inner_prec=F32)
    finally:
        mdwf.mdwf_destroy(h)
    print("point sources", [i.as_dict() for i in info[:2]])
    assert st == 0
    assert all(i.true_res <= 1e-10 for i in info)
    for r in (0, 11):  # spin 0 colour 0 on s = Ls - 1, and spin 3 colour 2 on s = 0
        normal, first = oracle_residuals(x[r], b[r], U, p)
        assert normal <= 1.05e-10, (r, normal)
        assert first <= 1e-8, (r, first)


@pytest.fixture(scope="module")
def c5_links():
    dims = (32, 32, 32, 64)
    return dims, sy.gauge_field(dims, 0.15, sy.config_seed("gauge", 5))


def test_apply_32x32x32x64_Ls16_eight_masses_f16n(c5_links):
    dims, U = c5_links
    Ls = 16
    _, odd = oracle.split(sy.gaussian_field(dims, Ls, sy.config_seed("source", 5)), dims)
    batch = batch_of_copies(odd, 8)
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.01, U) as c:
        got = c.apply(batch, F16N, False, nrhs=8, masses=C5_MASSES)
    for r in (0, 7):
        ref = oracle.m(odd, U, oracle.Params(dims, Ls, 1.8, 1.5, 0.5, C5_MASSES[r]))
        _, el2 = rel_err(got[r], np.exp(1j * r) * (r + 1) * ref)
        assert el2 <= 3e-3, (r, el2)


def test_cgne_32x32x32x64_Ls16_eight_masses_mixed_f16n(c5_links):
    """8 Gaussian sources at the 8 masses in one batched solve (host buffers),
    FP16+norm inner iterations with FP64 reliable updates, autotuned tiles."""
    dims, U = c5_links
    Ls = 16
    b = sy.gaussian_field(dims, Ls, sy.config_seed("source", 5), nrhs=8)
    x = np.zeros_like(b)
    h = mdwf.mdwf_create(dims, Ls, 1.8, 1.5, 0.5, 0.01, autotune=True)
    try:
        mdwf.mdwf_load_gauge(h, U)
        st, info = mdwf.mdwf_cgne(h, x, b, nrhs=8, mf_per_rhs=C5_MASSES, tol=1e-10, inner_prec=F16N,
                                  maxiter=40000)
    finally:
        mdwf.mdwf_destroy(h)
    for r, i in enumerate(info):
        print("mf", C5_MASSES[r], i.as_dict())
    assert st == 0, [i.as_dict() for i in info]
    assert all(i.true_res <= 1e-10 for i in info)
    for r in (0, 7):
        p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, C5_MASSES[r])
        normal, first = oracle_residuals(x[r], b[r], U, p)
        assert normal <= 1.05e-10, (r, normal)
        assert first <= 1e-8, (r, first)


def test_cgne_16x16x16x32_Ls16_zolotarev_mixed_f32():
    """The bench lattice (16^3 x 32, Ls = 16, links eps = 0.2) with per-slice Zolotarev
    coefficients for |lambda| in [0.05, 0.756]: the fused iteration with dense
    s-operators, mixed FP32/FP64 to 1e-10, checked through the oracle's residuals."""
    from paper_1206_5214_gb300 import zolotarev
    dims, Ls, mf = (16, 16, 16, 32), 16, 0.01
    b5s, c5s = zolotarev.zolotarev_coefficients(Ls, 0.05, 0.756)
    U = sy.gauge_field(dims, 0.2, sy.config_seed("gauge", 2))
    b = sy.gaussian_field(dims, Ls, sy.config_seed("source", 2))
    p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, mf, b5s=tuple(b5s), c5s=tuple(c5s))
    h = mdwf.mdwf_create(dims, Ls, 1.8, 1.5, 0.5, mf)
    try:
        mdwf.mdwf_load_gauge(h, torch.from_numpy(U).cuda())
        mdwf.mdwf_set_s_coefficients(h, list(b5s), list(c5s))
        bd = torch.from_numpy(b).cuda()
        xd = torch.zeros_like(bd)
        st, info = mdwf.mdwf_cgne(h, xd, bd, tol=1e-10, inner_prec=F32)
        x = xd.cpu().numpy()
    finally:
        mdwf.mdwf_destroy(h)
    print("zolotarev", info[0].as_dict())
    assert st == 0 and info[0].true_res <= 1e-10
    normal, first = oracle_residuals(x, b, U, p)
    assert normal <= 1.05e-10, normal
    assert first <= 1e-8, first


def test_force_16x16x16x32_Ls16_finite_differences():
    """The force workload (16^3 x 32, Ls = 16, mf = 0.02, links eps = 0.2): dS/dU along a
    random su(3) direction and dS/db5 against central differences (h = 1e-5) of S, with
    FP64 solves to 1e-13 so that the difference quotients resolve the derivatives."""
    dims, Ls, mf = (16, 16, 16, 32), 16, 0.02
    U = sy.gauge_field(dims, 0.2, sy.config_seed("gauge", 4))
    _, phi = oracle.split(sy.gaussian_field(dims, Ls, sy.config_seed("source", 4)), dims)
    rng = np.random.default_rng(44)
    a = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
    w = 0.5 * (a - np.conj(np.swapaxes(a, -1, -2)))
    w -= np.trace(w, axis1=-2, axis2=-1)[..., None, None] / 3.0 * np.eye(3)
    lam, v = np.linalg.eigh(1j * w)

    def expm(t):
        return np.einsum("...ij,...j,...kj->...ik", v, np.exp(-1j * t * lam), np.conj(v))

    phid = torch.from_numpy(phi).cuda()

    def action(Ux, b5=1.5, derivs=False):
        h = mdwf.mdwf_create(dims, Ls, 1.8, b5, 0.5, mf)
        try:
            mdwf.mdwf_load_gauge(h, torch.from_numpy(np.ascontiguousarray(Ux)).cuda())
            G = torch.empty(U.shape, dtype=torch.complex128, device="cuda") if derivs else None
            S, db5, dc5, st, info = mdwf.mdwf_force(h, G, phid, tol=1e-13)
            assert st == 0, info.as_dict()
            return S, (G.cpu().numpy() if derivs else None), db5
        finally:
            mdwf.mdwf_destroy(h)

    S0, G, db5 = action(U, derivs=True)
    eps = 1e-5
    fd = (action(expm(eps) @ U)[0] - action(expm(-eps) @ U)[0]) / (2 * eps)
    an = float(np.sum(np.real(np.conj(G) * (w @ U))))
    assert an == pytest.approx(fd, rel=1e-4)
    fd_b5 = (action(U, b5=1.5 + eps)[0] - action(U, b5=1.5 - eps)[0]) / (2 * eps)
    assert db5 == pytest.approx(fd_b5, rel=1e-4)
