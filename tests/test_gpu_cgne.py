"""GPU CGNE solves (prepare -> CG on M^dag M -> reconstruct) against the FP64
oracle: plain FP64 and mixed FP32 / FP16+norm with FP64 reliable updates.

Bar: the reported FP64 true residual |M^dag b' - M^dag M x| / |M^dag b'| is
<= 1e-10, the oracle recomputes it from the GPU solution and agrees, and on
lattices where the oracle solves too the solutions agree to cond * 1e-10.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle
import paper_1206_5214_gb300 as mdwf
import synthetic as sy

pytestmark = pytest.mark.gpu

F64, F32, F16N = mdwf.MDWF_F64, mdwf.MDWF_F32, mdwf.MDWF_F16N


def oracle_residual(x_full, b_full, U, p):
    """|M^dag b' - M^dag M x_o| / |M^dag b'| computed by the oracle."""
    bp = oracle.prepare(b_full, U, p)
    src = oracle.m(bp, U, p, dagger=True)
    _, xo = oracle.split(x_full, p.dims)
    r = src - oracle.mdagm(xo, U, p)
    return np.linalg.norm(r) / np.linalg.norm(src)


def gpu_solve(dims, Ls, b5, c5, mf, U, b, inner, nrhs=1, masses=None, host=False, graph=True, tol=1e-10,
              staged=None, maxiter=20000):
    h = mdwf.mdwf_create(dims, Ls, 1.8, b5, c5, mf)
    try:
        if staged is not None and inner != F64:
            mdwf.mdwf_set_staging(h, inner, staged)
        if host:
            mdwf.mdwf_load_gauge(h, np.ascontiguousarray(U))
            bb = np.ascontiguousarray(b)
            x = np.zeros_like(bb)
        else:
            mdwf.mdwf_load_gauge(h, torch.from_numpy(U).cuda())
            bb = torch.from_numpy(np.ascontiguousarray(b)).cuda()
            x = torch.zeros_like(bb)
        st, info = mdwf.mdwf_cgne(h, x, bb, nrhs=nrhs, mf_per_rhs=masses, tol=tol, inner_prec=inner,
                                  use_graph=graph, maxiter=maxiter, raise_on_error=maxiter == 20000)
        xs = x if host else x.cpu().numpy()
        return st, info, xs
    finally:
        mdwf.mdwf_destroy(h)


@pytest.mark.parametrize("staged", [0, 1, 2, 3, 4], ids=["default", "cp.async", "bulk", "prefetch", "registers"])
@pytest.mark.parametrize("b5,c5", [(1.0, 0.0), (1.5, 0.5)], ids=["shamir", "moebius"])
@pytest.mark.parametrize("inner", [F64, F32, F16N], ids=["f64", "mixed-f32", "mixed-f16n"])
def test_cgne_4x4x4x4_matches_oracle_solve(b5, c5, inner, staged):
    """4^4, Ls = 8, M5 = 1.8, mf = 0.01, eps = 0.3, one Gaussian source, CGNE to 1e-10."""
    dims, Ls = (4, 4, 4, 4), 8
    U = sy.gauge_field(dims, 0.3, 1001)
    b = sy.gaussian_field(dims, Ls, 2001)
    p = oracle.Params(dims, Ls, 1.8, b5, c5, 0.01)
    x_ref, st_ref, it_ref, rel_ref = oracle.solve(b, U, p, tol=1e-12)
    assert st_ref == 0
    if inner == F64 and staged:
        pytest.skip("the FP64 operator has no staged variant")
    st, info, x = gpu_solve(dims, Ls, b5, c5, 0.01, U, b, inner, staged=staged)
    assert st == 0, info[0].as_dict()
    assert info[0].true_res <= 1e-10
    xs = x[0] if x.ndim == 8 else x
    assert oracle_residual(xs, b, U, p) <= 1.05e-10
    # two solutions with normal-equation residuals <= 1e-10 differ by at most
    # kappa(M^dag M) * 2e-10; kappa stays below 1e4 on these 4^4 x 8 lattices
    err = np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref)
    assert err <= 2e-6, err
    # and the first-order system is solved: |b' - M x_o| / |b'| from the oracle, which
    # the solve reports as res_m (formed with the reconstruction's hop as M's first)
    bp = oracle.prepare(b, U, p)
    _, xo = oracle.split(xs, dims)
    res_m = np.linalg.norm(bp - oracle.m(xo, U, p)) / np.linalg.norm(bp)
    assert res_m <= 1e-8
    assert abs(info[0].res_m - res_m) <= 1e-3 * res_m, (info[0].res_m, res_m)
    if inner != F64:
        assert info[0].reliable_updates >= 1


@pytest.mark.parametrize("graph", [True, False])
def test_cgne_multi_mass_batch(graph):
    """One batched solve of 3 sources at uneven masses, each checked by the oracle."""
    dims, Ls = (4, 4, 4, 4), 8
    masses = [0.005, 0.02, 0.05]
    U = sy.gauge_field(dims, 0.3, 1001)
    b = sy.gaussian_field(dims, Ls, 2011, nrhs=3)
    st, info, x = gpu_solve(dims, Ls, 1.5, 0.5, 0.01, U, b, F32, nrhs=3, masses=masses, graph=graph)
    assert st == 0
    for r, m in enumerate(masses):
        p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, m)
        assert info[r].true_res <= 1e-10
        assert oracle_residual(x[r], b[r], U, p) <= 1.05e-10
    # lighter masses need more iterations
    assert info[0].iters >= info[2].iters


def test_cgne_host_buffers_and_point_sources():
    """Host-memory b and x; 12 spin-colour point sources on the walls."""
    dims, Ls = (4, 4, 4, 4), 8
    U = sy.gauge_field(dims, 0.3, 1003)
    b = sy.point_sources(dims, Ls)
    st, info, x = gpu_solve(dims, Ls, 1.5, 0.5, 0.005, U, b, F32, nrhs=12, host=True)
    assert st == 0
    p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, 0.005)
    for r in (0, 5, 11):
        assert oracle_residual(x[r], b[r], U, p) <= 1.05e-10


def test_cgne_zero_source():
    dims, Ls = (4, 4, 2, 2), 4
    U = sy.gauge_field(dims, 0.3, 1004)
    b = np.zeros((Ls, 2, 2, 4, 4, 4, 3), complex)
    st, info, x = gpu_solve(dims, Ls, 1.5, 0.5, 0.01, U, b, F32)
    assert st == 0 and np.count_nonzero(x) == 0


def test_cgne_maxiter_reports_noconv():
    dims, Ls = (4, 4, 4, 4), 8
    U = sy.gauge_field(dims, 0.3, 1001)
    b = sy.gaussian_field(dims, Ls, 2001)
    h = mdwf.mdwf_create(dims, Ls, 1.8, 1.5, 0.5, 0.01)
    try:
        mdwf.mdwf_load_gauge(h, torch.from_numpy(U).cuda())
        bb = torch.from_numpy(b).cuda()
        x = torch.zeros_like(bb)
        st, info = mdwf.mdwf_cgne(h, x, bb, maxiter=5, inner_prec=F64, raise_on_error=False)
        assert st == 4 and info[0].status == 4
        assert info[0].iters <= 8 and info[0].true_res > 1e-10
    finally:
        mdwf.mdwf_destroy(h)


@pytest.mark.parametrize("inner", [F32, F16N], ids=["mixed-f32", "mixed-f16n"])
def test_cgne_full_16x16x16x32(inner):
    """16^3 x 32, Ls = 16, alpha = 2: the mixed solve reaches 1e-10, checked by the oracle."""
    dims, Ls = (16, 16, 16, 32), 16
    U = sy.gauge_field(dims, 0.2, 1002)
    b = sy.gaussian_field(dims, Ls, 2002)
    p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, 0.01)
    st, info, x = gpu_solve(dims, Ls, 1.5, 0.5, 0.01, U, b, inner)
    assert st == 0, info[0].as_dict()
    assert info[0].true_res <= 1e-10
    assert oracle_residual(x[0] if x.ndim == 8 else x, b, U, p) <= 1.05e-10


@pytest.mark.parametrize("inner", [F64, F32], ids=["f64", "mixed-f32"])
def test_cgne_warm_start(inner):
    """guess=True starts the CG from the odd part of the x passed in (restart /
    resume): the converged solution needs no iteration, a perturbed one fewer
    than a cold start, and both still solve the system (oracle residual)."""
    dims, Ls = (4, 4, 4, 4), 8
    U = sy.gauge_field(dims, 0.3, 1091)
    b = sy.gaussian_field(dims, Ls, 2091)
    p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, 0.01)
    h = mdwf.mdwf_create(dims, Ls, 1.8, 1.5, 0.5, 0.01)
    try:
        mdwf.mdwf_load_gauge(h, torch.from_numpy(U).cuda())
        bb = torch.from_numpy(b).cuda()
        x = torch.zeros_like(bb)
        st, cold = mdwf.mdwf_cgne(h, x, bb, tol=1e-10, inner_prec=inner)
        assert st == 0
        st, again = mdwf.mdwf_cgne(h, x, bb, tol=1e-10, inner_prec=inner, guess=True)
        assert st == 0 and again[0].iters == 0
        rng = np.random.default_rng(4)
        noise = torch.from_numpy(rng.standard_normal(b.shape) + 0j).cuda()
        x2 = x + 1e-4 * noise * torch.linalg.vector_norm(x) / torch.linalg.vector_norm(noise)
        st, warm = mdwf.mdwf_cgne(h, x2, bb, tol=1e-10, inner_prec=inner, guess=True)
        assert st == 0 and 0 < warm[0].iters < cold[0].iters
        # a zero source gives x = 0 whatever the guess
        z = torch.zeros_like(bb)
        xz = x.clone()
        st, _ = mdwf.mdwf_cgne(h, xz, z, tol=1e-10, inner_prec=inner, guess=True)
        assert st == 0 and int(torch.count_nonzero(xz)) == 0
        xs = x2.cpu().numpy()
    finally:
        mdwf.mdwf_destroy(h)
    assert oracle_residual(xs, b, U, p) <= 1.05e-10


@pytest.mark.parametrize("inner", [F64, F32], ids=["f64", "mixed-f32"])
def test_cgne_nan_source_is_reported_per_rhs(inner):
    """Failure detection on the host side of a solve: a NaN planted in one source
    of a batch ends that right-hand side with MDWF_EBREAKDOWN while the other
    converges; the call returns normally."""
    dims, Ls = (4, 4, 2, 4), 6
    U = sy.gauge_field(dims, 0.3, 1093)
    b = sy.gaussian_field(dims, Ls, 2093, nrhs=2)
    b[1, 2, 0, 1, 0, 1, 3, 2] = np.nan
    h = mdwf.mdwf_create(dims, Ls, 1.8, 1.5, 0.5, 0.02)
    try:
        mdwf.mdwf_load_gauge(h, torch.from_numpy(U).cuda())
        bb = torch.from_numpy(b).cuda()
        x = torch.zeros_like(bb)
        st, info = mdwf.mdwf_cgne(h, x, bb, nrhs=2, tol=1e-10, inner_prec=inner, raise_on_error=False)
    finally:
        mdwf.mdwf_destroy(h)
    assert st == 5
    assert info[0].status == 0 and info[0].true_res <= 1e-10
    assert info[1].status == 5


@pytest.mark.parametrize("staged", [0, 1], ids=["no-t-field", "t-field"])
@pytest.mark.parametrize("b5,c5", [(1.0, 0.0), (1.5, 0.5)], ids=["shamir", "moebius"])
@pytest.mark.parametrize("inner", [F32, F16N], ids=["mixed-f32", "mixed-f16n"])
def test_cgne_4x4x4x4_Ls16_matches_oracle(inner, b5, c5, staged):
    """Ls = 16 (the fused iteration's Ls-specialised kernels and the shuffled M_phi^dag of
    its last hop) to 1e-10, checked through the oracle's residuals. With the default load
    strategy the iteration keeps no t field (its last hop forms t = I^dag v by shuffles);
    the cp.async staging keeps and reads t, so both forms are checked."""
    dims, Ls, mf = (4, 4, 4, 4), 16, 0.01
    U = sy.gauge_field(dims, 0.3, 1092)
    b = sy.gaussian_field(dims, Ls, 2092)
    p = oracle.Params(dims, Ls, 1.8, b5, c5, mf)
    st, info, x = gpu_solve(dims, Ls, b5, c5, mf, U, b, inner, staged=staged)
    assert st == 0 and info[0].true_res <= 1e-10
    assert oracle_residual(x, b, U, p) <= 1.05e-10


def test_Ls16_iteration_without_t_field_matches_t_field():
    """The Ls = 16 iteration without a t field forms t = A (cf z' + I p) and v = A^dag t
    in one column pass and |t|^2 from the columns; the iteration that stores t applies
    A and A^dag in two passes. In exact arithmetic both are the CG of the plain FP64
    solve, reliable updates included, so after 16 iterations (cut off by maxiter) the
    three iterates agree up to FP32 rounding, while a wrong |t|^2 or v would move the
    iterate at order one; run to 1e-10, both FP32 forms converge to the same solution."""
    dims, Ls, mf = (4, 4, 4, 8), 16, 0.01
    U = sy.gauge_field(dims, 0.3, 1096)
    b = sy.gaussian_field(dims, Ls, 2096)
    st64, info64, x64 = gpu_solve(dims, Ls, 1.5, 0.5, mf, U, b, F64, maxiter=16)
    assert st64 == mdwf.MDWF_ENOCONV
    for staged in (0, 1):
        st, info, x = gpu_solve(dims, Ls, 1.5, 0.5, mf, U, b, F32, staged=staged, maxiter=16)
        assert st == mdwf.MDWF_ENOCONV and info[0].iters == info64[0].iters
        assert np.linalg.norm(x - x64) <= 1e-4 * np.linalg.norm(x64), staged
    runs = [gpu_solve(dims, Ls, 1.5, 0.5, mf, U, b, F32, staged=st) for st in (0, 1)]
    assert all(st == 0 and info[0].true_res <= 1e-10 for st, info, _ in runs)
    # two solutions with residuals <= 1e-10 differ by at most kappa(M^dag M) * 2e-10
    x0, x1 = runs[0][2], runs[1][2]
    assert np.linalg.norm(x0 - x1) <= 1e-5 * np.linalg.norm(x1)


@pytest.mark.parametrize("inner,dims,Ls,seed,delta", [
    (F16N, (8, 8, 8, 8), 16, 1097, 0.0),
    (F16N, (4, 4, 4, 4), 8, 1001, 0.01),
    (F32, (4, 4, 4, 4), 8, 1001, 1e-4),
    (F32, (4, 4, 4, 8), 16, 1096, 1e-6),
    (F32, (8, 8, 8, 8), 16, 1097, 1e-4),
], ids=["f16n-8x8x8x8-default", "f16n-4x4x4x4-Ls8-1e-2", "f32-4x4x4x4-Ls8-1e-4", "f32-4x4x4x8-1e-6",
        "f32-8x8x8x8-1e-4"])
def test_mixed_solve_safeguards(inner, dims, Ls, seed, delta):
    """Cases in which the inner iteration, with p kept unchanged across reliable updates,
    drifted from the true residual and broke down (a small delta) or diverged (FP16
    storage on a rough 8^4 field). With the search direction corrected at each update
    (its component along the new residual removed, beta from the true |r|^2), a forced
    update when the inner |r| climbs and a roll-back after a breakdown, every one reaches
    1e-10, confirmed by the oracle's residual."""
    U = sy.gauge_field(dims, 0.3, seed)
    b = sy.gaussian_field(dims, Ls, seed + 1000)
    p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, 0.01)
    h = mdwf.mdwf_create(dims, Ls, 1.8, 1.5, 0.5, 0.01)
    try:
        mdwf.mdwf_load_gauge(h, torch.from_numpy(U).cuda())
        bb = torch.from_numpy(np.ascontiguousarray(b)).cuda()
        x = torch.zeros_like(bb)
        st, info = mdwf.mdwf_cgne(h, x, bb, tol=1e-10, inner_prec=inner, delta=delta, raise_on_error=False)
        xs = x.cpu().numpy()
    finally:
        mdwf.mdwf_destroy(h)
    assert st == 0 and info[0].true_res <= 1e-10, info[0].as_dict()
    assert oracle_residual(xs, b, U, p) <= 1.05e-10


@pytest.mark.parametrize("inner", [F32, F16N], ids=["mixed-f32", "mixed-f16n"])
def test_near_fp64_limit_with_no_threshold(inner):
    """delta = 1e-30 never triggers an update on its own: the inner iteration runs until
    its estimate says 1e-14 or it breaks down. The corrected directions, restarts and
    roll-backs still take the solve to a true residual of 1e-14, near the FP64 limit,
    confirmed by the oracle."""
    dims, Ls = (4, 4, 4, 4), 8
    U = sy.gauge_field(dims, 0.3, 1001)
    b = sy.gaussian_field(dims, Ls, 2001)
    p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, 0.01)
    h = mdwf.mdwf_create(dims, Ls, 1.8, 1.5, 0.5, 0.01)
    try:
        mdwf.mdwf_load_gauge(h, torch.from_numpy(U).cuda())
        bb = torch.from_numpy(np.ascontiguousarray(b)).cuda()
        x = torch.zeros_like(bb)
        st, info = mdwf.mdwf_cgne(h, x, bb, tol=1e-14, inner_prec=inner, delta=1e-30, maxiter=4000,
                                  raise_on_error=False)
        xs = x.cpu().numpy()
    finally:
        mdwf.mdwf_destroy(h)
    assert st == 0 and info[0].true_res <= 1e-14 and info[0].restarts >= 1, info[0].as_dict()
    assert oracle_residual(xs, b, U, p) <= 2e-14


def test_roll_back_after_inner_breakdown():
    """With an unreachable target (1e-30) and threshold the inner FP32 iteration runs on
    until it breaks down; each breakdown rolls back to the last reliable update (more
    restarts than updates: an update restarts p at most once). The solve ends at maxiter
    with MDWF_ENOCONV, a finite x and the FP64 residual at its floor."""
    dims, Ls = (4, 4, 2, 4), 6
    U = sy.gauge_field(dims, 0.3, 1093)
    b = sy.gaussian_field(dims, Ls, 2093)
    h = mdwf.mdwf_create(dims, Ls, 1.8, 1.5, 0.5, 0.01)
    try:
        mdwf.mdwf_load_gauge(h, torch.from_numpy(U).cuda())
        bb = torch.from_numpy(np.ascontiguousarray(b)).cuda()
        x = torch.zeros_like(bb)
        st, info = mdwf.mdwf_cgne(h, x, bb, tol=1e-30, inner_prec=F32, delta=1e-30, maxiter=3000,
                                  raise_on_error=False)
        finite = bool(torch.isfinite(x).all())
    finally:
        mdwf.mdwf_destroy(h)
    assert st == mdwf.MDWF_ENOCONV and finite
    assert info[0].restarts > info[0].reliable_updates, info[0].as_dict()
    assert info[0].true_res <= 1e-14


def test_default_delta_takes_no_restart():
    """At the default threshold a well-behaved FP32 solve neither restarts p nor breaks
    down: every reliable update finds the true residual within twice the inner one."""
    dims, Ls, mf = (4, 4, 4, 8), 16, 0.01
    U = sy.gauge_field(dims, 0.3, 1096)
    b = sy.gaussian_field(dims, Ls, 2096)
    st, info, _ = gpu_solve(dims, Ls, 1.5, 0.5, mf, U, b, F32)
    assert st == 0 and info[0].restarts == 0 and info[0].reliable_updates >= 2


def test_cgne_Ls16_multi_mass_without_t_field():
    """Three masses in one Ls = 16 mixed FP32 solve with the t field dropped: each
    right-hand side's I^dag takes its own mass in the wrap-around term."""
    dims, Ls = (4, 4, 4, 4), 16
    masses = [0.005, 0.05, 0.3]
    U = sy.gauge_field(dims, 0.3, 1095)
    b = sy.gaussian_field(dims, Ls, 2095, nrhs=3)
    st, info, x = gpu_solve(dims, Ls, 1.5, 0.5, 0.01, U, b, F32, nrhs=3, masses=masses)
    assert st == 0 and all(i.true_res <= 1e-10 for i in info)
    for r, m in enumerate(masses):
        p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, m)
        assert oracle_residual(x[r], b[r], U, p) <= 1.05e-10, r


def test_cgne_max_batch():
    """64 right-hand sides with 64 masses in one mixed FP32 solve (4x2x2x2, Ls = 4): every
    slot reaches 1e-10 and solves D_DW(m_r) x = b_r by the oracle."""
    dims, Ls, n = (4, 2, 2, 2), 4, 64
    U = sy.gauge_field(dims, 0.3, 1094)
    b = sy.gaussian_field(dims, Ls, 2094, nrhs=n)
    masses = list(np.linspace(0.01, 0.5, n))
    h = mdwf.mdwf_create(dims, Ls, 1.8, 1.5, 0.5, 0.01)
    try:
        mdwf.mdwf_load_gauge(h, torch.from_numpy(U).cuda())
        bb = torch.from_numpy(np.ascontiguousarray(b)).cuda()
        x = torch.zeros_like(bb)
        st, info = mdwf.mdwf_cgne(h, x, bb, nrhs=n, mf_per_rhs=masses, tol=1e-10, inner_prec=F32)
        xs = x.cpu().numpy()
    finally:
        mdwf.mdwf_destroy(h)
    assert st == 0 and all(i.true_res <= 1e-10 for i in info)
    for r in range(0, n, 9):
        p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, masses[r])
        res = b[r] - oracle.ddw(xs[r], U, p)
        assert np.linalg.norm(res) / np.linalg.norm(b[r]) <= 1e-7, r


@pytest.mark.parametrize("inner", [F32, F16N], ids=["mixed-f32", "mixed-f16n"])
def test_reliable_updates_per_rhs(inner):
    """In a batch of masses each right-hand side takes its own FP64 reliable
    updates, when its own inner residual asks for one, while the others' inner
    iterations go on untouched: every right-hand side of the batch takes the
    same iterations and reliable updates as its solve alone (the batched
    kernels and the fixed-order reductions compute each right-hand side as the
    single solve does), and solves its system."""
    dims, Ls = (4, 4, 4, 4), 8
    masses = [0.005, 0.05, 0.8]
    U = sy.gauge_field(dims, 0.3, 1096)
    b = sy.gaussian_field(dims, Ls, 2096, nrhs=3)
    st, info, x = gpu_solve(dims, Ls, 1.5, 0.5, 0.01, U, b, inner, nrhs=3, masses=masses)
    assert st == 0 and all(i.true_res <= 1e-10 for i in info), [i.as_dict() for i in info]
    for r, m in enumerate(masses):
        st1, info1, _ = gpu_solve(dims, Ls, 1.5, 0.5, m, U, b[r], inner)
        assert st1 == 0
        assert (info[r].iters, info[r].reliable_updates) == (info1[0].iters, info1[0].reliable_updates), \
            (r, info[r].as_dict(), info1[0].as_dict())
        p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, m)
        assert oracle_residual(x[r], b[r], U, p) <= 1.05e-10, r
