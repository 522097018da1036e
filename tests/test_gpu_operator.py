"""GPU parity of the red/black Moebius operator M, M^dag and the layouts,
called through the C ABI and compared element by element with the FP64 oracle.

Tolerances (written here, derived from the arithmetic):
  F64  : max |gpu - oracle| <= 1e-12 * max |oracle|   (rounding of ~3e3 flops per output)
  F32  : max |gpu - oracle| <= 1e-5  * max |oracle|   (FP32 eps 6e-8 times the same chain)
  F16N : |gpu - oracle|_2  <= 3e-3 * |oracle|_2       (FP16 storage, 2^-11 of each site's max,
                                                       on input, intermediate and output)
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
from _pins import gauge_rotate, rotate_field

pytestmark = pytest.mark.gpu

F64, F32, F16N = mdwf.MDWF_F64, mdwf.MDWF_F32, mdwf.MDWF_F16N
TOL_MAX = {F64: 1e-12, F32: 1e-5}
TOL_L2_F16N = 3e-3


def check(gpu, ref, prec):
    emax, el2 = rel_err(gpu, ref)
    if prec == F16N:
        assert el2 <= TOL_L2_F16N, (emax, el2)
    else:
        assert emax <= TOL_MAX[prec], (emax, el2)
    return emax, el2


def setup(dims, Ls, b5, c5, mf, eps, seed, M5=1.8):
    U = sy.gauge_field(dims, eps, 1000 + seed)
    psi = sy.gaussian_field(dims, Ls, 2000 + seed)
    _, odd = oracle.split(psi, dims)
    p = oracle.Params(dims, Ls, M5, b5, c5, mf)
    return U, odd, p


# ------------------------------------------------------------------ layouts

@pytest.mark.parametrize("prec", [F64, F32, F16N])
def test_import_export_roundtrip(prec):
    dims, Ls = (4, 4, 2, 6), 6
    U, odd, p = setup(dims, Ls, 1.5, 0.5, 0.01, 0.3, 1)
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.01, U) as c:
        back = c.download(c.upload(odd, prec), prec)[0]
    if prec == F64:
        assert np.array_equal(back, odd)
    elif prec == F32:
        f = odd.view(np.float64).astype(np.float32).astype(np.float64).view(np.complex128)
        assert np.array_equal(back, f)
    else:
        # per (site, s) the error is below 2^-11 of that site's max |real component|
        re = odd.view(np.float64).reshape(Ls, -1, 24)
        err = np.abs(back.view(np.float64).reshape(Ls, -1, 24) - re).max(axis=-1)
        assert np.all(err <= 2.0 ** -11 * np.abs(re).max(axis=-1) * 1.0001)


# ------------------------------------------------------------- small lattice

@pytest.mark.parametrize("b5,c5", [(1.0, 0.0), (1.5, 0.5), (2.5, 1.5), (1.0, 1.0), (1.0, 3.0)],
                         ids=["shamir", "moebius", "moebius-alpha4", "borici", "auto-dense"])
@pytest.mark.parametrize("prec", [F64, F32, F16N])
@pytest.mark.parametrize("dagger", [False, True])
def test_apply_parity_4x4x4x4(b5, c5, prec, dagger):
    """4^4 lattice, Ls = 8, mf = 0.01, eps = 0.3: Shamir, Moebius, Borici (b5 = c5) and
    |M-/M+| > 0.9 (c5 = 3), where the context applies the s-operators as dense tables."""
    dims, Ls = (4, 4, 4, 4), 8
    U, odd, p = setup(dims, Ls, b5, c5, 0.01, 0.3, 1)
    ref = oracle.m(odd, U, p, dagger=dagger)
    with Ctx(dims, Ls, 1.8, b5, c5, 0.01, U) as c:
        got = c.apply(odd, prec, dagger)[0]
    check(got, ref, prec)


@pytest.mark.parametrize("b5,c5", [(1.5, 0.5), (1.0, 0.0), (2.5, 1.5)])
@pytest.mark.parametrize("dagger", [False, True])
def test_dense_tables_match_recursion(b5, c5, dagger):
    """The Ls x Ls factors applied as dense host-built matrices and by the
    closed-form elimination give the same operator; both match the oracle."""
    dims, Ls = (4, 4, 2, 4), 12
    U, odd, p = setup(dims, Ls, b5, c5, 0.03, 0.3, 6)
    ref = oracle.m(odd, U, p, dagger=dagger)
    with Ctx(dims, Ls, 1.8, b5, c5, 0.03, U, dense_s=True) as cd, Ctx(dims, Ls, 1.8, b5, c5, 0.03, U) as cr:
        for prec in (F64, F32):
            a = cd.apply(odd, prec, dagger)[0]
            b = cr.apply(odd, prec, dagger)[0]
            check(a, ref, prec)
            check(b, ref, prec)


@pytest.mark.parametrize("dims,Ls", [((6, 2, 2, 4), 4), ((4, 2, 2, 2), 12), ((2, 2, 2, 2), 2), ((8, 2, 4, 2), 16)],
                         ids=["Vh48-Ls4", "Vh16-Ls12", "Vh8-Ls2", "Vh64-Ls16"])
@pytest.mark.parametrize("dagger", [False, True])
def test_apply_ragged_and_edge_shapes(dims, Ls, dagger):
    """Site counts that leave a ragged last block, the smallest lattice and Ls = 2."""
    U, odd, p = setup(dims, Ls, 1.5, 0.5, 0.05, 0.3, 2)
    ref = oracle.m(odd, U, p, dagger=dagger)
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.05, U) as c:
        for prec in (F64, F32):
            check(c.apply(odd, prec, dagger)[0], ref, prec)


@pytest.mark.parametrize("prec", [F64, F32])
@pytest.mark.parametrize("dagger", [False, True])
def test_apply_multi_rhs_multi_mass(prec, dagger):
    """One launch over 3 right-hand sides with different masses."""
    dims, Ls = (4, 4, 2, 4), 8
    masses = [0.001, 0.02, 0.05]
    U = sy.gauge_field(dims, 0.2, 1005)
    srcs = sy.gaussian_field(dims, Ls, 2005, nrhs=3)
    odd = np.stack([oracle.split(srcs[r], dims)[1] for r in range(3)])
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.01, U) as c:
        got = c.apply(odd, prec, dagger, nrhs=3, masses=masses)
    for r, m in enumerate(masses):
        ref = oracle.m(odd[r], U, oracle.Params(dims, Ls, 1.8, 1.5, 0.5, m), dagger=dagger)
        check(got[r], ref, prec)


def test_adjoint_identity_f64():
    dims, Ls = (4, 4, 4, 2), 8
    U, x, p = setup(dims, Ls, 1.5, 0.5, 0.02, 0.3, 3)
    y = oracle.split(sy.gaussian_field(dims, Ls, 2103), dims)[1]
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.02, U) as c:
        my = c.apply(y, F64)[0]
        mdx = c.apply(x, F64, dagger=True)[0]
    lhs, rhs = np.vdot(x, my), np.vdot(mdx, y)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


@pytest.mark.parametrize("prec", [F64, F32])
def test_gauge_covariance(prec):
    """M[U^Omega](Omega psi) = Omega M[U] psi and likewise for M^dag, with a random SU(3)
    Omega(x) per site and U^Omega_mu(x) = Omega(x) U_mu(x) Omega(x+mu)^dag, on an
    anisotropic 4x4x2x6 lattice (Ls = 6) so that forward and backward neighbours differ."""
    dims, Ls = (4, 4, 2, 6), 6
    U, odd, p = setup(dims, Ls, 1.5, 0.5, 0.02, 0.3, 5)
    Om = sy.gauge_transform(dims, 3005)
    UO = gauge_rotate(U, Om)

    def rot(f):
        return oracle.split(rotate_field(oracle.join(np.zeros_like(f), f, dims), Om), dims)[1]

    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.02, U) as c:
        a, ad = c.apply(odd, prec)[0], c.apply(odd, prec, dagger=True)[0]
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.02, UO) as c:
        b, bd = c.apply(rot(odd), prec)[0], c.apply(rot(odd), prec, dagger=True)[0]
    tol = 2 * TOL_MAX[prec]          # two GPU results, each within TOL_MAX of the exact one
    assert rel_err(b, rot(a))[0] <= tol
    assert rel_err(bd, rot(ad))[0] <= tol


def test_linearity_and_zero():
    dims, Ls = (4, 4, 2, 2), 4
    U, a, p = setup(dims, Ls, 1.5, 0.5, 0.02, 0.3, 4)
    b = oracle.split(sy.gaussian_field(dims, Ls, 2104), dims)[1]
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.02, U) as c:
        z = c.apply(np.zeros_like(a), F64)[0]
        assert np.count_nonzero(z) == 0
        lin = c.apply(2.0 * a - 3.0 * b, F64)[0]
        sep = 2.0 * c.apply(a, F64)[0] - 3.0 * c.apply(b, F64)[0]
    assert np.abs(lin - sep).max() <= 1e-12 * np.abs(sep).max()


def test_errors_reported():
    dims, Ls = (4, 4, 4, 4), 8
    h = mdwf.mdwf_create(dims, Ls, 1.8, 1.5, 0.5, 0.01)
    try:
        buf = torch.empty(mdwf.mdwf_field_bytes(h, F64, 1), dtype=torch.uint8, device="cuda")
        out = torch.empty_like(buf)
        with pytest.raises(mdwf.MdwfError) as e:
            mdwf.mdwf_apply(h, out, buf, F64)
        assert e.value.status == 7  # no gauge
        U = torch.from_numpy(sy.unit_gauge(dims)).cuda()
        mdwf.mdwf_load_gauge(h, U)
        with pytest.raises(mdwf.MdwfError) as e:
            mdwf.mdwf_apply(h, buf, buf, F64)
        assert e.value.status == 1  # out aliases in
        with pytest.raises(mdwf.MdwfError):
            mdwf.mdwf_apply(h, out, buf, 7)
    finally:
        mdwf.mdwf_destroy(h)


# ------------------------------------------------------------ full sizes

@pytest.fixture(scope="module")
def c2_case():
    """16^3 x 32, Ls = 16, M5 = 1.8, mf = 0.01, b5 + c5 = 2, b5 - c5 = 1, eps = 0.2."""
    dims, Ls = (16, 16, 16, 32), 16
    U, odd, p = setup(dims, Ls, 1.5, 0.5, 0.01, 0.2, 2)
    refs = {d: oracle.m(odd, U, p, dagger=d) for d in (False, True)}
    return dims, Ls, U, odd, refs


@pytest.mark.parametrize("prec", [F64, F32, F16N])
def test_apply_parity_full_16x16x16x32(c2_case, prec):
    dims, Ls, U, odd, refs = c2_case
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.01, U) as c:
        for d in (False, True):
            check(c.apply(odd, prec, d)[0], refs[d], prec)


@pytest.mark.parametrize("b5,c5", [(1.0, 0.0), (2.5, 1.5)], ids=["alpha1", "alpha4"])
def test_apply_parity_full_16x16x16x32_other_alpha(b5, c5):
    dims, Ls = (16, 16, 16, 32), 16
    U, odd, p = setup(dims, Ls, b5, c5, 0.01, 0.2, 2)
    ref = oracle.m(odd, U, p)
    with Ctx(dims, Ls, 1.8, b5, c5, 0.01, U) as c:
        check(c.apply(odd, F32)[0], ref, F32)


def test_autotune_keeps_results_and_cache(tmp_path):
    """The autotuner's choice is one of the candidate shapes, the operator is
    unchanged by it, and the JSON cache restores it without re-tuning."""
    from paper_1206_5214_gb300 import tuning
    dims, Ls = (8, 4, 4, 4), 16
    U, odd, p = setup(dims, Ls, 1.5, 0.5, 0.02, 0.3, 7)
    ref = oracle.m(odd, U, p)
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.02, U) as c:
        path = str(tmp_path / "tune.json")
        sb = tuning.tuned(c.h, "test-gpu", dims, Ls, F32, 1, path)
        assert sb in (128 // Ls, 64 // Ls, 32 // Ls)
        assert mdwf.mdwf_get_tuning(c.h, F32, 1) == sb
        check(c.apply(odd, F32)[0], ref, F32)
        mdwf.mdwf_set_tuning(c.h, F32, 1, 0)
        assert tuning.tuned(c.h, "test-gpu", dims, Ls, F32, 1, path) == sb   # from the cache
        for shape in (1, 2, 4, 8):
            mdwf.mdwf_set_tuning(c.h, F32, 1, shape)
            check(c.apply(odd, F32)[0], ref, F32)


@pytest.mark.parametrize("mode", [mdwf.STAGE_AUTO, mdwf.STAGE_CP_ASYNC, mdwf.STAGE_BULK, mdwf.STAGE_PREFETCH],
                         ids=["default", "cp.async", "bulk", "prefetch"])
@pytest.mark.parametrize("prec", [F32, F16N])
@pytest.mark.parametrize("dims,Ls", [((8, 4, 4, 4), 16), ((6, 2, 2, 4), 6), ((6, 4, 2, 2), 12), ((4, 2, 2, 6), 32)],
                         ids=["Ls16", "ragged-Ls6", "ragged-Ls12", "Ls32"])
def test_staged_loads_match_plain(mode, prec, dims, Ls):
    """Neighbour spinors staged in shared memory (per-thread cp.async, or whole
    columns by bulk copies) or prefetched into a second register buffer give
    the operator of the plain loads (the same
    arithmetic), and all match the oracle. Vh is not a multiple of the sites per
    block in the ragged cases, so the last block has idle site rows; at Ls = 12
    a site row straddles two warps."""
    U, odd, p = setup(dims, Ls, 1.5, 0.5, 0.02, 0.3, 8)
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.02, U) as c:
        if prec == F16N and mode == mdwf.STAGE_BULK and Ls % 4:
            with pytest.raises(mdwf.MdwfError):
                mdwf.mdwf_set_staging(c.h, prec, mode)
            return
        for dagger in (False, True):
            ref = oracle.m(odd, U, p, dagger=dagger)
            mdwf.mdwf_set_staging(c.h, prec, mdwf.STAGE_REGISTERS)
            a = c.apply(odd, prec, dagger)[0]
            mdwf.mdwf_set_staging(c.h, prec, mode)
            assert mdwf.mdwf_get_staging(c.h, prec) == mode
            b = c.apply(odd, prec, dagger)[0]
            assert np.abs(a - b).max() <= 1e-6 * np.abs(a).max()
            check(b, ref, prec)
        assert mdwf.mdwf_device_status(c.h) == mdwf.MDWF_OK
        if mode != mdwf.STAGE_AUTO:
            with pytest.raises(mdwf.MdwfError):
                mdwf.mdwf_set_staging(c.h, F64, mode)
        with pytest.raises(mdwf.MdwfError):
            mdwf.mdwf_set_staging(c.h, prec, 5)


@pytest.mark.parametrize("arrivals", [0, 1, 2])
def test_bounded_device_wait(arrivals):
    """A device-side wait on an mbarrier that never completes (fewer arrivals
    than expected) gives up within its limit and is reported as MDWF_ETIMEOUT;
    the mark is cleared by the report and the context stays usable."""
    import time
    dims, Ls = (4, 4, 2, 2), 8
    U, odd, p = setup(dims, Ls, 1.5, 0.5, 0.02, 0.3, 10)
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.02, U) as c:
        t0 = time.perf_counter()
        st = mdwf.mdwf_selftest_wait(c.h, arrivals)
        assert time.perf_counter() - t0 < 10.0
        assert st == (mdwf.MDWF_OK if arrivals == 2 else mdwf.MDWF_ETIMEOUT)
        assert mdwf.mdwf_device_status(c.h) == mdwf.MDWF_OK
        check(c.apply(odd, F32)[0], oracle.m(odd, U, p), F32)


@pytest.mark.parametrize("prec", [F64, F32])
def test_apply_parity_Ls32(prec):
    """The largest Ls (32): one s-column fills a warp; M and M^dag against the oracle."""
    dims, Ls = (4, 4, 2, 2), 32
    U, odd, p = setup(dims, Ls, 1.5, 0.5, 0.01, 0.3, 9)
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.01, U) as c:
        for d in (False, True):
            check(c.apply(odd, prec, d)[0], oracle.m(odd, U, p, dagger=d), prec)


@pytest.mark.parametrize("prec", [F32, F16N])
def test_adjoint_Ls16_masses_and_block_shapes(prec):
    """Ls = 16: the bidiagonal s-operator of M^dag runs on warp shuffles when every warp
    holds two whole columns (an even number of sites per block) and through shared memory
    otherwise; three masses in one launch (the wrap-around term carries each -m). Both
    against the oracle, for 8, 2, 3 and 1 sites per block."""
    dims, Ls = (4, 4, 2, 4), 16
    masses = [0.01, 0.1, 0.7]
    U = sy.gauge_field(dims, 0.3, 1091)
    srcs = sy.gaussian_field(dims, Ls, 2091, nrhs=3)
    odd = np.stack([oracle.split(srcs[r], dims)[1] for r in range(3)])
    refs = [oracle.m(odd[r], U, oracle.Params(dims, Ls, 1.8, 1.5, 0.5, m), dagger=True) for r, m in enumerate(masses)]
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.01, U) as c:
        for sb in (8, 2, 3, 1):
            mdwf.mdwf_set_tuning(c.h, prec, 3, sb)
            got = c.apply(odd, prec, True, nrhs=3, masses=masses)
            for r in range(3):
                check(got[r], refs[r], prec)


def test_max_batch_of_right_hand_sides():
    """The largest batch, 64 right-hand sides with 64 masses, in one launch (M and M^dag)
    on a 4x2x2x2 lattice, Ls = 4: every slot against the oracle; 65 is refused."""
    dims, Ls, n = (4, 2, 2, 2), 4, 64
    U = sy.gauge_field(dims, 0.3, 1093)
    srcs = sy.gaussian_field(dims, Ls, 2093, nrhs=n)
    odd = np.stack([oracle.split(srcs[r], dims)[1] for r in range(n)])
    masses = list(np.linspace(0.005, 0.5, n))
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.01, U) as c:
        for dagger in (False, True):
            got = c.apply(odd, F32, dagger, nrhs=n, masses=masses)
            for r in range(n):
                ref = oracle.m(odd[r], U, oracle.Params(dims, Ls, 1.8, 1.5, 0.5, masses[r]), dagger=dagger)
                check(got[r], ref, F32)
        with pytest.raises(mdwf.MdwfError):
            c.apply(np.concatenate([odd, odd[:1]]), F32, False, nrhs=n + 1)
