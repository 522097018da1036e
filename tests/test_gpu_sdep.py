"""GPU operator and solve with per-slice Moebius coefficients b5(s), c5(s)
(Eq. DWaction with D+^(s) = b5(s) D_W + 1, D-^(s) = c5(s) D_W - 1), against the
FP64 oracle with the same per-slice arrays. Tolerances as in the
constant-coefficient parity tests: F64 1e-12 and F32 1e-5 of max |oracle|
elementwise, F16N 3e-3 in the 2-norm."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle
import paper_1206_5214_gb300 as mdwf
import synthetic as sy
from _pins import dense_of
from _gpu import Ctx, rel_err

pytestmark = pytest.mark.gpu

F64, F32, F16N = mdwf.MDWF_F64, mdwf.MDWF_F32, mdwf.MDWF_F16N


def check(gpu, ref, prec):
    emax, el2 = rel_err(gpu, ref)
    if prec == F16N:
        assert el2 <= 3e-3, (emax, el2)
    else:
        assert emax <= {F64: 1e-12, F32: 1e-5}[prec], (emax, el2)


def cosine_profile(Ls, a5=1.0, amp=0.3, centre=1.5):
    """b5(s) = centre + amp cos(2 pi (s + 1/2) / Ls), c5(s) = b5(s) - a5 (b5 - c5 fixed)."""
    b = [centre + amp * np.cos(2 * np.pi * (s + 0.5) / Ls) for s in range(Ls)]
    return b, [x - a5 for x in b]


def generic_profile(Ls, seed):
    """b5(s) in [1, 2.5], c5(s) in [0, 1.5] drawn independently: no symmetry, b5 - c5 varies."""
    rng = np.random.default_rng(seed)
    return list(1.0 + 1.5 * rng.random(Ls)), list(1.5 * rng.random(Ls))


def zolotarev_profile(Ls):
    """The Zolotarev form (b5(s) - c5(s) = 1) for |H_T| in [0.05, 1]."""
    from paper_1206_5214_gb300.zolotarev import zolotarev_coefficients
    return zolotarev_coefficients(Ls, 0.05, 1.0)


PROFILES = {
    "cosine": lambda Ls: cosine_profile(Ls),
    "zolotarev": zolotarev_profile,
    "generic": lambda Ls: generic_profile(Ls, 5),
    "symmetric": lambda Ls: (lambda b, c: (b[:Ls // 2] + b[:Ls // 2][::-1], c[:Ls // 2] + c[:Ls // 2][::-1]))(
        *generic_profile(Ls, 6)),
}


def setup(dims, Ls, prof, mf, seed):
    U = sy.gauge_field(dims, 0.3, 1000 + seed)
    _, odd = oracle.split(sy.gaussian_field(dims, Ls, 2000 + seed), dims)
    b, c = prof
    p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, mf, b5s=tuple(b), c5s=tuple(c))
    return U, odd, p


@pytest.mark.parametrize("name", sorted(PROFILES))
@pytest.mark.parametrize("prec", [F64, F32, F16N])
@pytest.mark.parametrize("dagger", [False, True])
def test_apply_parity_per_slice(name, prec, dagger):
    """4^4, Ls = 8, mf = 0.02: M and M^dag with per-slice coefficients."""
    dims, Ls = (4, 4, 4, 4), 8
    prof = PROFILES[name](Ls)
    U, odd, p = setup(dims, Ls, prof, 0.02, 41)
    ref = oracle.m(odd, U, p, dagger=dagger)
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.02, U) as c:
        mdwf.mdwf_set_s_coefficients(c.h, *prof)
        check(c.apply(odd, prec, dagger)[0], ref, prec)


def test_reset_and_readback():
    """Setting, reading back and resetting the coefficients; a singular I is
    refused and leaves the coefficients in force unchanged."""
    dims, Ls = (4, 4, 2, 4), 6
    prof = cosine_profile(Ls)
    U, odd, p = setup(dims, Ls, prof, 0.03, 42)
    p0 = p.with_(b5s=None, c5s=None)
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.03, U) as c:
        b, cc, per = mdwf.mdwf_get_s_coefficients(c.h, Ls)
        assert not per and b == [1.5] * Ls and cc == [0.5] * Ls
        mdwf.mdwf_set_s_coefficients(c.h, *prof)
        check(c.apply(odd, F64)[0], oracle.m(odd, U, p), F64)
        # M+(s) = M-(s) = 0 for every s (up to rounding) makes I singular
        with pytest.raises(mdwf.MdwfError) as e:
            mdwf.mdwf_set_s_coefficients(c.h, [-1 / 2.2] * Ls, [1 / 2.2] * Ls)
        assert e.value.status == 1
        b, cc, per = mdwf.mdwf_get_s_coefficients(c.h, Ls)
        assert per and np.allclose(b, prof[0]) and np.allclose(cc, prof[1])
        check(c.apply(odd, F64)[0], oracle.m(odd, U, p), F64)
        mdwf.mdwf_set_s_coefficients(c.h, None, None)
        assert not mdwf.mdwf_get_s_coefficients(c.h, Ls)[2]
        check(c.apply(odd, F64)[0], oracle.m(odd, U, p0), F64)


@pytest.mark.parametrize("prec", [F64, F32])
def test_multi_mass_per_slice(prec):
    dims, Ls = (4, 4, 2, 4), 8
    prof = generic_profile(Ls, 7)
    masses = [0.005, 0.03, 0.1]
    U = sy.gauge_field(dims, 0.3, 1043)
    srcs = sy.gaussian_field(dims, Ls, 2043, nrhs=3)
    odd = np.stack([oracle.split(srcs[r], dims)[1] for r in range(3)])
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.01, U) as c:
        mdwf.mdwf_set_s_coefficients(c.h, *prof)
        for dagger in (False, True):
            got = c.apply(odd, prec, dagger, nrhs=3, masses=masses)
            for r, m in enumerate(masses):
                p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, m, b5s=tuple(prof[0]), c5s=tuple(prof[1]))
                check(got[r], oracle.m(odd[r], U, p, dagger=dagger), prec)


@pytest.mark.parametrize("inner", [F64, F32, F16N], ids=["f64", "mixed-f32", "mixed-f16n"])
def test_cgne_per_slice(inner):
    """prepare -> CGNE -> reconstruct to 1e-10 with the cosine profile; the
    oracle checks the normal-equation and the first-order residuals."""
    dims, Ls = (4, 4, 4, 4), 8
    prof = cosine_profile(Ls)
    U = sy.gauge_field(dims, 0.3, 1044)
    b = sy.gaussian_field(dims, Ls, 2044)
    p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, 0.02, b5s=tuple(prof[0]), c5s=tuple(prof[1]))
    h = mdwf.mdwf_create(dims, Ls, 1.8, 1.5, 0.5, 0.02)
    try:
        mdwf.mdwf_set_s_coefficients(h, *prof)
        mdwf.mdwf_load_gauge(h, torch.from_numpy(U).cuda())
        bb = torch.from_numpy(b).cuda()
        x = torch.zeros_like(bb)
        st, info = mdwf.mdwf_cgne(h, x, bb, tol=1e-10, inner_prec=inner)
        assert st == 0 and info[0].true_res <= 1e-10
        xs = x.cpu().numpy()
    finally:
        mdwf.mdwf_destroy(h)
    bp = oracle.prepare(b, U, p)
    src = oracle.m(bp, U, p, dagger=True)
    _, xo = oracle.split(xs, dims)
    assert np.linalg.norm(src - oracle.mdagm(xo, U, p)) / np.linalg.norm(src) <= 1.05e-10
    assert np.linalg.norm(bp - oracle.m(xo, U, p)) / np.linalg.norm(bp) <= 1e-8
    # the reconstructed 5d solution solves D_DW x = b
    r = b - oracle.ddw(xs, U, p)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-7


def test_noalloc_refuses_per_slice():
    dims, Ls = (4, 4, 2, 2), 4
    U = sy.gauge_field(dims, 0.3, 1045)
    _, phi = oracle.split(sy.gaussian_field(dims, Ls, 2045), dims)
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.05, U) as c:
        mdwf.mdwf_set_s_coefficients(c.h, *cosine_profile(Ls))
        a = c.upload(phi, F32)
        out = c.alloc(F32)
        with pytest.raises(mdwf.MdwfError) as e:
            mdwf.mdwf_apply_noalloc(c.h, out, a, F32)
        assert e.value.status == 1


def oracle_action(phi, U, p):
    """S = phi^dag (M^dag M)^-1 phi with the oracle's M^dag M as a dense matrix."""
    A = dense_of(lambda v: oracle.mdagm(v, U, p), phi.size, phi.shape)
    return float(np.real(np.vdot(phi.reshape(-1), np.linalg.solve(A, phi.reshape(-1)))))


def su3_direction(shape, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(shape + (3, 3)) + 1j * rng.standard_normal(shape + (3, 3))
    h = 0.5 * (a - np.conj(np.swapaxes(a, -1, -2)))
    return h - np.trace(h, axis1=-2, axis2=-1)[..., None, None] / 3.0 * np.eye(3)


def expm_ah(w):
    lam, v = np.linalg.eigh(1j * w)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(-1j * lam), np.conj(v))


def gpu_force(dims, Ls, mf, U, phi, prof):
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, mf, U) as c:
        if prof is not None:
            mdwf.mdwf_set_s_coefficients(c.h, *prof)
        G = torch.empty(U.shape, dtype=torch.complex128, device="cuda")
        S, db, dc, st, info = mdwf.mdwf_force(c.h, G, torch.from_numpy(phi).cuda(), tol=1e-13)
        assert st == 0
        return S, G.cpu().numpy(), db, dc


def test_force_per_slice_against_oracle_action():
    """4x2x2x2, Ls = 4, a generic profile: S, dS/dU along a random su(3) direction and
    every dS/db5(s), dS/dc5(s) against central differences (h = 1e-5) of the oracle's
    action S = phi^dag (M^dag M)^-1 phi (dense)."""
    dims, Ls, mf = (4, 2, 2, 2), 4, 0.05
    prof = generic_profile(Ls, 11)
    U = sy.gauge_field(dims, 0.3, 1047)
    _, phi = oracle.split(sy.gaussian_field(dims, Ls, 2047), dims)
    p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, mf, b5s=tuple(prof[0]), c5s=tuple(prof[1]))
    S, G, db, dc = gpu_force(dims, Ls, mf, U, phi, prof)
    assert np.shape(db) == (Ls,) and np.shape(dc) == (Ls,)
    assert S == pytest.approx(oracle_action(phi, U, p), rel=1e-10)
    h = 1e-5
    w = su3_direction(U.shape[:-2], 47)
    fd = (oracle_action(phi, expm_ah(h * w) @ U, p) - oracle_action(phi, expm_ah(-h * w) @ U, p)) / (2 * h)
    an = float(np.sum(np.real(np.conj(G) * (w @ U))))
    assert an == pytest.approx(fd, rel=1e-6)
    for which, got in (("b5s", db), ("c5s", dc)):
        scale = np.abs(got).max()
        for s in range(Ls):
            up, dn = list(getattr(p, which)), list(getattr(p, which))
            up[s] += h
            dn[s] -= h
            fd = (oracle_action(phi, U, p.with_(**{which: tuple(up)})) -
                  oracle_action(phi, U, p.with_(**{which: tuple(dn)}))) / (2 * h)
            assert abs(got[s] - fd) <= 1e-6 * scale, (which, s, got[s], fd)


def test_force_per_slice_sums_to_constant_derivatives():
    """A constant profile set per slice: dS/dU as with constant coefficients, and the
    per-slice derivatives add up to dS/db5 and dS/dc5."""
    dims, Ls, mf = (4, 4, 2, 2), 6, 0.05
    U = sy.gauge_field(dims, 0.3, 1048)
    _, phi = oracle.split(sy.gaussian_field(dims, Ls, 2048), dims)
    S0, G0, db0, dc0 = gpu_force(dims, Ls, mf, U, phi, None)
    S1, G1, db1, dc1 = gpu_force(dims, Ls, mf, U, phi, ([1.5] * Ls, [0.5] * Ls))
    assert S1 == pytest.approx(S0, rel=1e-11)
    assert np.abs(G1 - G0).max() <= 1e-9 * np.abs(G0).max()
    assert float(np.sum(db1)) == pytest.approx(db0, rel=1e-9)
    assert float(np.sum(dc1)) == pytest.approx(dc0, rel=1e-9)


def test_apply_parity_full_16x16x16x32_per_slice():
    """16^3 x 32, Ls = 16, the cosine profile, F32 and F64, M and M^dag."""
    dims, Ls = (16, 16, 16, 32), 16
    prof = cosine_profile(Ls)
    U = sy.gauge_field(dims, 0.2, 1046)
    _, odd = oracle.split(sy.gaussian_field(dims, Ls, 2046), dims)
    p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, 0.01, b5s=tuple(prof[0]), c5s=tuple(prof[1]))
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.01, U) as c:
        mdwf.mdwf_set_s_coefficients(c.h, *prof)
        for d in (False, True):
            ref = oracle.m(odd, U, p, dagger=d)
            for prec in (F64, F32):
                check(c.apply(odd, prec, d)[0], ref, prec)


def test_cgne_multi_mass_per_slice():
    """Three masses in one mixed FP32 solve with per-slice coefficients: the fused
    iteration with one dense table per right-hand side; each solution against the
    oracle's residuals at its own mass."""
    dims, Ls = (4, 4, 2, 4), 8
    prof = generic_profile(Ls, 9)
    masses = [0.01, 0.04, 0.2]
    U = sy.gauge_field(dims, 0.3, 1045)
    b = sy.gaussian_field(dims, Ls, 2045, nrhs=3)
    h = mdwf.mdwf_create(dims, Ls, 1.8, 1.5, 0.5, 0.01)
    try:
        mdwf.mdwf_set_s_coefficients(h, *prof)
        mdwf.mdwf_load_gauge(h, torch.from_numpy(U).cuda())
        bb = torch.from_numpy(np.ascontiguousarray(b)).cuda()
        x = torch.zeros_like(bb)
        st, info = mdwf.mdwf_cgne(h, x, bb, nrhs=3, mf_per_rhs=masses, tol=1e-10, inner_prec=F32)
        assert st == 0 and all(i.true_res <= 1e-10 for i in info)
        xs = x.cpu().numpy()
    finally:
        mdwf.mdwf_destroy(h)
    for r, m in enumerate(masses):
        p = oracle.Params(dims, Ls, 1.8, 1.5, 0.5, m, b5s=tuple(prof[0]), c5s=tuple(prof[1]))
        res = b[r] - oracle.ddw(xs[r], U, p)
        assert np.linalg.norm(res) / np.linalg.norm(b[r]) <= 1e-7, r


@pytest.mark.parametrize("inner", [F64, F32], ids=["f64", "mixed-f32"])
def test_cgne_dense_tables_match_structured(inner):
    """Constant coefficients with the s-operators as dense tables (dense_s) give the
    solve of the structured recursion (the fused iteration with dense epilogues)."""
    dims, Ls = (4, 4, 4, 4), 8
    U = sy.gauge_field(dims, 0.3, 1046)
    b = sy.gaussian_field(dims, Ls, 2046)
    out = []
    for dense in (False, True):
        h = mdwf.mdwf_create(dims, Ls, 1.8, 1.5, 0.5, 0.02, dense_s=dense)
        try:
            mdwf.mdwf_load_gauge(h, torch.from_numpy(U).cuda())
            bb = torch.from_numpy(b).cuda()
            x = torch.zeros_like(bb)
            st, info = mdwf.mdwf_cgne(h, x, bb, tol=1e-11, inner_prec=inner)
            assert st == 0 and info[0].true_res <= 1e-11
            out.append(x.cpu().numpy())
        finally:
            mdwf.mdwf_destroy(h)
    # both stop at 1e-11 in M^dag M: the iterates agree to about cond(M^dag M) x 1e-11
    assert np.linalg.norm(out[0] - out[1]) <= 1e-6 * np.linalg.norm(out[0])
