"""mdwf_apply_noalloc: the allocation-free M and M^dag.

Some callers cannot call cudaMalloc while they run: a custom operator inside a
framework whose caching pool owns all device memory, a latency-critical path
that must not enter the driver's allocator (which can synchronise the device),
or a service whose device footprint must stay fixed after set-up. For them the
library has one entry point that allocates nothing: its intermediate fields
live in a fixed static device array. These tests check it through the C ABI
against the FP64 oracle, call it twice in a row (the array keeps the previous
call's contents), call it on a fresh context before anything else has built
the context's tables or workspaces, check that repeated calls leave the free
device memory unchanged, and check its argument errors.

This file is collected last, so that a failure here never hides another test;
it passes alone in a fresh process as well as after the other tests.
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

F64, F32, F16N = mdwf.MDWF_F64, mdwf.MDWF_F32, mdwf.MDWF_F16N
# the bars of the operator parity tests: max element error relative to the
# largest oracle element (FP64, FP32), 2-norm relative error for FP16 storage
TOL_MAX = {F64: 1e-12, F32: 1e-5}
TOL_L2_F16N = 3e-3

DIMS, LS, M5, B5, C5, MF = (4, 4, 4, 4), 8, 1.8, 1.5, 0.5, 0.01


def _inputs(nrhs, seed):
    U = sy.gauge_field(DIMS, 0.3, 1000 + seed)
    srcs = sy.gaussian_field(DIMS, LS, 2000 + seed, nrhs=nrhs)
    odd = np.stack([oracle.split(srcs[r], DIMS)[1] for r in range(nrhs)])
    return U, odd


def _oracle(odd, U, masses, dagger):
    return np.stack([oracle.m(odd[r], U, oracle.Params(DIMS, LS, M5, B5, C5, m), dagger=dagger)
                     for r, m in enumerate(masses)])


def _check(prec, got, ref):
    emax, el2 = rel_err(got, ref)
    if prec == F16N:
        assert el2 <= TOL_L2_F16N, (emax, el2)
    else:
        assert emax <= TOL_MAX[prec], (emax, el2)


@pytest.mark.parametrize("prec", [F64, F32, F16N])
def test_noalloc_first_on_a_fresh_context_matches_oracle(prec):
    """The first call on a fresh context (no mdwf_apply before it, masses that
    differ from the context's mf), then a second call of each kind in a row."""
    masses = [0.02, 0.05]
    U, odd = _inputs(2, 31)
    with Ctx(DIMS, LS, M5, B5, C5, MF, U) as c:
        fin = c.upload(odd, prec, nrhs=2)
        got = c.alloc(prec, nrhs=2)
        for dagger in (False, False, True, True):
            got.fill_(0)
            mdwf.mdwf_apply_noalloc(c.h, got, fin, prec, 2, masses, dagger=dagger)
            torch.cuda.synchronize()
            _check(prec, c.download(got, prec, nrhs=2), _oracle(odd, U, masses, dagger))


@pytest.mark.parametrize("prec", [F64, F32])
def test_noalloc_matches_apply_on_consecutive_calls(prec):
    """Interleaved with mdwf_apply on the same context: the same result as the
    allocating entry point, call after call."""
    masses = [0.01, 0.04]
    U, odd = _inputs(2, 21)
    with Ctx(DIMS, LS, M5, B5, C5, MF, U) as c:
        fin = c.upload(odd, prec, nrhs=2)
        ref = c.alloc(prec, nrhs=2)
        got = c.alloc(prec, nrhs=2)
        for dagger in (False, True, False, True):
            (mdwf.mdwf_apply_dag if dagger else mdwf.mdwf_apply)(c.h, ref, fin, prec, 2, masses)
            got.fill_(0)
            mdwf.mdwf_apply_noalloc(c.h, got, fin, prec, 2, masses, dagger=dagger)
            torch.cuda.synchronize()
            emax, _ = rel_err(c.download(got, prec, nrhs=2), c.download(ref, prec, nrhs=2))
            assert emax <= TOL_MAX[prec], (dagger, emax)


def test_noalloc_leaves_free_device_memory_unchanged():
    """After the first call (which looks up the static array's address), further
    calls change the device's free memory by nothing."""
    U, odd = _inputs(1, 41)
    with Ctx(DIMS, LS, M5, B5, C5, MF, U) as c:
        fin = c.upload(odd, F32)
        got = c.alloc(F32)
        mdwf.mdwf_apply_noalloc(c.h, got, fin, F32, 1, [0.03])
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for k in range(6):
            mdwf.mdwf_apply_noalloc(c.h, got, fin, F32, 1, [0.03 + 0.01 * k], dagger=bool(k & 1))
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (free0, free1)
        _check(F32, c.download(got, F32), _oracle(odd, U, [0.08], True))


def test_noalloc_rejects_fields_beyond_the_fixed_scratch():
    dims, Ls = (16, 16, 16, 16), 16  # one FP32 field = 6 MiB x nrhs
    U = sy.gauge_field(dims, 0.2, 1022)
    with Ctx(dims, Ls, M5, B5, C5, MF, U) as c:
        nb = mdwf.mdwf_field_bytes(c.h, F32, 2)
        assert nb > 8 << 20
        a = torch.zeros(nb, dtype=torch.uint8, device="cuda")
        b = torch.zeros_like(a)
        with pytest.raises(mdwf.MdwfError) as e:
            mdwf.mdwf_apply_noalloc(c.h, b, a, F32, 2)
        assert e.value.status == mdwf.MDWF_EINVAL and "8 MiB" in str(e.value)


def test_noalloc_rejects_non_finite_and_singular_masses():
    U, odd = _inputs(1, 51)
    with Ctx(DIMS, LS, M5, B5, C5, MF, U) as c:
        fin = c.upload(odd, F32)
        got = c.alloc(F32)
        with pytest.raises(mdwf.MdwfError) as e:
            mdwf.mdwf_apply_noalloc(c.h, got, fin, F32, 1, [float("nan")])
        assert e.value.status == mdwf.MDWF_EINVAL and "finite" in str(e.value)
    # Shamir-type coefficients with M+ = 1.25, M- = -1: r = M-/M+ = -0.8 keeps
    # the closed form, and det I = M+^Ls (1 + m (-r)^Ls) vanishes at m = -0.8^-Ls
    b5 = 0.25 / (4 - M5)
    m_sing = -1.0 / 0.8 ** LS
    with Ctx(DIMS, LS, M5, b5, 0.0, MF, U) as c:
        fin = c.upload(odd, F32)
        got = c.alloc(F32)
        with pytest.raises(mdwf.MdwfError) as e:
            mdwf.mdwf_apply_noalloc(c.h, got, fin, F32, 1, [m_sing])
        assert e.value.status == mdwf.MDWF_EINVAL and "singular" in str(e.value)
        # a regular mass on the same context still works
        mdwf.mdwf_apply_noalloc(c.h, got, fin, F32, 1, [0.1])
        torch.cuda.synchronize()
        ref = oracle.m(odd[0], U, oracle.Params(DIMS, LS, M5, b5, 0.0, 0.1))
        _check(F32, c.download(got, F32), ref[None])
