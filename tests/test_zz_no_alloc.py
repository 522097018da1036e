"""mdwf_apply_noalloc against mdwf_apply.

The allocation-free entry point serves callers that must not allocate device
memory while they run (a framework's pool owns all memory, a latency-critical
path, a fixed footprint). It must give the same M and M^dag as mdwf_apply on
consecutive calls, since its fixed scratch keeps the previous call's contents.
This file is collected last so that a failure here never hides another test.
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

TOL = {mdwf.MDWF_F64: 1e-12, mdwf.MDWF_F32: 1e-5}


@pytest.mark.parametrize("prec", [mdwf.MDWF_F64, mdwf.MDWF_F32])
def test_noalloc_apply_matches_apply_twice(prec):
    dims, Ls = (4, 4, 4, 4), 8
    masses = [0.01, 0.04]
    U = sy.gauge_field(dims, 0.3, 1021)
    srcs = sy.gaussian_field(dims, Ls, 2021, nrhs=2)
    odd = np.stack([oracle.split(srcs[r], dims)[1] for r in range(2)])
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.01, U) as c:
        fin = c.upload(odd, prec, nrhs=2)
        ref = c.alloc(prec, nrhs=2)
        got = c.alloc(prec, nrhs=2)
        for dagger in (False, True, False, True):  # two calls of each in a row
            (mdwf.mdwf_apply_dag if dagger else mdwf.mdwf_apply)(c.h, ref, fin, prec, 2, masses)
            got.fill_(0)
            mdwf.mdwf_apply_noalloc(c.h, got, fin, prec, 2, masses, dagger=dagger)
            torch.cuda.synchronize()
            a = c.download(got, prec, nrhs=2)
            b = c.download(ref, prec, nrhs=2)
            emax, _ = rel_err(a, b)
            assert emax <= TOL[prec], (dagger, emax)


def test_noalloc_rejects_fields_beyond_the_fixed_scratch():
    dims, Ls = (16, 16, 16, 16), 16  # one FP32 field = 6 MiB x nrhs
    U = sy.gauge_field(dims, 0.2, 1022)
    with Ctx(dims, Ls, 1.8, 1.5, 0.5, 0.01, U) as c:
        nb = mdwf.mdwf_field_bytes(c.h, mdwf.MDWF_F32, 2)
        assert nb > 8 << 20
        a = torch.zeros(nb, dtype=torch.uint8, device="cuda")
        b = torch.zeros_like(a)
        with pytest.raises(mdwf.MdwfError) as e:
            mdwf.mdwf_apply_noalloc(c.h, b, a, mdwf.MDWF_F32, 2)
        assert e.value.status == 1 and "8 MiB" in str(e.value)
