"""The t-slab domain decomposition on one GPU (loopback): the lattice cut into
n slabs along t, one context per slab, the faces (spin-projected half spinors,
the backward ones transported by the sending slab) delivered between the
stages by device copies. M and M^dag of the slabs, joined, must equal the
oracle's M and M^dag of the whole lattice element by element: FP64 within
1e-12, FP32 within 1e-5 of the largest oracle element, the bars of the
operator tests."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle
import paper_1206_5214_gb300 as mdwf
import synthetic as sy
from paper_1206_5214_gb300 import domain
from _gpu import rel_err

pytestmark = pytest.mark.gpu

F64, F32 = mdwf.MDWF_F64, mdwf.MDWF_F32
TOL = {F64: 1e-12, F32: 1e-5}


def slab_apply(dims, Ls, b5, c5, mf, U, odd, n, prec, dagger, masses=None, mu=0.0, dense_s=False):
    """M (or M^dag) of the odd fields `odd` (nrhs, Ls, Vh, 4, 3) through n slabs."""
    part = domain.SlabPartition(dims, n)
    nrhs = odd.shape[0]
    ctxs, ins, outs = [], [], []
    try:
        for r in range(n):
            h = mdwf.mdwf_create_slab(part.local_dims, Ls, 1.8, b5, c5, mf, dense_s=dense_s)
            ctxs.append(h)
            mdwf.mdwf_load_gauge(h, torch.from_numpy(part.gauge(U, r)).cuda())
            if mu:
                mdwf.mdwf_set_chemical_potential(h, mu)
            nb = mdwf.mdwf_field_bytes(h, prec, nrhs)
            fi = torch.empty(nb, dtype=torch.uint8, device="cuda")
            src = torch.from_numpy(np.ascontiguousarray(part.odd(odd, r))).cuda()
            mdwf.mdwf_field_import(h, fi, src, prec, nrhs)
            ins.append(fi)
            outs.append(torch.empty_like(fi))
        domain.apply_local(mdwf, ctxs, outs, ins, prec, nrhs, masses, dagger)
        got = []
        for r in range(n):
            o = torch.empty((nrhs, Ls, part.vh_local, 4, 3), dtype=torch.complex128, device="cuda")
            mdwf.mdwf_field_export(ctxs[r], o, outs[r], prec, nrhs)
            got.append(o.cpu().numpy())
        torch.cuda.synchronize()
        return part.join_odd(got)
    finally:
        for h in ctxs:
            mdwf.mdwf_destroy(h)


def oracle_m(dims, Ls, b5, c5, masses, U, odd, dagger, mu=0.0):
    return np.stack([oracle.m(odd[r], U, oracle.Params(dims, Ls, 1.8, b5, c5, m, mu=mu), dagger=dagger)
                     for r, m in enumerate(masses)])


@pytest.mark.parametrize("n", [1, 2, 4])
@pytest.mark.parametrize("prec", [F64, F32], ids=["f64", "f32"])
@pytest.mark.parametrize("dagger", [False, True], ids=["M", "Mdag"])
def test_slabs_match_oracle(n, prec, dagger):
    """4^3 x 8, Ls = 8, Moebius b5 = 1.5, c5 = 0.5, two right-hand sides at two masses."""
    dims, Ls = (4, 4, 4, 8), 8
    masses = [0.01, 0.07]
    U = sy.gauge_field(dims, 0.3, 1201)
    b = sy.gaussian_field(dims, Ls, 2201, nrhs=2)
    odd = np.stack([oracle.split(b[r], dims)[1] for r in range(2)])
    got = slab_apply(dims, Ls, 1.5, 0.5, masses[0], U, odd, n, prec, dagger, masses=masses)
    ref = oracle_m(dims, Ls, 1.5, 0.5, masses, U, odd, dagger)
    emax, _ = rel_err(got, ref)
    assert emax <= TOL[prec], emax


@pytest.mark.parametrize("prec", [F64, F32], ids=["f64", "f32"])
def test_slabs_shamir_chemical_potential_dense_tables(prec):
    """Shamir coefficients, a chemical potential on the time links (the halo terms
    carry e^{+-mu}) and dense Ls x Ls tables, 8 slabs of 2 t-slices on 2^3 x 16, Ls = 6."""
    dims, Ls, mu = (2, 2, 2, 16), 6, 0.25
    U = sy.gauge_field(dims, 0.3, 1202)
    odd = oracle.split(sy.gaussian_field(dims, Ls, 2202), dims)[1][None]
    for dagger in (False, True):
        got = slab_apply(dims, Ls, 1.0, 0.0, 0.02, U, odd, 8, prec, dagger, mu=mu, dense_s=True)
        ref = oracle_m(dims, Ls, 1.0, 0.0, [0.02], U, odd, dagger, mu=mu)
        emax, _ = rel_err(got, ref)
        assert emax <= TOL[prec], (dagger, emax)


def test_one_slab_equals_the_whole_lattice_operator():
    """A single slab whose faces wrap onto itself is the periodic lattice: the
    same M as mdwf_apply, to FP64 rounding."""
    dims, Ls = (4, 4, 2, 4), 4
    U = sy.gauge_field(dims, 0.3, 1203)
    odd = oracle.split(sy.gaussian_field(dims, Ls, 2203), dims)[1][None]
    got = slab_apply(dims, Ls, 1.5, 0.5, 0.03, U, odd, 1, F64, False)
    h = mdwf.mdwf_create(dims, Ls, 1.8, 1.5, 0.5, 0.03)
    try:
        mdwf.mdwf_load_gauge(h, torch.from_numpy(U).cuda())
        nb = mdwf.mdwf_field_bytes(h, F64, 1)
        fi = torch.empty(nb, dtype=torch.uint8, device="cuda")
        fo = torch.empty_like(fi)
        mdwf.mdwf_field_import(h, fi, torch.from_numpy(odd).cuda(), F64, 1)
        mdwf.mdwf_apply(h, fo, fi, F64, 1)
        o = torch.empty((1, Ls, 64, 4, 3), dtype=torch.complex128, device="cuda")
        mdwf.mdwf_field_export(h, o, fo, F64, 1)
        ref = o.cpu().numpy()
    finally:
        mdwf.mdwf_destroy(h)
    emax, _ = rel_err(got, ref)
    assert emax <= 1e-13, emax


def test_slab_context_refuses_whole_lattice_calls():
    dims, Ls = (4, 4, 4, 4), 4
    U = sy.gauge_field((4, 4, 4, 8), 0.3, 1204)
    part = domain.SlabPartition((4, 4, 4, 8), 2)
    h = mdwf.mdwf_create_slab(dims, Ls, 1.8, 1.5, 0.5, 0.01)
    try:
        mdwf.mdwf_load_gauge(h, torch.from_numpy(part.gauge(U, 0)).cuda())
        nb = mdwf.mdwf_field_bytes(h, F32, 1)
        a = torch.zeros(nb, dtype=torch.uint8, device="cuda")
        b = torch.zeros_like(a)
        with pytest.raises(mdwf.MdwfError) as e:
            mdwf.mdwf_apply(h, b, a, F32, 1)
        assert e.value.status == mdwf.MDWF_EINVAL
        assert mdwf.mdwf_slab_face_bytes(h, mdwf.MDWF_F16N, 1) == 0
        with pytest.raises(mdwf.MdwfError):
            mdwf.mdwf_slab_stage(h, 0, None, a, mdwf.MDWF_F16N, 1, send=b)
    finally:
        mdwf.mdwf_destroy(h)
    # and an ordinary context refuses the stages
    h = mdwf.mdwf_create((4, 4, 4, 8), Ls, 1.8, 1.5, 0.5, 0.01)
    try:
        with pytest.raises(mdwf.MdwfError):
            mdwf.mdwf_slab_stage(h, 0, None, a, F32, 1, send=b)
    finally:
        mdwf.mdwf_destroy(h)
