"""The seeded input recipe (synthetic/): links U = exp(i eps H) with H Gaussian,
traceless and Hermitian, so U is unitary with det U = 1 to FP64 rounding and
within O(eps) of the identity; Gaussian sources with N(0, 1) real components;
point sources placed on the walls; seeds that reproduce the same arrays."""
import numpy as np

import synthetic as sy


def test_links_are_special_unitary():
    U = sy.gauge_field((4, 4, 2, 2), 0.2, 1002).reshape(-1, 3, 3)
    eye = np.eye(3)
    uu = np.einsum("nij,nkj->nik", U, np.conj(U))
    assert np.abs(uu - eye).max() < 1e-13
    assert np.abs(np.linalg.det(U) - 1.0).max() < 1e-13


def test_links_near_identity_scale_with_eps():
    d = {}
    for eps in (0.05, 0.2, 0.8):
        U = sy.gauge_field((4, 2, 2, 2), eps, 7).reshape(-1, 3, 3)
        d[eps] = np.sqrt((np.abs(U - np.eye(3)) ** 2).sum(axis=(1, 2))).mean()
    assert d[0.05] < d[0.2] < d[0.8]
    # for small eps, U - 1 ~ i eps H: the mean distance grows linearly with eps
    assert 3.8 < d[0.2] / d[0.05] < 4.05


def test_generator_of_the_links_is_traceless_hermitian():
    """log U / (i eps) recovers H: Hermitian with zero trace."""
    eps = 0.3
    U = sy.gauge_field((2, 2, 2, 2), eps, 11).reshape(-1, 3, 3)
    w, v = np.linalg.eig(U)
    H = np.einsum("nij,nj,njk->nik", v, np.angle(w) / eps, np.linalg.inv(v))
    assert np.abs(H - np.conj(np.swapaxes(H, 1, 2))).max() < 1e-10
    assert np.abs(np.trace(H, axis1=1, axis2=2)).max() < 1e-10


def test_seeds_reproduce_and_separate():
    a = sy.gauge_field((2, 2, 2, 2), 0.2, 5)
    assert np.array_equal(a, sy.gauge_field((2, 2, 2, 2), 0.2, 5))
    assert not np.array_equal(a, sy.gauge_field((2, 2, 2, 2), 0.2, 6))
    f = sy.gaussian_field((2, 2, 2, 2), 4, 9)
    assert np.array_equal(f, sy.gaussian_field((2, 2, 2, 2), 4, 9))
    assert sy.config_seed("gauge", 2) == 1002 and sy.config_seed("source", 2) == 2002
    assert sy.config_seed("transform", 5) == 3005


def test_gaussian_components():
    f = sy.gaussian_field((8, 8, 4, 4), 8, 2002)
    x = np.concatenate([f.real.ravel(), f.imag.ravel()])
    assert x.size == 2 * 8 * 8 * 8 * 4 * 4 * 12
    assert abs(x.mean()) < 0.02 and abs(x.var() - 1.0) < 0.02
    assert abs(np.mean(f.real * f.imag)) < 0.02
    b = sy.gaussian_field((2, 2, 2, 2), 4, 3, nrhs=3)
    assert b.shape == (3, 4, 2, 2, 2, 2, 4, 3)


def test_point_sources_on_the_walls():
    Ls = 6
    b = sy.point_sources((4, 2, 2, 2), Ls, origin=(1, 0, 1, 0))
    assert b.shape == (12, Ls, 2, 2, 2, 4, 4, 3)
    assert np.count_nonzero(b) == 12 and np.all(b[b != 0] == 1.0)
    for k in range(12):
        spin, col = divmod(k, 3)
        s = 0 if spin >= 2 else Ls - 1
        assert b[k, s, 0, 1, 0, 1, spin, col] == 1.0


def test_unit_gauge_and_transform():
    U = sy.unit_gauge((2, 2, 2, 2)).reshape(-1, 3, 3)
    assert np.array_equal(U, np.broadcast_to(np.eye(3), U.shape))
    g = sy.gauge_transform((2, 2, 2, 2), 3001).reshape(-1, 3, 3)
    assert np.abs(np.einsum("nij,nkj->nik", g, np.conj(g)) - np.eye(3)).max() < 1e-13
    assert np.abs(np.linalg.det(g) - 1.0).max() < 1e-13


def test_device_generators_match_the_host_recipe():
    """The torch-side draws used for the largest batched workloads: the same
    shapes and distribution as the host recipe, reproducible by seed, and the
    same placement of the point sources."""
    torch = __import__("pytest").importorskip("torch")
    f = sy.gaussian_field_device((8, 8, 4, 4), 8, 2005, nrhs=2, device="cpu")
    assert f.shape == (2, 8, 4, 4, 8, 8, 4, 3) and f.dtype == torch.complex128
    x = torch.cat([f.real.ravel(), f.imag.ravel()]).numpy()
    assert abs(x.mean()) < 0.02 and abs(x.var() - 1.0) < 0.02
    assert torch.equal(f, sy.gaussian_field_device((8, 8, 4, 4), 8, 2005, nrhs=2, device="cpu"))
    assert not torch.equal(f, sy.gaussian_field_device((8, 8, 4, 4), 8, 2006, nrhs=2, device="cpu"))
    b = sy.point_sources_device((4, 2, 2, 2), 6, origin=(1, 0, 1, 0), device="cpu")
    assert np.array_equal(b.numpy(), sy.point_sources((4, 2, 2, 2), 6, origin=(1, 0, 1, 0)))
