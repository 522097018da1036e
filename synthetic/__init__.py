"""Seeded synthetic inputs for the Moebius domain-wall operator.

This module only *draws* inputs. It holds none of the operator's arithmetic:
no Wilson hopping, no fifth-dimension coupling, no Schur complement. The CPU
oracle, the GPU tests and the benchmark all consume the arrays made here, so
the two sides are fed identical data.

Conventions (shared data formats, not arithmetic):

* lattice ``dims = (X, Y, Z, T)``; directions mu = 0..3 are x, y, z, t.
* gauge field ``U``: complex128, shape ``(T, Z, Y, X, 4, 3, 3)``;
  ``U[t, z, y, x, mu]`` is the link U_mu(x) from x to x + mu (row-major 3x3).
* 5d fermion field: complex128, shape ``(Ls, T, Z, Y, X, 4, 3)``
  (``[s][t][z][y][x][spin][colour]``); a batch of ``nrhs`` fields prepends an
  axis. Spin components 0, 1 are the gamma5 = +1 (P+) half and 2, 3 the
  gamma5 = -1 (P-) half of the chiral basis both sides use.
* gauge transformation ``Omega``: complex128, shape ``(T, Z, Y, X, 3, 3)``.

Links follow the recipe U = exp(i eps H) with H a Gaussian traceless Hermitian
3x3 matrix (entries of A complex normal, H = (A + A^dag)/2 - tr/3), built by
eigen-decomposition, and are not re-unitarised afterwards.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "config_seed",
    "su3_near_identity",
    "gauge_field",
    "gauge_transform",
    "gaussian_field",
    "point_sources",
    "unit_gauge",
    "gaussian_field_device",
    "point_sources_device",
]


def config_seed(kind: str, cfg: int) -> int:
    """Seed of input ``kind`` for configuration number ``cfg`` (1-based).

    gauge = 1000 + cfg, source = 2000 + cfg, transform = 3000 + cfg.
    """
    base = {"gauge": 1000, "source": 2000, "transform": 3000}[kind]
    return base + int(cfg)


def su3_near_identity(n: int, eps: float, rng: np.random.Generator) -> np.ndarray:
    """``n`` matrices exp(i eps H), H Gaussian traceless Hermitian; shape (n, 3, 3)."""
    a = rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1).real / 3.0
    h = h - tr[:, None, None] * np.eye(3)[None]
    w, v = np.linalg.eigh(h)
    phase = np.exp(1j * eps * w)
    return np.einsum("nij,nj,nkj->nik", v, phase, np.conj(v))


def _vol(dims) -> int:
    x, y, z, t = (int(d) for d in dims)
    return x * y * z * t


def gauge_field(dims, eps: float, seed: int) -> np.ndarray:
    """Random SU(3) links near the identity, shape (T, Z, Y, X, 4, 3, 3)."""
    x, y, z, t = (int(d) for d in dims)
    rng = np.random.default_rng(seed)
    u = su3_near_identity(_vol(dims) * 4, eps, rng)
    return np.ascontiguousarray(u.reshape(t, z, y, x, 4, 3, 3))


def unit_gauge(dims) -> np.ndarray:
    """The free field U_mu(x) = 1."""
    x, y, z, t = (int(d) for d in dims)
    u = np.zeros((t, z, y, x, 4, 3, 3), dtype=np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1.0
    return u


def gauge_transform(dims, seed: int) -> np.ndarray:
    """Random SU(3) matrix per site (the link recipe with eps = 1), shape (T, Z, Y, X, 3, 3)."""
    x, y, z, t = (int(d) for d in dims)
    rng = np.random.default_rng(seed)
    g = su3_near_identity(_vol(dims), 1.0, rng)
    return np.ascontiguousarray(g.reshape(t, z, y, x, 3, 3))


def gaussian_field(dims, Ls: int, seed: int, nrhs: int | None = None) -> np.ndarray:
    """5d field with every real component drawn N(0, 1).

    Shape (Ls, T, Z, Y, X, 4, 3), or (nrhs, Ls, ...) when ``nrhs`` is given.
    """
    x, y, z, t = (int(d) for d in dims)
    rng = np.random.default_rng(seed)
    shape = (Ls, t, z, y, x, 4, 3) if nrhs is None else (nrhs, Ls, t, z, y, x, 4, 3)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return re + 1j * im


def point_sources(dims, Ls: int, origin=(0, 0, 0, 0)) -> np.ndarray:
    """The 12 spin x colour point sources at ``origin`` placed on the walls.

    Source k = 3 * spin + colour is a unit delta in (spin, colour) at the 4d
    site ``origin = (x, y, z, t)``. It is placed on the domain walls the way
    the 4d quark field lives there: its gamma5 = -1 spin half (spins 2, 3) on
    slice s = 0 and its gamma5 = +1 half (spins 0, 1) on slice s = Ls - 1.
    This is a placement of unit entries, nothing is computed.
    Shape (12, Ls, T, Z, Y, X, 4, 3).
    """
    x, y, z, t = (int(d) for d in dims)
    ox, oy, oz, ot = origin
    b = np.zeros((12, Ls, t, z, y, x, 4, 3), dtype=np.complex128)
    for spin in range(4):
        for col in range(3):
            k = 3 * spin + col
            s = 0 if spin >= 2 else Ls - 1
            b[k, s, ot, oz, oy, ox, spin, col] = 1.0
    return b


def gaussian_field_device(dims, Ls: int, seed: int, nrhs: int, device="cuda"):
    """A batch of ``nrhs`` Gaussian 5d fields drawn on ``device`` by torch's
    seeded generator (every real component N(0, 1)), for workloads whose
    host-side draw would take minutes (tens of GB). Same shape and
    distribution as :func:`gaussian_field`, a different stream of numbers.
    Shape (nrhs, Ls, T, Z, Y, X, 4, 3), complex128.
    """
    import torch
    x, y, z, t = (int(d) for d in dims)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    re_im = torch.randn((nrhs, Ls, t, z, y, x, 4, 3, 2), dtype=torch.float64, device=device, generator=g)
    return torch.view_as_complex(re_im)


def point_sources_device(dims, Ls: int, origin=(0, 0, 0, 0), device="cuda"):
    """:func:`point_sources` built directly in device memory (a torch tensor)."""
    import torch
    x, y, z, t = (int(d) for d in dims)
    ox, oy, oz, ot = origin
    b = torch.zeros((12, Ls, t, z, y, x, 4, 3), dtype=torch.complex128, device=device)
    for spin in range(4):
        for col in range(3):
            s = 0 if spin >= 2 else Ls - 1
            b[3 * spin + col, s, ot, oz, oy, ox, spin, col] = 1.0
    return b
