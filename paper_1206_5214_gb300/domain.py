"""Domain decomposition of the lattice along t: the host side.

The library applies M on one t-slab at a time (mdwf_create_slab,
mdwf_slab_stage); this module holds what the host does around it:

* the partition (:class:`SlabPartition`): slab r of n holds the global
  t-slices r T/n .. (r+1) T/n - 1; T/n is even, so that the even/odd parity
  of a site is the same in the slab as in the whole lattice, and the odd
  sites of slab r (user order, t slowest) are one contiguous block of the
  lattice's odd sites;
* the face delivery between the stages of an application: face 0 of slab r
  goes to slab r - 1, face 1 to slab r + 1 (periodic). :func:`deliver_local`
  does it with device copies for slabs that live in one process (several
  slabs on one GPU), :func:`exchange` with point-to-point messages of
  torch.distributed for one slab per rank (NCCL for device tensors across
  GPUs, gloo for host tensors);
* :func:`apply_local`, the three stages with the deliveries between them.

Only the 4d hopping term couples slabs (Sec. 3: the Ls x Ls factors are
site-local), so the fifth dimension is never split.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

FACE_TAGS = (11, 12)  # message tags of face 0 and face 1 (transports that match by tag)


@dataclass(frozen=True)
class SlabPartition:
    dims: tuple  # (X, Y, Z, T) of the whole lattice
    n: int       # slabs along t

    def __post_init__(self):
        X, Y, Z, T = self.dims
        if self.n < 1 or T % self.n:
            raise ValueError(f"T = {T} does not split into {self.n} slabs")
        tl = T // self.n
        if tl < 2 or tl % 2:
            raise ValueError(f"each slab needs an even number >= 2 of t-slices, got {tl}")

    @property
    def local_dims(self) -> tuple:
        X, Y, Z, T = self.dims
        return (X, Y, Z, T // self.n)

    @property
    def vh_local(self) -> int:
        X, Y, Z, T = self.local_dims
        return X * Y * Z * T // 2

    def t_range(self, r: int) -> tuple:
        tl = self.local_dims[3]
        return (r * tl, (r + 1) * tl)

    def below(self, r: int) -> int:
        return (r - 1) % self.n

    def above(self, r: int) -> int:
        return (r + 1) % self.n

    # ---------------------------------------------------------- splitting
    def gauge(self, U: np.ndarray, r: int) -> np.ndarray:
        """The slab's links: U (T, Z, Y, X, 4, 3, 3) restricted to its t-slices."""
        t0, t1 = self.t_range(r)
        return np.ascontiguousarray(U[t0:t1])

    def odd(self, f, r: int):
        """The slab's part of an odd field in user order, (..., Ls, Vh, 4, 3): a
        contiguous block of sites (numpy array or torch tensor)."""
        v = self.vh_local
        return f[..., r * v:(r + 1) * v, :, :]

    def join_odd(self, parts: list) -> np.ndarray:
        return np.concatenate(parts, axis=-3)


def deliver_local(sends: list, recvs: list) -> None:
    """Face delivery for slabs in one process: send buffers (torch tensors of
    mdwf_slab_face_bytes bytes, [face 0 | face 1]) into the neighbours' receive
    buffers, as device copies on the current stream."""
    n = len(sends)
    for r in range(n):
        half = sends[r].numel() // 2
        recvs[(r - 1) % n][:half].copy_(sends[r][:half])
        recvs[(r + 1) % n][half:].copy_(sends[r][half:])


def exchange(send, recv, rank: int, world: int, dist, group=None) -> None:
    """Face delivery with one slab per rank: face 0 of this rank's send to rank - 1,
    face 1 to rank + 1; recv face 0 from rank + 1, face 1 from rank - 1.

    Every rank posts its two sends and then its two receives in the same
    order (face 0, face 1), with the faces' tags, so that transports that
    match by order (NCCL) and by tag (gloo) pair them the same way, also for
    two ranks, where both neighbours are the same rank.
    """
    if world == 1:  # one slab: both faces wrap around onto itself
        recv.copy_(send)
        return
    half = send.numel() // 2
    below, above = (rank - 1) % world, (rank + 1) % world
    if send.is_cuda:
        ops = [dist.P2POp(dist.isend, send[:half], below, group),
               dist.P2POp(dist.isend, send[half:], above, group),
               dist.P2POp(dist.irecv, recv[:half], above, group),
               dist.P2POp(dist.irecv, recv[half:], below, group)]
        for w in dist.batch_isend_irecv(ops):
            w.wait()
        return
    reqs = [dist.isend(send[:half].contiguous(), below, group=group, tag=FACE_TAGS[0]),
            dist.isend(send[half:].contiguous(), above, group=group, tag=FACE_TAGS[1])]
    r0 = recv[:half]
    r1 = recv[half:]
    reqs.append(dist.irecv(r0, above, group=group, tag=FACE_TAGS[0]))
    reqs.append(dist.irecv(r1, below, group=group, tag=FACE_TAGS[1]))
    for q in reqs:
        q.wait()


def apply_local(mdwf, ctxs: list, outs: list, ins: list, prec: int, nrhs: int = 1, masses=None,
                dagger: bool = False, faces=None) -> list:
    """out_r = M in_r (or M^dag) on every slab of one process, slabs r = 0..n-1
    in order, with the faces delivered between the stages. faces: optional
    [(send, recv)] per slab (device tensors), allocated when not given."""
    import torch
    n = len(ctxs)
    if faces is None:
        nb = mdwf.mdwf_slab_face_bytes(ctxs[0], prec, nrhs)
        faces = [(torch.empty(nb, dtype=torch.uint8, device="cuda"), torch.empty(nb, dtype=torch.uint8, device="cuda"))
                 for _ in range(n)]
    sends = [f[0] for f in faces]
    recvs = [f[1] for f in faces]
    for r in range(n):
        mdwf.mdwf_slab_stage(ctxs[r], 0, None, ins[r], prec, nrhs, masses, dagger, send=sends[r])
    deliver_local(sends, recvs)
    for r in range(n):
        mdwf.mdwf_slab_stage(ctxs[r], 1, None, None, prec, nrhs, masses, dagger, send=sends[r], recv=recvs[r])
    deliver_local(sends, recvs)
    for r in range(n):
        mdwf.mdwf_slab_stage(ctxs[r], 2, outs[r], ins[r], prec, nrhs, masses, dagger, recv=recvs[r])
    return faces
