"""Host side of the t-slab domain decomposition, on the CPU: the partition of
the lattice into slabs, the split and join of links and odd fields, and the
face exchange between ranks over gloo (world sizes 1, 2 and 3), each rank
holding one slab's face buffers. The device side (the faces' contents and the
halo terms of the hops) is checked against the oracle by tests/test_gpu_slabs.py."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1206_5214_gb300 import domain  # noqa: E402


def test_partition_rules():
    p = domain.SlabPartition((4, 4, 4, 16), 4)
    assert p.local_dims == (4, 4, 4, 4) and p.vh_local == 128
    assert [p.t_range(r) for r in range(4)] == [(0, 4), (4, 8), (8, 12), (12, 16)]
    assert (p.below(0), p.above(3)) == (3, 0)
    for dims, n in (((4, 4, 4, 12), 4), ((4, 4, 4, 8), 3), ((4, 4, 4, 8), 8), ((4, 4, 4, 8), 0)):
        with pytest.raises(ValueError):
            domain.SlabPartition(dims, n)  # odd, uneven, 1-slice or no slabs


def test_split_and_join_follow_the_t_coordinate():
    """The odd sites of slab r (user order: checkerboard index with t slowest)
    are the lattice's odd sites whose t lies in the slab; links split by t."""
    X, Y, Z, T = dims = (4, 2, 2, 8)
    p = domain.SlabPartition(dims, 2)
    Vh = X * Y * Z * T // 2
    # t-coordinate of every odd site from the checkerboard index
    t_of = np.arange(Vh) // (X * Y * Z // 2)
    f = np.broadcast_to(t_of[None, :, None, None], (3, Vh, 4, 3)).astype(np.complex128)
    for r in range(2):
        t0, t1 = p.t_range(r)
        blk = p.odd(f, r)
        assert blk.shape == (3, p.vh_local, 4, 3)
        assert np.all((blk.real >= t0) & (blk.real < t1))
    assert np.array_equal(p.join_odd([p.odd(f, 0), p.odd(f, 1)]), f)
    U = np.arange(T * Z * Y * X * 4 * 9, dtype=np.complex128).reshape(T, Z, Y, X, 4, 3, 3)
    assert np.array_equal(np.concatenate([p.gauge(U, 0), p.gauge(U, 1)]), U)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _pattern(rank, face, n):
    return torch.full((n,), 16 * rank + face + 1, dtype=torch.uint8)


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_1206_5214_gb300 import domain as dm
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        half = 96
        send = torch.cat([_pattern(rank, 0, half), _pattern(rank, 1, half)])
        recv = torch.zeros(2 * half, dtype=torch.uint8)
        for _ in range(2):  # two exchanges in a row, as between the stages of one M
            recv.zero_()
            dm.exchange(send, recv, rank, world, dist)
        q.put((rank, recv[:half].tolist(), recv[half:].tolist()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_face_exchange_gloo(world):
    """Face 0 of rank r arrives at rank r - 1, face 1 at rank r + 1 (periodic)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, f0, f1 in res:
        assert f0 == _pattern((rank + 1) % world, 0, 96).tolist(), rank
        assert f1 == _pattern((rank - 1) % world, 1, 96).tolist(), rank


def test_face_exchange_single_slab_and_local_delivery():
    """One slab wraps onto itself; slabs of one process deliver by copies."""
    send = torch.cat([_pattern(0, 0, 8), _pattern(0, 1, 8)])
    recv = torch.zeros(16, dtype=torch.uint8)
    domain.exchange(send, recv, 0, 1, None)
    assert torch.equal(recv, send)
    sends = [torch.cat([_pattern(r, 0, 8), _pattern(r, 1, 8)]) for r in range(3)]
    recvs = [torch.zeros(16, dtype=torch.uint8) for _ in range(3)]
    domain.deliver_local(sends, recvs)
    for r in range(3):
        assert torch.equal(recvs[r][:8], _pattern((r + 1) % 3, 0, 8))
        assert torch.equal(recvs[r][8:], _pattern((r - 1) % 3, 1, 8))
