"""Host logic of bench.py for N > 1 ranks, as two gloo processes on the CPU:
every rank draws its own inputs of the same shape (weak scaling, no
data-path collective) and the step time is the maximum over ranks."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    wl = bench.Workload("plain", "popc", rank=rank)
    digest = int(np.bitwise_xor.reduce(wl.images[0].view(np.uint64).ravel()) & 0x7fffffff)
    ms = bench.max_over_ranks(1.5 + rank, dist, "cpu")
    q.put((rank, wl.n, wl.descriptors_per_step, wl.pairs_per_step, digest, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_weak_scaling_host_logic():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, n0, d0, p0, h0, m0), (r1, n1, d1, p1, h1, m1) = res
    assert (n0, d0, p0) == (n1, d1, p1) == (2000, 4000, 2 * 1000 * 1000)  # same shape per rank
    assert h0 != h1                    # independent inputs
    assert m0 == m1 == 2.5             # the slowest rank's time on every rank
