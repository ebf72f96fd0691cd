"""Host logic of the N > 1 bench path, run as world-size-2 gloo ranks on the CPU.

The single-instance path runs replicas (one per rank, no data-path collective); the
batched path gives each rank a contiguous slice of the instance list.  What crosses
ranks is only the timing reduction: max of the step time, sum of the converged
null vectors.
"""

import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [120.0, 95.5][rank]
        units = [500.0, 498.0][rank]
        t, u = bench.reduce_over_ranks(ms, units, dist, "cpu")
        dist.barrier()
        q.put((rank, t, u, bench.rank_slice(4096, world, rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_slice():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, t, u, _ in out:
        assert t == 120.0 and u == 998.0  # max time, summed units: every rank agrees
    assert out[0][3] == (0, 2048) and out[1][3] == (2048, 4096)


@pytest.mark.parametrize("count,world", [(4096, 1), (4096, 3), (7, 4), (1, 2)])
def test_rank_slices_partition_the_instances(count, world):
    slices = [bench.rank_slice(count, world, r) for r in range(world)]
    covered = [i for lo, hi in slices for i in range(lo, hi)]
    assert covered == list(range(count))
    sizes = [hi - lo for lo, hi in slices]
    assert max(sizes) - min(sizes) <= 1


def test_single_rank_reduction_is_identity():
    assert bench.reduce_over_ranks(12.5, 3.0, None, "cpu") == (12.5, 3.0)
