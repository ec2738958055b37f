"""The N > 1 path of bench.py's measurement (replicas only: one process per
GPU, no collective in the data path) with two gloo ranks on the CPU: the
timed region's barrier, the max over ranks and the whole-job throughput."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    t = bench.max_over_ranks(times[rank], world)
    e = bench.max_over_ranks(times[rank] / 2, world)
    out[rank] = (t, e, bench.job_throughput(world, 1000, 10, t))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("times", [(3.0, 5.0), (7.5, 2.25)])
def test_max_over_two_gloo_ranks(times):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(2, _free_port(), times, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    slow = max(times)
    for r in range(2):
        t, e, v = res[r]
        assert t == slow and e == slow / 2
        assert v == pytest.approx(2 * 1000 * 10 / (slow * 1e-3))


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(4.5, 1) == 4.5
    assert bench.job_throughput(1, 5, 2, 1.0) == pytest.approx(10_000.0)
