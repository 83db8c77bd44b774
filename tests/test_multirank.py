"""Host logic of the multi-GPU (replica) benchmark path on CPU: two gloo ranks
with different step times; the job throughput uses every rank's pixels over the
slowest rank's time, and the timing reduction is a max."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 150.0][rank]
    slowest = bench.max_over_ranks(local_ms, dist)
    value = bench.job_throughput(world, 1920 * 1080, 10, slowest)
    out[rank] = (slowest, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_weak_scaling_aggregation():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 150.0
    want = 2 * 1920 * 1080 * 10 / 0.150 / 1e6
    assert out[0][1] == pytest.approx(want) and out[1][1] == pytest.approx(want)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.job_throughput(1, 100, 4, 2.0) == pytest.approx(100 * 4 / 0.002 / 1e6)
