"""Multi-rank bookkeeping of the benchmark (replicas only: each rank runs an independent
solve; the ranks share a barrier and the maximum of their times) on CPU ranks over gloo."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rep = bench.Replicas(world, torch.device("cpu"))
    rep.barrier()
    t = rep.max(times[rank])
    v = rep.value(1000.0, t)
    rep.barrier()
    out.put((rank, t, v))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_max_over_ranks_and_whole_job_value(world):
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    times = [0.5 + 0.25 * r for r in range(world)]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, times, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = max(times)
    for rank, t, v in res:
        assert t == slowest                               # every rank sees the slowest time
        assert v == pytest.approx(world * 1000.0 / slowest)  # N x one rank's units / that time


def test_single_rank_needs_no_process_group():
    import bench
    rep = bench.Replicas(1, torch.device("cpu"))
    rep.barrier()
    assert rep.max(1.25) == 1.25
    assert rep.value(10.0, 2.0) == 5.0
