"""Multi-rank host logic of bench.py on CPU: two gloo ranks, each with its
own batch (weak scaling), agree on the slowest rank's time and on the
whole-job throughput; no data-path collective is involved."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method="env://")
    w, r, lr = bench.world_info()
    my_ms = 100.0 + 50.0 * r                       # rank 1 is the slower one
    slowest = bench.max_over_ranks(my_ms)
    value = bench.job_throughput(12_800_000, 10, slowest, w)
    out.put((r, w, lr, slowest, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_slowest_time_and_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, world, local, slowest, value) in enumerate(res):
        assert (rank, world, local) == (r, 2, r)
        assert slowest == 150.0
        assert value == pytest.approx(2 * 12_800_000 * 10 / 0.150)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(100, 2, 1000.0, 1) == pytest.approx(200.0)
