"""The bench's replica aggregation across ranks (two gloo ranks on the CPU):
the slowest rank's time, every rank's bytes."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r + 1) ms for the product and 10 - r ms for the build
        worst = bench.max_over_ranks([rank + 1.0, 10.0 - rank])
        gbs = bench.whole_job_gbs(2e9, worst[0], world)
        out.put((rank, worst, gbs))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, worst, gbs in res:
        assert worst == [2.0, 10.0]  # element-wise maximum over both ranks
        # 2 ranks x 2 GB in the slowest rank's 2 ms
        assert gbs == pytest.approx(2 * 2e9 / 2e-3 / 1e9)


def test_max_over_ranks_without_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([1.5, 2.5]) == [1.5, 2.5]
    assert bench.whole_job_gbs(1e9, 1.0, 1) == pytest.approx(1000.0)
