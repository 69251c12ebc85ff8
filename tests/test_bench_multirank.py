"""The multi-rank pieces of bench.py on CPU ranks (gloo, world size 2):
the slowest rank's time is taken and the value counts every rank's work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank
    m = bench.max_over_ranks(ms, dist, "cpu")
    v = bench.whole_job_mlups(1000, 10, 5, world, m)
    dist.barrier()
    q.put((rank, m, v))
    dist.destroy_process_group()


@pytest.mark.timeout(240)
def test_max_over_ranks_and_whole_job_value():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    try:
        out = [q.get(timeout=120) for _ in range(world)]
    finally:
        for p in ps:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    for p in ps:
        assert p.exitcode == 0
    for rank, m, v in out:
        assert m == 150.0
        assert abs(v - 1000 * 10 * 5 * world / 0.150 / 1e6) < 1e-9


def test_single_process_needs_no_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
