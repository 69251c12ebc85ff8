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


def test_serial_fifo_latencies_from_service_times():
    """The serial baseline at a given arrival rate: one FIFO server fed the
    measured service times (start = max(arrival, previous finish))."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)

    class R:
        def __init__(self, rid, arrival):
            self.rid, self.arrival = rid, arrival

    reqs = [R(0, 0.0), R(1, 0.5), R(2, 3.0), R(3, 3.1)]
    service = {0: 1.0, 1: 1.0, 2: 0.2, 3: 0.5}
    out = {rid: (lat, t) for rid, lat, t in bench._fifo_latencies(reqs, service)}
    assert out[0] == (1.0, 1.0)
    assert out[1] == (1.5, 2.0)          # waits for request 0
    assert abs(out[2][0] - 0.2) < 1e-12 and abs(out[2][1] - 3.2) < 1e-12   # server idle at 3.0
    assert abs(out[3][0] - 0.6) < 1e-12 and abs(out[3][1] - 3.7) < 1e-12
