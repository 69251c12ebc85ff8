"""Slabs along q^2 on one GPU: the lattice split into 2 and 3 runs of
columns, each a grid of its own, with the halo strips exchanged after every
step (the slabs' kernels never wait on one another: the host orders every
launch and copy), gives the unsplit lattice's state bit for bit in FP64 and
within FP32 rounding, and the same residual and conservation values."""
import math

import numpy as np
import pytest

import clbm_inputs as I
from oracle import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _mods():
    from paper_2301_01868_gb300 import clbm, slab
    return clbm, slab


def annulus(Q, n1):
    n2 = I.n_theta(n1, 1.0, 2.0)
    return n2, I.polar_edges(1.0, 2.0, n1)


def run_pair(Q, prec, parts, kind, n1, n2, edges, case, steps, seed=3, step2=1.0, bc=(1, 0)):
    clbm, slab = _mods()
    st = torch.cuda.Stream()
    full = clbm.Grid(Q, n1, n2, edges, kind=kind, step2=step2, precision=prec, bc_lo=bc[0], bc_hi=bc[1],
                     stream=st)
    full.set_case(*case)
    S = slab.SlabSet(parts, Q, n1, n2, edges, kind=kind, step2=step2, precision=prec, bc_lo=bc[0],
                     bc_hi=bc[1])
    S.set_case(*case)
    # a j-dependent start, from the oracle's rest state (host input to both)
    o = O.Grid(Q, n1, n2, O.POLAR if kind == clbm.POLAR else O.PLANAR, edges=edges, step2=step2,
               bc_lo=bc[0], bc_hi=bc[1])
    o.set_case(case[0], case[1], case[2], case[3], case[4] if len(case) > 4 else (0.0, 0.0))
    o.init_rest()
    start = o.state() * (1.0 + I.smooth_field((Q, n1, n2), seed=seed, amplitude=1e-3))
    full.set_state(start)
    S.set_state(start)
    full.residual()
    S.residual()
    full.step(steps)
    S.step(steps)
    return full, S


@pytest.mark.parametrize("Q", [21, 9])
@pytest.mark.parametrize("parts", [1, 2, 3])
def test_fp64_slabs_equal_the_whole_lattice_bit_for_bit(Q, parts):
    clbm, _ = _mods()
    n1 = 16
    n2, e = annulus(Q, n1)
    U0 = clbm.wall_speed_polar(0.02, 1.0, n2, 1.0 / n1)
    full, S = run_pair(Q, 0, parts, clbm.POLAR, n1, n2, e, (0.8, 1.0, U0, 0.0), 120)
    assert np.array_equal(S.state(), full.state())
    r_f, c_f = full.residual()
    r_s, c_s = S.residual()
    assert r_s == pytest.approx(r_f, rel=1e-12)
    np.testing.assert_allclose(c_s, c_f, rtol=1e-12, atol=1e-15 * abs(c_f[0]))
    full.close()
    S.close()


@pytest.mark.parametrize("prec", [1, 2])
def test_fp32_and_fp16_slabs_of_a_stretched_channel(prec):
    """Planar channel with a body force and a moving wall, split in 3; the
    pipelined TMA update runs on every slab."""
    clbm, _ = _mods()
    n1, n2 = 24, 200
    e = I.geometric_stretch_edges(n1, 1.04, float(n1))
    case = (0.7, 1.0, 0.0, 0.004, (0.0, 2e-6))
    full, S = run_pair(21, prec, 3, clbm.PLANAR, n1, n2, e, case, 150, bc=(0, 1))
    a, b = S.state(), full.state()
    rest_dev = np.abs(b - b.mean(axis=(1, 2), keepdims=True)).max()
    assert np.abs(a - b).max() <= (1e-6 if prec == 1 else 1e-3) * rest_dev
    m_f = full.moments(names=("Ut1", "Ut2"))
    m_s = S.moments(names=("Ut1", "Ut2"))
    num = ((m_s["Ut1"] - m_f["Ut1"]) ** 2 + (m_s["Ut2"] - m_f["Ut2"]) ** 2).sum()
    den = (m_f["Ut1"] ** 2 + m_f["Ut2"] ** 2).sum()
    assert math.sqrt(num / den) <= (1e-5 if prec == 1 else 2e-3)
    full.close()
    S.close()


def test_halo_strip_counts():
    clbm, _ = _mods()
    for Q, per_row in ((21, 12), (9, 3)):
        g = clbm.Grid(Q, 8, 16, I.uniform_edges(8), precision=1)
        H = 3 if Q == 21 else 1
        assert g.halo_values() == per_row * (8 + 2 * H)
        g.close()


def test_narrow_slab_is_rejected():
    clbm, _ = _mods()
    g = clbm.Grid(21, 8, 2, I.uniform_edges(8), precision=1)
    g.set_case(0.8)
    buf = torch.empty(g.halo_values(), dtype=torch.float32, device="cuda")
    with pytest.raises(clbm.ClbmError):
        g.halo_pack(0, buf)
    g.close()


def _slab_rank(rank, world, port, q):
    """One rank of a gloo process group with its slab on the one GPU (the
    kernels of the ranks never wait on each other: every exchange goes
    through the host between launches)."""
    import os
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2301_01868_gb300 import clbm, slab
        from oracle import oracle as Orc
        n1 = 16
        n2, e = annulus(21, n1)
        U0 = clbm.wall_speed_polar(0.02, 1.0, n2, 1.0 / n1)
        s = slab.Slab(21, n1, n2, e, kind=clbm.POLAR, precision=0, bc_lo=clbm.MOVING, bc_hi=clbm.NOSLIP,
                      stream=torch.cuda.Stream())
        s.set_case(0.8, 1.0, U0, 0.0)
        o = Orc.Grid(21, n1, n2, Orc.POLAR, edges=e, bc_lo=Orc.MOVING, bc_hi=Orc.NOSLIP)
        o.set_case(0.8, 1.0, U0, 0.0)
        o.init_rest()
        start = o.state() * (1.0 + I.smooth_field((21, n1, n2), seed=3, amplitude=1e-3))
        s.set_state(np.ascontiguousarray(start[:, :, s.j0:s.j1]))
        s.residual()
        s.step(80)
        res, cons = s.residual()
        q.put((rank, s.j0, s.j1, s.state(), res, cons))
        s.close()
    finally:
        dist.destroy_process_group()


def test_distributed_slabs_over_gloo_ranks_equal_the_whole_lattice():
    """Two processes, a gloo group, one slab each (slab.Slab, the class a
    multi-GPU run uses, exchanging its strips through host memory): the
    gathered state equals the unsplit lattice's bit for bit in FP64, and
    the reduced residual and conservation values equal its own."""
    import socket
    import torch.multiprocessing as mp
    clbm, _ = _mods()
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_slab_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted([q.get(timeout=300) for _ in range(2)], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    n1 = 16
    n2, e = annulus(21, n1)
    full, _ = run_pair(21, 0, 1, clbm.POLAR, n1, n2, e,
                       (0.8, 1.0, clbm.wall_speed_polar(0.02, 1.0, n2, 1.0 / n1), 0.0), 80)
    whole = full.state()
    assert out[0][1] == 0 and out[-1][2] == n2
    joined = np.concatenate([st for _, _, _, st, _, _ in out], axis=2)
    assert np.array_equal(joined, whole)
    r_f, c_f = full.residual()
    for _, _, _, _, res, cons in out:
        assert res == pytest.approx(r_f, rel=1e-12)
        np.testing.assert_allclose(cons, c_f, rtol=1e-12, atol=1e-15 * abs(c_f[0]))
    full.close()


def test_bench_slab_mode_runs_on_one_rank():
    """bench.py --slab on one rank (the slab is its own neighbour): one JSON
    line with strong scaling and the slab's columns."""
    import json
    import os
    import subprocess
    import sys
    from conftest import ROOT
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--slab", "--workload",
                          "circular_couette_d2q21_fp32_128x512", "--steps", "2", "--warmup", "1",
                          "--chunk", "5"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads([ln for ln in out.stdout.splitlines() if ln.strip()][-1])
    assert d["scaling"] == "strong" and d["n_gpus"] == 1 and d["value"] > 0
    assert d["config"]["slab_columns"] == [0, 512]
    assert d["gpu_launches"] > 0
