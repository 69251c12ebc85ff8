"""Slabs along q^2 on CPU ranks (gloo, world size 2 and 3): the partition of
the columns, the neighbour exchange of halo strips (send_lo reaches the lower
neighbour's recv_hi, send_hi the upper neighbour's recv_lo) and the
reduction of the residual parts over the ranks; and, on a streaming model of
the update (each population moved by its c_alpha, Eq. 12, on the stored
layout with ghost columns), that the strips the library packs -- the
populations with c2 > 0 at depths 1..c2 toward the upper neighbour and c2 < 0
toward the lower one, 12 per side for D2Q21 -- make a split lattice stream
exactly as the whole one."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from conftest import ROOT  # noqa: F401


def _slab():
    from paper_2301_01868_gb300 import slab
    return slab


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_covers_the_ring():
    S = _slab()
    for n2, parts in ((100, 1), (100, 3), (7, 7), (4096, 8), (101, 4)):
        r = S.partition(n2, parts)
        assert r[0][0] == 0 and r[-1][1] == n2
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        w = [b - a for a, b in r]
        assert max(w) - min(w) <= 1
    with pytest.raises(ValueError):
        S.partition(3, 4)
    assert S.neighbours(0, 3) == (2, 1) and S.neighbours(2, 3) == (1, 0)


def test_combine_parts_matches_the_residual_definition():
    S = _slab()
    parts = [4.0, 16.0, 10.0, 0.1, -0.2, 3.0, 5.0, 0.7, 0.0]
    res, cons = S.combine_parts(parts, 10)
    assert res == pytest.approx(2.0 / (10 * 4.0))
    assert list(cons) == [10.0, 0.1, -0.2, 3.0, 5.0, 0.7]
    assert S.combine_parts(parts, 0)[0] == float("inf")
    assert S.combine_parts([0.0, 0.0] + parts[2:], 5)[0] == 0.0


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        S = _slab()
        send_lo = torch.full((5,), 10.0 * rank + 1.0)
        send_hi = torch.full((5,), 10.0 * rank + 2.0)
        recv_lo = torch.zeros(5)
        recv_hi = torch.zeros(5)
        S.exchange(send_lo, send_hi, recv_lo, recv_hi, rank, world)
        lo, hi = S.neighbours(rank, world)
        ok_x = bool((recv_lo == 10.0 * lo + 2.0).all() and (recv_hi == 10.0 * hi + 1.0).all())
        parts = np.array([1.0 + rank, 2.0, 3.0, 0.5 * rank, -rank, 1.0, 2.0, 0.1 * (rank + 1), 0.0])
        tot = S.reduce_parts(parts, rank, world)
        q.put((rank, ok_x, tot.tolist()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_exchange_and_reduction_over_gloo_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ok_x, tot in out:
        assert ok_x, rank
        assert tot[0] == pytest.approx(sum(1.0 + r for r in range(world)))
        assert tot[7] == pytest.approx(0.1 * world)          # max |u| takes the maximum
        assert tot[4] == pytest.approx(-sum(range(world)))


# --------------------------------------------------------- streaming model
GC = 8


def lattice(Q):
    from oracle import oracle as O
    c, _, _, _, _ = O.lattice(Q)
    return c


def stream_step(state, c, n2):
    """Pull streaming on the stored layout [Q][rows][GC + n2 + GC]: the
    interior column j takes population a from column j - c2 (ghost columns
    beyond the ends), rows unchanged (the row shift does not cross a cut)."""
    out = state.copy()
    for a in range(len(c)):
        c2 = int(c[a][1])
        out[a, :, GC:GC + n2] = state[a, :, GC - c2:GC - c2 + n2]
    return out


def wrap(state, n2):
    s = state.copy()
    s[:, :, :GC] = s[:, :, n2:n2 + GC]
    s[:, :, GC + n2:] = s[:, :, GC:2 * GC]
    return s


def strips(c, sign):
    """(population, depth) of one side's strips, in the library's order."""
    out = []
    for a in range(1, len(c)):
        c2 = int(c[a][1])
        if c2 * sign > 0:
            out += [(a, d) for d in range(1, abs(c2) + 1)]
    return out


@pytest.mark.parametrize("Q,count", [(21, 12), (9, 3)])
def test_the_strips_make_a_split_lattice_stream_as_the_whole(Q, count):
    c = lattice(Q)
    assert len(strips(c, 1)) == len(strips(c, -1)) == count
    rows, n2, parts = 5, 24, 3
    rng = np.random.default_rng(1)
    whole = np.zeros((Q, rows, n2 + 2 * GC))
    whole[:, :, GC:GC + n2] = rng.standard_normal((Q, rows, n2))
    cuts = _slab().partition(n2, parts)
    slabs = []
    for j0, j1 in cuts:
        s = np.full((Q, rows, j1 - j0 + 2 * GC), np.nan)   # ghosts unknown until exchanged
        s[:, :, GC:GC + j1 - j0] = whole[:, :, GC + j0:GC + j1]
        slabs.append(s)
    for _ in range(7):
        whole = stream_step(wrap(whole, n2), c, n2)
        # exchange: pack both sides, unpack from the neighbours
        packs = []
        for s, (j0, j1) in zip(slabs, cuts):
            w = j1 - j0
            lo = {(a, d): s[a, :, GC + d - 1].copy() for a, d in strips(c, -1)}
            hi = {(a, d): s[a, :, GC + w - d].copy() for a, d in strips(c, 1)}
            packs.append((lo, hi))
        for r, (s, (j0, j1)) in enumerate(zip(slabs, cuts)):
            w = j1 - j0
            from_lo = packs[(r - 1) % parts][1]
            from_hi = packs[(r + 1) % parts][0]
            for (a, d), v in from_lo.items():
                s[a, :, GC - d] = v
            for (a, d), v in from_hi.items():
                s[a, :, GC + w + d - 1] = v
        slabs = [stream_step(s, c, j1 - j0) for s, (j0, j1) in zip(slabs, cuts)]
        joined = np.concatenate([s[:, :, GC:GC + j1 - j0] for s, (j0, j1) in zip(slabs, cuts)], axis=2)
        assert np.array_equal(joined, whole[:, :, GC:GC + n2])
