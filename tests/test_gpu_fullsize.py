"""Parity at the full benchmark sizes, in the launch configuration bench.py
times (automatic kernel choice: the pipelined TMA update for FP32): one time
step from a seeded state on the whole grid, then the updated populations of
sampled cells -- corners, wall rows, tile and block edges, the periodic seam
and seeded random cells -- against the oracle's collision of that one cell
from the same state (the oracle computes cells one by one, so the full grid
costs it nothing beyond memory).  2-D: the annulus 1024 x 4096 of every 2-D
bench workload (D2Q21 FP32, FP16 and BF16 storage, D2Q9 FP32);
3-D: the D3Q39 FP32 extruded annulus 128 x 804 x 32.  Plus properties that
hold at any size after many steps from rest: finite residual, conserved
mass.  The oracle starts from its own rest state, perturbed by the seeded
field and rounded on the host as the grid stores it."""
import math

import numpy as np
import pytest

import clbm_inputs as I
from conftest import storage_rounded
from oracle import oracle as O
from oracle import oracle3d as O3

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _clbm():
    from paper_2301_01868_gb300 import clbm
    return clbm


def samples_2d(n1, n2, seed=11, nrand=48):
    rng = np.random.default_rng(seed)
    rows = [1, 2, 3, 8, 9, 16, 17, n1 // 2, n1 - 2, n1 - 1, n1]
    cols = [1, 2, 3, 4, 5, 63, 64, 65, 128, n2 // 2, n2 - 4, n2 - 1, n2]
    cells = {(i, j) for i in rows for j in cols[::3]} | {(i, j) for i in rows[::2] for j in cols}
    cells |= {(int(a), int(b)) for a, b in zip(rng.integers(1, n1 + 1, nrand), rng.integers(1, n2 + 1, nrand))}
    return sorted(cells)


# the bench's 2-D workloads: (Q, storage, tolerance of the sampled one-step
# change): FP32 and 16-bit storage round the stored deviations
WORKLOADS_2D = [(21, "fp32", 1e-4), (21, "fp16", 2e-3), (21, "bf16", 2e-2), (9, "fp32", 1e-4)]


@pytest.mark.parametrize("Q,prec,tol", WORKLOADS_2D)
def test_fullsize_2d_bench_grid_one_step_matches_oracle_on_sampled_cells(Q, prec, tol):
    c = _clbm()
    n1, n2, R1, R2, CR, tau, uw = 1024, 4096, 1.0, 2.0, 0.35, 0.8, 0.01
    e = I.polar_edges(R1, R2, n1, CR)
    dx = (R2 - R1) / n1
    U0 = uw * dx / (R1 * math.sin(2.0 * math.pi / n2))
    o = O.Grid(Q, n1, n2, O.POLAR, edges=e, bc_lo=O.MOVING, bc_hi=O.NOSLIP)
    o.set_case(tau, 1.0, U0, 0.0)
    o.init_rest()
    rest = o.state()
    st = rest * (1.0 + I.smooth_field((Q, n1, n2), seed=5, amplitude=2e-3))
    st_stored = storage_rounded(rest, st, prec)   # the start as the grid stores it
    o.set_state(st_stored)
    g = c.Grid(Q, n1, n2, e, kind=c.POLAR, precision=prec, bc_lo=c.MOVING, bc_hi=c.NOSLIP)
    g.set_case(tau, 1.0, U0, 0.0)
    g.set_state(st)
    g.step(1)
    out = g.state()
    num = den = 0.0
    for (i, j) in samples_2d(n1, n2):
        ref = o.collide_one(i, j)["Npost"]
        got = out[:, i - 1, j - 1]
        num += float(((got - ref) ** 2).sum())
        den += float(((ref - st_stored[:, i - 1, j - 1]) ** 2).sum())
    assert math.sqrt(num / den) <= tol
    # properties after many steps on the full grid, from rest with the wall
    # moving (a j-dependent start grows on these anisotropic cells: D2Q21's
    # j-dependent modes, a property of the method the oracle shares)
    g.set_case(tau, 1.0, U0, 0.0)
    _, c0 = g.residual()
    g.step(200)
    res, c1 = g.residual()
    assert math.isfinite(res)
    assert abs(c1[0] - c0[0]) <= (1e-6 if prec == "fp32" else 1e-4) * abs(c0[0])
    g.close()


def test_fullsize_3d_bench_grid_one_step_matches_oracle_on_sampled_cells():
    c = _clbm()
    n1, n2, n3, R1, R2, CR, tau, uw = 128, 804, 32, 1.0, 2.0, 0.35, 0.8, 0.01
    e = I.polar_edges(R1, R2, n1, CR)
    dx = (R2 - R1) / n1
    U0 = uw * dx / (R1 * math.sin(2.0 * math.pi / n2))
    o = O3.Grid(n1, n2, n3, O3.ANNULUS, edges=e, step3=dx, bc_lo=O3.MOVING, bc_hi=O3.NOSLIP)
    o.set_case(tau, 1.0, U0, 0.0)
    o.init_rest()
    rest = o.state()
    st = rest * (1.0 + I.smooth_field((39 * n1, n2, n3), seed=7, amplitude=2e-3).reshape(rest.shape))
    st_stored = storage_rounded(rest, st, "fp32")
    o.set_state(st_stored)
    g = c.Grid3(n1, n2, n3, e, kind=c.ANNULUS3, step3=dx, precision="fp32", bc_lo=c.MOVING,
                bc_hi=c.NOSLIP)
    g.set_case(tau, 1.0, U0, 0.0)
    g.set_state(st)
    g.step(1)
    out = g.state()
    rng = np.random.default_rng(13)
    cells = {(i, j, k) for i in (1, 2, 3, 64, 126, 127, 128) for j in (1, 2, 402, 803, 804)
             for k in (1, 2, 31, 32)}
    cells |= {(int(a), int(b), int(d)) for a, b, d in
              zip(rng.integers(1, n1 + 1, 40), rng.integers(1, n2 + 1, 40), rng.integers(1, n3 + 1, 40))}
    num = den = 0.0
    for (i, j, k) in sorted(cells):
        ref = o.collide_one(i, j, k)["Npost"]
        got = out[:, i - 1, j - 1, k - 1]
        num += float(((got - ref) ** 2).sum())
        den += float(((ref - st_stored[:, i - 1, j - 1, k - 1]) ** 2).sum())
    assert math.sqrt(num / den) <= 1e-4
    g.set_case(tau, 1.0, U0, 0.0)
    m0 = g.totals()[0]
    g.step(100)
    assert abs(g.totals()[0] - m0) <= 1e-6 * abs(m0)
    g.close()
