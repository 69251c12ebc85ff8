"""Batched stepping: lattices of uneven shapes advanced together give the
same result as each advanced alone, for every tile variant."""
import math

import numpy as np
import pytest

import clbm_inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _clbm():
    from paper_2301_01868_gb300 import clbm
    return clbm


def make_grid(kind, Q, prec, n1, n2, stream, seed, iters=0):
    c = _clbm()
    rng = np.random.default_rng(seed)
    tau = float(rng.uniform(0.6, 1.0))
    if kind == "polar":
        e = I.polar_edges(1.0, 2.0, n1, 0.3)
        g = c.Grid(Q, n1, n2, e, kind=c.POLAR, precision=prec, bc_lo=c.MOVING, bc_hi=c.NOSLIP,
                   stream=stream)
        g.set_case(tau, 1.0, c.wall_speed_polar(0.02, 1.0, n2, 1.0 / n1), 0.0, force_iterations=iters)
    else:
        e = I.geometric_stretch_edges(n1, 1.03, float(n1))
        g = c.Grid(Q, n1, n2, e, kind=c.PLANAR, step2=1.0, precision=prec, bc_lo=c.NOSLIP,
                   bc_hi=c.MOVING, stream=stream)
        nu = (1 / 3 if Q == 9 else 2 / 3) * (tau - 0.5)
        g.set_case(tau, 1.0, 0.0, 0.01, (0.0, 8 * nu * 0.02 / n1 ** 2), force_iterations=iters)
    return g


SHAPES = [("polar", 12, 50), ("planar", 9, 33), ("polar", 20, 130), ("planar", 17, 257),
          ("planar", 4, 5), ("polar", 16, 64)]


def build(Q, prec, stream, iters=(0,) * len(SHAPES)):
    return [make_grid(k, Q, prec, n1, n2, stream, s, it)
            for s, ((k, n1, n2), it) in enumerate(zip(SHAPES, iters))]


@pytest.mark.parametrize("Q,prec", [(21, 0), (9, 0), (21, 1), (9, 1)])
@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
def test_batch_matches_lattices_alone(Q, prec, variant):
    if variant == 4 and prec == 0:
        pytest.skip("the pipelined TMA variant stores 16/32-bit populations")
    c = _clbm()
    stream = torch.cuda.Stream()
    alone = build(Q, prec, stream)
    mixed = build(Q, prec, stream)
    for g in alone:
        g.set_kernel(1)
        g.step(61)
    b = c.Batch(mixed)
    b.set_variant(variant)
    b.step(61)
    b.residual()
    for ga, gm in zip(alone, mixed):
        assert gm.t == 61
        sa, sm = ga.state(), gm.state()
        scale = np.abs(sa).max()
        tol = 1e-13 if prec == 0 else 1e-6
        assert np.abs(sa - sm).max() <= tol * scale
    b.close()


@pytest.mark.parametrize("Q,prec", [(9, 0), (21, 1)])
def test_batch_with_implicit_force_lattices(Q, prec):
    """Lattices that iterate the force (Sec. 2) share a batch with lagged ones."""
    c = _clbm()
    stream = torch.cuda.Stream()
    iters = (1, 0, 2, 0, 1, 1)
    alone = build(Q, prec, stream, iters)
    mixed = build(Q, prec, stream, iters)
    for g in alone:
        g.set_kernel(1)
        g.step(41)
        g.residual()
        g.step(10)
    b = c.Batch(mixed)
    b.set_variant(1)
    b.step(41)
    b.residual()
    b.step(10)
    res, cons = b.residual()
    tol = 1e-13 if prec == 0 else 1e-6
    for k, (ga, gm) in enumerate(zip(alone, mixed)):
        sa, sm = ga.state(), gm.state()
        assert np.abs(sa - sm).max() <= tol * np.abs(sa).max()
        r, cs = ga.residual()
        assert abs(res[k] - r) <= (1e-12 if prec == 0 else 1e-4) * abs(r)
    b.close()


def test_batch_residual_matches_single_residuals():
    c = _clbm()
    stream = torch.cuda.Stream()
    grids = build(21, 0, stream)
    ref = build(21, 0, stream)
    b = c.Batch(grids)
    b.residual()
    for g in ref:
        g.residual()
    b.step(30)
    for g in ref:
        g.step(30)
    res, cons = b.residual()
    for k, g in enumerate(ref):
        r, cs = g.residual()
        assert abs(res[k] - r) <= 1e-12 * abs(r)
        np.testing.assert_allclose(cons[k], cs, rtol=1e-12, atol=1e-14)
    b.close()


def test_grid_stepped_alone_between_batch_steps():
    c = _clbm()
    stream = torch.cuda.Stream()
    grids = build(9, 0, stream)
    ref = build(9, 0, stream)
    b = c.Batch(grids)
    b.step(5)
    grids[2].step(3)          # one lattice runs on its own
    b.step(4)
    for k, g in enumerate(ref):
        g.set_kernel(1)
        g.step(12 if k == 2 else 9)
    for ga, gm in zip(ref, grids):
        assert ga.t == gm.t
        np.testing.assert_allclose(gm.state(), ga.state(), rtol=0, atol=1e-13)
    b.close()


def test_autotuner_picks_a_variant():
    c = _clbm()
    stream = torch.cuda.Stream()
    grids = build(21, 1, stream)
    b = c.Batch(grids)
    best, ms = b.tune(steps=3)
    usable = ms > 0
    assert usable[:4].all() and usable[4]      # FP32: the TMA variant is usable too
    assert 0 <= best < 5 and ms[best] == ms[usable].min()
    t0 = grids[0].t
    b.step(10)
    assert grids[0].t == t0 + 10
    b.close()


@pytest.mark.parametrize("Q,prec", [(9, 1), (21, 2)])
@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
def test_batch_matches_lattices_alone_more_storage(Q, prec, variant):
    """D2Q9 with FP32 storage and D2Q21 with FP16 storage: the batch gives the
    lattices' own results (the single-lattice path runs the per-cell kernel)."""
    c = _clbm()
    stream = torch.cuda.Stream()
    alone = build(Q, prec, stream)
    mixed = build(Q, prec, stream)
    for g in alone:
        g.set_kernel(1)
        g.step(300)
    b = c.Batch(mixed)
    if variant == 4 and prec == 2:
        # FP16 rows of 5 cells are shorter than a 16-byte chunk: no TMA maps
        with pytest.raises(c.ClbmError):
            b.set_variant(variant)
        b.close()
        return
    b.set_variant(variant)
    b.step(300)
    for ga, gm in zip(alone, mixed):
        sa, sm = ga.state(), gm.state()
        dev = np.abs(sa - sa.mean(axis=(1, 2), keepdims=True)).max()
        assert np.abs(sa - sm).max() <= (1e-6 if prec == 1 else 2e-3) * max(dev, 1e-12)
    b.close()


def test_batch_residual_isolates_an_unstable_lattice():
    """One lattice with a non-finite density: its residual is NaN, every other
    lattice's residual is still returned and matches its own."""
    c = _clbm()
    stream = torch.cuda.Stream()
    grids = build(21, 0, stream)
    ref = build(21, 0, stream)
    st = grids[2].state()
    st[:, 3, 5] = np.nan
    grids[2].set_state(st)
    b = c.Batch(grids)
    b.residual()
    b.step(20)
    for g in ref:
        g.residual()
        g.step(20)
    res, _ = b.residual()
    assert np.isnan(res[2])
    for k, g in enumerate(ref):
        if k != 2:
            r, _ = g.residual()
            assert abs(res[k] - r) <= 1e-12 * abs(r)
    b.close()
