"""Checkpoint / resume and run-to-run determinism on the GPU.

A grid saved after some steps and restored into a fresh grid of the same
description continues bit for bit: the same state, residual and conservation
totals as the grid that never stopped.  Two grids given the same inputs give
identical bits (the update has no atomics and the reductions a fixed order).
"""
import math

import numpy as np
import pytest

import clbm_inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _clbm():
    from paper_2301_01868_gb300 import clbm
    return clbm


def annulus(c, Q, prec, n1=24, n2=150):
    e = I.polar_edges(1.0, 2.0, n1, 0.35)
    g = c.Grid(Q, n1, n2, e, kind=c.POLAR, precision=prec, bc_lo=c.MOVING, bc_hi=c.NOSLIP)
    return g, e


def start(c, g, Q, n1, n2, seed=5):
    g.set_case(0.8, 1.0, c.wall_speed_polar(0.01, 1.0, n2, 1.0 / n1), 0.0, (0.0, 1e-6))
    st = g.state() * (1.0 + I.smooth_field((Q, n1, n2), seed=seed, amplitude=2e-3))
    g.set_state(st)


@pytest.mark.parametrize("Q,prec", [(21, 0), (21, 1), (21, 2), (21, 3), (9, 1)])
def test_restore_continues_bit_for_bit(Q, prec):
    c = _clbm()
    n1, n2 = 24, 150
    a, e = annulus(c, Q, prec, n1, n2)
    start(c, a, Q, n1, n2)
    a.step(120)
    a.residual()
    a.step(7)
    blob = a.checkpoint()
    a.step(150)
    ra = a.residual()
    sa = a.state()
    b, _ = annulus(c, Q, prec, n1, n2)        # fresh grid, no case given
    b.restore(blob)
    assert b.t == 127
    b.step(150)
    rb = b.residual()
    assert b.t == a.t
    assert np.array_equal(b.state(), sa)
    assert rb[0] == ra[0] and np.array_equal(rb[1], ra[1])
    # rewinding the saved grid itself gives the same continuation
    a.restore(blob)
    a.step(150)
    assert np.array_equal(a.state(), sa)


def test_restore_keeps_the_no_flow_adjustment_and_the_kernel_choice():
    c = _clbm()
    n1, n2 = 24, 150
    a, _ = annulus(c, 21, 1, n1, n2)
    a.set_case(0.8, 1.0, 0.0, 0.0)
    a.no_flow_adjust(500)
    a.set_kernel(1)
    a.step(40)
    blob = a.checkpoint()
    a.step(60)
    sa = a.state()
    b, _ = annulus(c, 21, 1, n1, n2)
    b.set_kernel(1)
    b.restore(blob)
    b.step(60)
    assert np.array_equal(b.state(), sa)


def test_general_grid_restore():
    c = _clbm()
    n1, n2 = 14, 22
    P = I.mapped_nodes(I.wavy_channel(n1, n2, amp=0.15), n1, n2, "extend")

    def make():
        return c.Grid(21, n1, n2, None, kind=c.GENERAL, nodes=P, dx=1.0, precision=0)

    a = make()
    a.set_case(0.8, 1.0, 0.0, 0.0, (0.0, 1e-5))
    a.step(50)
    blob = a.checkpoint()
    a.step(50)
    b = make()
    b.restore(blob)
    b.step(50)
    assert np.array_equal(b.state(), a.state())


def test_restore_refuses_another_grid():
    c = _clbm()
    a, _ = annulus(c, 21, 1, 24, 150)
    a.set_case(0.8)
    blob = a.checkpoint()
    for other in (annulus(c, 21, 1, 24, 152)[0], annulus(c, 21, 2, 24, 150)[0],
                  annulus(c, 9, 1, 24, 150)[0]):
        with pytest.raises(c.ClbmError):
            other.restore(blob)
    bad = bytearray(blob)
    bad[:8] = b"NOTACKPT"
    with pytest.raises(c.ClbmError):
        a.restore(bytes(bad))


@pytest.mark.parametrize("kernel", [1, 3])
def test_two_runs_are_bitwise_identical(kernel):
    c = _clbm()
    n1, n2 = 64, 402
    out = []
    for _ in range(2):
        g, _ = annulus(c, 21, 1, n1, n2)
        g.set_kernel(kernel)
        start(c, g, 21, n1, n2, seed=9)
        g.step(200)
        r0 = g.residual()
        g.step(100)
        out.append((g.state(), g.residual(), r0))
        g.close()
    (s0, r0, q0), (s1, r1, q1) = out
    assert np.array_equal(s0, s1)
    assert r0[0] == r1[0] and np.array_equal(r0[1], r1[1])
    assert math.isfinite(r0[0])
