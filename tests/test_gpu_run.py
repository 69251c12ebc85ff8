"""Multi-step launches of the pipelined update (kernels 5 and 6): one
cooperative launch runs many time steps, its CTAs ordering the steps among
themselves (a tile of step s waits until step s - 1 has finished the
neighbouring row bands).  The arithmetic is that of kernels 3 and 4 tile for
tile, so the states must be equal bit for bit to the one-launch-per-step
kernels' at every step count (odd counts end in the other buffer), on grids
from one tile (every tile waits on the step before) to many tiles per SM;
the oracle comparisons of these kernels are in test_gpu_parity.py."""
import numpy as np
import pytest

import clbm_inputs as I
from oracle import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _clbm():
    from paper_2301_01868_gb300 import clbm
    return clbm


def polar(n1, n2, Q=21, prec=1, CR=0.35, uw=0.02):
    c = _clbm()
    R1, R2 = 1.0, 2.0
    g = c.Grid(Q, n1, n2, I.polar_edges(R1, R2, n1, CR), kind=c.POLAR, precision=prec, bc_lo=c.MOVING,
               bc_hi=c.NOSLIP)
    g.set_case(0.8, 1.0, c.wall_speed_polar(uw, R1, n2, (R2 - R1) / n1), 0.0)
    return g


def planar(n1, n2, Q=21, prec=1):
    c = _clbm()
    g = c.Grid(Q, n1, n2, I.uniform_edges(n1), kind=c.PLANAR, precision=prec, bc_lo=c.MOVING,
               bc_hi=c.MOVING)
    g.set_case(0.9, 1.0, 0.02, -0.01, (1e-6, 2e-6))
    return g


def random_start(make, seed=3, amp=5e-3):
    g = make()
    st = g.state()
    g.close()
    return st * (1.0 + I.smooth_field(st.shape, seed=seed, amplitude=amp))


def run(make, kernel, start, steps):
    g = make()
    g.set_kernel(kernel)
    g.set_state(start)
    for n in steps:
        g.step(n)
    out = g.state(), g.moments(), g.t
    g.close()
    return out


PAIRS = [(1, 3, 5), (2, 4, 6), (3, 4, 6)]     # (precision, single-step kernel, multi-step kernel)


@pytest.mark.parametrize("prec,k1,kr", PAIRS)
@pytest.mark.parametrize("shape", [(4, 8), (19, 131), (27, 139), (64, 640)])
def test_multi_step_runs_equal_single_step_launches_bit_for_bit(prec, k1, kr, shape):
    """From one tile (4 x 8) to 70 tiles; step counts 1, 2, odd and long
    (the single-step kernel replays its 10-launch graph there)."""
    n1, n2 = shape
    make = lambda: planar(n1, n2, prec=prec)
    st = random_start(make)
    steps = (1, 2, 7, 25)
    a = run(make, k1, st, steps)
    b = run(make, kr, st, steps)
    assert a[2] == b[2] == sum(steps)
    assert np.array_equal(a[0], b[0])
    for k in ("rho", "Ut1", "Ut2"):
        assert np.array_equal(a[1][k], b[1][k]), k


@pytest.mark.parametrize("Q", [9, 21])
@pytest.mark.parametrize("prec,k1,kr", [(1, 3, 5), (2, 4, 6)])
def test_multi_step_run_on_many_tiles_per_sm(Q, prec, k1, kr):
    """A channel of square cells with 10 to 27 tiles per SM, j-dependent
    random start, both walls moving, body force: 40 steps in one launch
    against 40 single-step launches, bit for bit; the automatic choice runs
    16-bit storage there as multi-step launches, FP32 as a launch per step."""
    make = lambda: planar(512, 4096, Q=Q, prec=prec)
    st = random_start(make, amp=1e-3)
    a = run(make, k1, st, (40,))
    b = run(make, kr, st, (40,))
    assert np.isfinite(a[0]).all()
    assert np.array_equal(a[0], b[0])
    g = make()
    g.step(1)                             # (the first step also fills the ghosts)
    l0 = g.launch_count()
    g.step(40)
    if prec == 1:
        assert g.launch_count() - l0 == 40
    else:
        assert g.launch_count() - l0 == 1     # one launch for the run
    g.close()


def test_small_grids_keep_one_launch_per_step_by_default():
    g = polar(24, 100)
    g.step(1)
    l0 = g.launch_count()
    g.step(40)
    assert g.launch_count() - l0 > 1
    g.close()


def test_run_longer_than_one_launch_and_profiling_counts_steps():
    """2500 steps (1 + 2499: three launches of at most 1000 steps); the
    profiling events record each launch as a whole and count its steps."""
    make = lambda: planar(16, 256)
    st = random_start(make)
    a = run(make, 3, st, (2500,))
    g = make()
    g.set_kernel(5)
    g.set_state(st)
    g.step(1)
    g.set_profiling(1)
    l0 = g.launch_count()
    g.step(2499)
    assert g.launch_count() - l0 == 3
    ms, launches = g.kernel_time()
    assert launches == 2499 and ms > 0.0
    assert np.array_equal(g.state(), a[0])
    g.close()


def test_general_grids_refuse_the_multi_step_kernels():
    c = _clbm()
    n1, n2 = 12, 40
    P = I.mapped_nodes(I.wavy_channel(n1, n2, amp=0.15), n1, n2, "extend")
    g = c.Grid(21, n1, n2, None, kind=c.GENERAL, nodes=P, dx=1.0, precision=1)
    for k in (5, 6):
        with pytest.raises(c.ClbmError):
            g.set_kernel(k)
    g.close()


def test_multi_step_run_matches_oracle_with_residual():
    """The annulus with a moving inner wall through the multi-step kernel:
    velocity against the oracle after 400 steps, and the residual of the
    last 100 against the oracle's."""
    c = _clbm()
    n1, n2 = 24, 160
    R1, R2 = 1.0, 2.0
    e = I.polar_edges(R1, R2, n1, 0.35)
    U0 = c.wall_speed_polar(0.02, R1, n2, (R2 - R1) / n1)
    o = O.Grid(21, n1, n2, O.POLAR, edges=e, bc_lo=O.MOVING, bc_hi=O.NOSLIP)
    o.set_case(0.8, 1.0, U0, 0.0)
    o.init_rest()
    g = polar(n1, n2)
    g.set_kernel(5)
    o.step(300)
    g.step(300)
    g.residual()
    d0 = o.diagnostics()
    o.step(100)
    g.step(100)
    res, cons = g.residual()
    d1 = o.diagnostics((d0["Ut1"], d0["Ut2"]), 100)
    mo, mg = o.moments(), g.moments()
    num = np.sqrt(((mg["Ut1"] - mo["Ut1"]) ** 2).sum() + ((mg["Ut2"] - mo["Ut2"]) ** 2).sum())
    den = np.sqrt((mo["Ut1"] ** 2).sum() + (mo["Ut2"] ** 2).sum())
    assert num / den <= 1e-5
    # the residual is |u(400) - u(300)| / (100 |u(400)|) = 1.6e-3: the
    # difference of two fields is 0.16 of either, which scales the FP32
    # velocity error by about 6 (the single-step kernel gives the same bits)
    assert res == pytest.approx(d1["res"], rel=5e-5)
    assert cons[3] == pytest.approx(d1["ke"], rel=2e-5)
    g.close()
