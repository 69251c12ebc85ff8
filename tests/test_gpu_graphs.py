"""clbm_step replays a captured CUDA graph for runs of more than 21 steps.
The graph holds the same launches as the plain path, so states must agree
bit for bit with step-by-step runs, across odd run lengths (the buffer
parity), a change of case (the graph is rebuilt) and a change of kernel;
launch counts and profiling keep working.  Grids on the legacy default
stream (which cannot be captured) keep to plain launches."""
import numpy as np
import pytest

import clbm_inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _grid(prec, Q=21, n1=24, stream=True):
    """The annulus 1 <= r <= 2 with near-square cells (n2 = round(2 pi n1)),
    inner wall moving, from a perturbed rest state."""
    from paper_2301_01868_gb300 import clbm
    n2 = I.n_theta(n1, 1.0, 2.0)
    e = I.polar_edges(1.0, 2.0, n1)
    g = clbm.Grid(Q, n1, n2, e, kind=clbm.POLAR, precision=prec, bc_lo=clbm.MOVING, bc_hi=clbm.NOSLIP,
                  stream=torch.cuda.Stream() if stream else None)
    g.set_case(0.8, 1.0, 0.02, 0.0)
    st = g.state()
    g.set_state(st * (1.0 + I.smooth_field(st.shape, seed=3, amplitude=2e-3)))
    return g


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_graph_replay_is_bitwise_the_plain_launches(prec):
    a, b = _grid(prec), _grid(prec)
    for n in (60, 23, 41, 100):
        for _ in range(n):
            a.step(1)        # plain launches (runs shorter than 22 steps)
        b.step(n)            # graph replays
        sa = a.state()
        assert np.isfinite(sa).all()
        assert np.array_equal(sa, b.state()), n
    assert a.t == b.t and a.launch_count() == b.launch_count()
    # a new case rebuilds the graph
    for g in (a, b):
        g.set_case(0.9, 1.0, 0.01, 0.0, g_ext=(0.0, 1e-6))
    for _ in range(40):
        a.step(1)
    b.step(40)
    assert np.array_equal(a.state(), b.state())
    if prec != "fp64":
        for g in (a, b):
            g.set_kernel(1)
        for _ in range(30):
            a.step(1)
        b.step(30)
        assert np.array_equal(a.state(), b.state())
    a.close()
    b.close()


def test_default_stream_grid_keeps_to_plain_launches():
    a, b = _grid("fp32", stream=False), _grid("fp32")
    a.step(50)
    b.step(50)
    assert np.array_equal(a.state(), b.state())
    a.close()
    b.close()


def test_profiling_samples_graph_replays():
    g = _grid("fp32")
    g.step(30)                       # capture outside the profiled run
    g.set_profiling(True, period=10)
    g.step(100)
    ms, n = g.kernel_time()
    assert n == 100 and ms > 0.0     # ten replays of ten launches each
    g.set_profiling(False)
    g.close()


def test_3d_graph_replay_is_bitwise_the_plain_launches():
    from paper_2301_01868_gb300 import clbm
    e = I.polar_edges(1.0, 2.0, 8, 0.35)
    grids = []
    for _ in range(2):
        g = clbm.Grid3(8, 50, 4, e, kind=clbm.ANNULUS3, step3=0.15, precision="fp32", bc_lo=clbm.MOVING,
                       bc_hi=clbm.NOSLIP, stream=torch.cuda.Stream())
        g.set_case(0.8, 1.0, 0.03, 0.0, (0.0, 0.0, 1e-6))
        grids.append(g)
    a, b = grids
    for n in (50, 23, 41):
        for _ in range(n):
            a.step(1)
        b.step(n)
        sa = a.state()
        assert np.isfinite(sa).all()
        assert np.array_equal(sa, b.state()), n
    for g in (a, b):
        g.set_case(0.9, 1.0, 0.01, 0.0)
    for _ in range(30):
        a.step(1)
    b.step(30)
    assert np.array_equal(a.state(), b.state())
    assert a.t == b.t
    a.close()
    b.close()
