"""General (non-separable) grids on the GPU: per-cell geometry and tables
against the FP64 oracle on the same node positions and seeded inputs."""
import numpy as np
import pytest

import clbm_inputs as I
from oracle import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _clbm():
    from paper_2301_01868_gb300 import clbm
    return clbm


def vel_err(m, ref):
    num = ((m["Ut1"] - ref["Ut1"]) ** 2 + (m["Ut2"] - ref["Ut2"]) ** 2).sum()
    den = (ref["Ut1"] ** 2 + ref["Ut2"] ** 2).sum()
    return float(np.sqrt(num / den))


class GCase:
    def __init__(self, Q, nodes, dx=1.0, bc=(0, 0), tau=0.8, U0=(0.0, 0.0), g=(0.0, 0.0), iters=0):
        self.Q, self.nodes, self.dx, self.bc, self.tau, self.U0, self.g, self.iters = \
            Q, nodes, dx, bc, tau, U0, g, iters
        self.n1, self.n2 = nodes.shape[0] - 8, nodes.shape[1] - 8

    def oracle(self):
        o = O.Grid(self.Q, self.n1, self.n2, O.GENERAL, nodes=self.nodes, dx=self.dx,
                   bc_lo=self.bc[0], bc_hi=self.bc[1])
        o.set_case(self.tau, 1.0, self.U0[0], self.U0[1], self.g)
        o.set_force_iterations(self.iters)
        o.init_rest()
        return o

    def gpu(self, prec):
        c = _clbm()
        g = c.Grid(self.Q, self.n1, self.n2, None, kind=c.GENERAL, nodes=self.nodes, dx=self.dx,
                   precision=prec, bc_lo=self.bc[0], bc_hi=self.bc[1])
        g.set_case(self.tau, 1.0, self.U0[0], self.U0[1], self.g, self.iters)
        return g


def wavy(Q, n1=14, n2=22, amp=0.15, **kw):
    return GCase(Q, I.mapped_nodes(I.wavy_channel(n1, n2, amp=amp), n1, n2, "extend"), **kw)


def run_pair(case, prec, steps, seed=7, amplitude=5e-3):
    o = case.oracle()
    g = case.gpu(prec)
    st = o.state()
    if amplitude:
        st = st * (1.0 + I.smooth_field(st.shape, seed=seed, amplitude=amplitude))
        o.set_state(st)
        g.set_state(st)
    o.step(steps)
    g.step(steps)
    return o, g, st


@pytest.mark.parametrize("Q", [9, 21])
def test_fp64_wavy_channel_random_start(Q):
    """No-slip walls, body force along the channel, j-dependent start."""
    case = wavy(Q, g=(0.0, 1e-5))
    o, g, st = run_pair(case, 0, 200)
    assert vel_err(g.moments(), o.moments()) <= 1e-12
    so = o.state()
    assert np.sqrt(((g.state() - so) ** 2).sum() / (so ** 2).sum()) <= 1e-13


@pytest.mark.parametrize("Q", [9, 21])
def test_fp64_wavy_channel_moving_wall_from_rest(Q):
    """Moving low wall (the map is orthogonal at the walls), 400 steps."""
    case = wavy(Q, bc=(1, 0), U0=(0.02, 0.0))
    o, g, _ = run_pair(case, 0, 400, amplitude=0.0)
    assert vel_err(g.moments(), o.moments()) <= 1e-12


def test_fp64_general_implicit_force():
    case = wavy(21, g=(0.0, 1e-5), iters=1)
    o, g, _ = run_pair(case, 0, 100)
    assert vel_err(g.moments(), o.moments()) <= 1e-12


@pytest.mark.parametrize("prec,tol", [(1, 1e-5), (2, 3e-3), (3, 5e-2)])
def test_lower_precision_wavy_channel(prec, tol):
    case = wavy(21, bc=(1, 0), U0=(0.05, 0.0), g=(0.0, 1e-5))
    o, g, _ = run_pair(case, prec, 300, amplitude=0.0)
    assert vel_err(g.moments(), o.moments()) <= tol


def test_general_path_matches_planar_kind_on_the_gpu():
    """The planar grid's own nodes through the general path: the same state
    as the planar kind on the GPU (FP64)."""
    c = _clbm()
    n1, n2 = 12, 18
    e = I.geometric_stretch_edges(n1, 1.06, float(n1))
    dx = (e[-1] - e[0]) / n1
    knots = np.concatenate([[0.0], np.arange(n1) + 0.5, [float(n1)]])
    vals = np.concatenate([[e[0]], 0.5 * (e[:-1] + e[1:]), [e[-1]]])
    P = I.mapped_nodes(lambda q1, q2: (np.interp(q1, knots, vals), q2 * dx), n1, n2, "mirror")
    a = c.Grid(21, n1, n2, e, kind=c.PLANAR, step2=dx, precision=0, bc_lo=c.MOVING, bc_hi=c.NOSLIP)
    b = c.Grid(21, n1, n2, None, kind=c.GENERAL, nodes=P, dx=dx, precision=0, bc_lo=c.MOVING,
               bc_hi=c.NOSLIP)
    for g in (a, b):
        g.set_case(0.9, 1.0, 0.01, 0.0, (1e-6, 0.0))
    st = a.state() * (1.0 + I.smooth_field((21, n1, n2), seed=2, amplitude=1e-2))
    a.set_state(st)
    b.set_state(st)
    a.step(150)
    b.step(150)
    sa = a.state()
    assert np.abs(b.state() - sa).max() <= 1e-12 * np.abs(sa - st).max()


def test_general_residual_conserves_mass():
    case = wavy(21, g=(0.0, 1e-5))
    g = case.gpu(0)
    _, c0 = g.residual()
    g.step(300)
    _, c1 = g.residual()
    assert abs(c1[0] - c0[0]) <= 1e-12 * abs(c0[0])


def test_general_no_flow_adjustment_matches_oracle():
    case = wavy(21, n1=10, n2=14, amp=0.1)
    o = case.oracle()
    g = case.gpu(0)
    r_o = o.no_flow_adjust(2000)
    r_g = g.no_flow_adjust(2000)
    assert np.abs(r_g - r_o).max() <= 1e-11
    o.step(50)
    g.step(50)
    assert np.abs(g.moments()["rho"] - o.moments()["rho"]).max() <= 1e-11


def test_general_grid_refuses_row_table_kernel_and_batches():
    c = _clbm()
    case = wavy(21)
    g = case.gpu(1)
    with pytest.raises(c.ClbmError):
        g.set_kernel(2)
    g.set_kernel(3)
    with pytest.raises(c.ClbmError):
        c.Batch([g])


@pytest.mark.parametrize("Q,prec,n1,n2", [(21, 1, 20, 150), (9, 1, 13, 70), (21, 2, 20, 150)])
def test_general_grid_pipelined_and_per_cell_kernels_agree(Q, prec, n1, n2):
    """The TMA-staged pipeline (per-cell tables read by the consumers) and
    the per-cell kernel give the same populations on a wavy channel with a
    moving wall, several tiles and ragged edges."""
    c = _clbm()
    case = wavy(Q, n1=n1, n2=n2, bc=(1, 0), U0=(0.03, 0.0), g=(0.0, 1e-5))
    out = []
    for k in (1, 3):
        g = case.gpu(prec)
        g.set_kernel(k)
        st = g.state() * (1.0 + I.smooth_field((Q, n1, n2), seed=4, amplitude=2e-3))
        g.set_state(st)
        g.step(40)
        out.append(g.state())
        g.close()
    a, b = out
    assert np.abs(a - b).max() <= 1e-6 * np.abs(a).max()


def test_general_grid_fp32_pipelined_matches_oracle():
    case = wavy(21, n1=20, n2=150, bc=(1, 0), U0=(0.03, 0.0), g=(0.0, 1e-5))
    o = case.oracle()
    g = case.gpu(1)
    g.set_kernel(3)
    o.step(200)
    g.step(200)
    assert vel_err(g.moments(), o.moments()) <= 1e-5
