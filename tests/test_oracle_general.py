"""The oracle on general (non-separable) grids given by node positions (Sec. 2
in full generality: the metric, volume and Theta of every cell from the
positions around it).

Pins: an affine map has Theta = 0 and a constant metric; the general path fed
with the planar / polar node positions reproduces the planar / polar kinds
(themselves pinned by the exact solutions); on a sheared (affine,
non-orthogonal) channel between no-slip walls the rest state is a fixed point
and body-force driven flow converges to the parabola; on a non-separable wavy
channel mass is conserved and every cell's momentum changes by J F.
"""
import math

import numpy as np
import pytest

import clbm_inputs as I
from oracle import exact as E
from oracle import oracle as O


def planar_nodes(edges, n2, step2):
    """The planar kind's own nodes: edge midpoints across, (j - 1/2) step2
    along, ghosts mirrored through the walls."""
    n1 = len(edges) - 1
    knots = np.concatenate([[0.0], np.arange(n1) + 0.5, [float(n1)]])
    vals = np.concatenate([[edges[0]], 0.5 * (edges[:-1] + edges[1:]), [edges[-1]]])
    return I.mapped_nodes(lambda q1, q2: (np.interp(q1, knots, vals), q2 * step2), n1, n2, "mirror")


def general(Q, nodes, dx, **kw):
    n1, n2 = nodes.shape[0] - 8, nodes.shape[1] - 8
    return O.Grid(Q, n1, n2, O.GENERAL, nodes=nodes, dx=dx, **kw)


@pytest.mark.parametrize("Q", [9, 21])
def test_affine_map_has_no_christoffel_terms(Q):
    n1, n2 = 6, 5
    P = I.mapped_nodes(I.sheared_channel(n1, n2, h=1.0, L2=1.5, shear=0.4), n1, n2, "extend")
    g = general(Q, P, 1.0)
    ref = g.node_geometry(1, 1)
    assert ref["J"] == pytest.approx(1.5, rel=1e-14)
    for i in range(1, n1 + 1):
        for j in range(1, n2 + 1):
            geo = g.node_geometry(i, j)
            assert geo["J"] == pytest.approx(ref["J"], rel=1e-13)
            np.testing.assert_allclose(geo["ginv"], ref["ginv"], rtol=0, atol=1e-13)
            for a in range(1, Q):
                assert np.abs(g.theta(i, j, a, 1)).max() <= 1e-13


@pytest.mark.parametrize("Q", [9, 21])
def test_general_path_reproduces_planar_kind(Q):
    """Stretched planar grid, both walls moving, j-dependent start: the
    general path with the same nodes gives the planar kind's state."""
    n1, n2 = 12, 10
    e = I.geometric_stretch_edges(n1, 1.08, float(n1))
    dx = (e[-1] - e[0]) / n1
    a = O.Grid(Q, n1, n2, O.PLANAR, edges=e, step2=dx, bc_lo=O.MOVING, bc_hi=O.MOVING)
    b = general(Q, planar_nodes(e, n2, dx), dx, bc_lo=O.MOVING, bc_hi=O.MOVING)
    for g in (a, b):
        g.set_case(0.9, 1.0, 0.01, -0.02, (1e-6, 2e-6))
        g.init_rest()
    st = a.state() * (1.0 + I.smooth_field((Q, n1, n2), seed=3, amplitude=1e-2))
    a.set_state(st)
    b.set_state(st)
    a.step(150)
    b.step(150)
    ref = a.state() - st
    assert np.abs(b.state() - a.state()).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("Q", [9, 21])
def test_general_path_reproduces_polar_kind(Q):
    """Uniform annulus (mirroring through the circles continues the map):
    circular Couette from rest, the general path against the polar kind.
    The general path evaluates every column's geometry, so rounding makes
    its state slightly j-dependent, and on these cells (aspect 1.3 to 2.5)
    D2Q21 amplifies j-dependent modes about 20-fold per 50 steps: the
    comparison stops at 100 steps."""
    n1, n2 = 8, 40
    R1, R2 = 1.0, 2.0
    dr = (R2 - R1) / n1
    e = I.polar_edges(R1, R2, n1)
    th = 2.0 * math.pi / n2
    P = I.mapped_nodes(lambda q1, q2: ((R1 + q1 * dr) * np.cos(q2 * th), (R1 + q1 * dr) * np.sin(q2 * th)),
                       n1, n2, "extend")
    a = O.Grid(Q, n1, n2, O.POLAR, edges=e, bc_lo=O.MOVING, bc_hi=O.NOSLIP)
    b = general(Q, P, dr, bc_lo=O.MOVING, bc_hi=O.NOSLIP)
    U0 = 0.02 * dr / (R1 * math.sin(th))
    for g in (a, b):
        g.set_case(0.8, 1.0, U0, 0.0)
        g.init_rest()
        g.step(100)
    ma, mb = a.moments(), b.moments()
    assert np.abs(mb["Ut2"] - ma["Ut2"]).max() <= 2e-12 * np.abs(ma["Ut2"]).max()
    assert np.abs(mb["rho"] - ma["rho"]).max() <= 1e-12


@pytest.mark.parametrize("Q", [9, 21])
def test_sheared_channel_rest_is_a_fixed_point_and_poiseuille_converges(Q):
    """Affine parallelogram cells (shear 0.3) between no-slip walls: the rest
    state stays at rest, and a body force along the walls drives the
    parabola u = g x (H - x) / (2 nu), approached as n1 grows."""
    T0 = 1.0 / 3.0 if Q == 9 else 2.0 / 3.0
    tau = 1.0
    nu = E.nu_of_tau(tau, T0)
    errs = []
    for n1 in (8, 16):
        n2 = 4
        P = I.mapped_nodes(I.sheared_channel(n1, n2, shear=0.3), n1, n2, "extend")
        rest = general(Q, P, 1.0)
        rest.set_case(tau)
        rest.init_rest()
        s0 = rest.state()
        rest.step(200)
        assert np.abs(rest.state() - s0).max() <= 1e-13
        g_acc = 1e-5 * (8.0 / n1) ** 2
        g = general(Q, P, 1.0)
        g.set_case(tau, 1.0, 0.0, 0.0, (0.0, g_acc))
        g.init_rest()
        g.step(int(12 * n1 * n1 / (math.pi ** 2 * nu)) + 500)
        u = g.moments()["Ut2"][:, 0]            # g_2 = (0, 1): Ut^2 is the wall-parallel speed
        x = np.arange(n1) + 0.5
        ex = E.planar_poiseuille(x, float(n1), g_acc, nu)
        errs.append(np.abs(u - ex).max() / ex.max())
    assert errs[1] < errs[0] < 0.05


def test_wavy_channel_conserves_mass_and_balances_momentum():
    """Non-separable grid (wall-normal lines bent along the channel), D2Q21,
    no-slip walls, j-dependent start: total mass is constant to rounding and
    each cell's collision changes its momentum by J F (Eqs. 15, 17)."""
    Q, n1, n2 = 21, 10, 12
    P = I.mapped_nodes(I.wavy_channel(n1, n2, amp=0.15), n1, n2, "extend")
    g = general(Q, P, 1.0)
    g.set_case(0.8, 1.0, 0.0, 0.0, (0.0, 1e-5))
    g.init_rest()
    st = g.state() * (1.0 + I.smooth_field((Q, n1, n2), seed=11, amplitude=5e-3))
    g.set_state(st)
    m0 = g.totals()[0]
    for _ in range(5):
        g.step(20)
        assert abs(g.totals()[0] - m0) <= 1e-13 * abs(m0)
    c, _, _, _, _ = O.lattice(Q)
    for (i, j) in ((1, 1), (3, 7), (10, 12), (5, 4)):
        o = g.collide_one(i, j)
        J = g.volume()[i - 1, j - 1]
        assert abs(o["Npost"].sum() - o["Nin"].sum()) <= 1e-13 * o["Nin"].sum()
        dp = c.T.astype(float) @ (o["Npost"] - o["Nin"])
        np.testing.assert_allclose(dp, J * o["F"], rtol=1e-10, atol=1e-15)
