"""Pins of the oracle's flow diagnostics (Sec. 3.1: a steady state is judged
by the kinetic energy and, for the circular flows, the angular momentum no
longer changing; mass is conserved throughout).

The diagnostics are checked against what the geometry and the mathematics
fix, not against a retyped formula:
  * a rigid rotation u = Omega z x x has angular momentum exactly 2 KE / Omega
    for any density field, and max |u| = Omega r at the outermost node;
  * a radial source flow u = s r_hat / r carries no angular momentum;
  * on the annulus the sums converge, at second order, to the closed-form
    integrals of the exact circular Couette profile (Eq. 27): KE, angular
    momentum and the J-weighted residual norms;
  * on the uniform channel of the planar Couette configuration (cells twice
    as long as wide) a uniform flow has speed 2 U^2 and the kinetic energy of
    the channel's area;
  * the general path fed with the annulus' node positions gives the polar
    kind's diagnostics for j-dependent fields (every column evaluated
    against column 1 turned about the origin);
  * the residual is 0 for an unchanged field, exactly eps / dt for a field
    scaled by 1 - eps, and +inf without a previous field.
"""
import math

import numpy as np
import pytest

import clbm_inputs as I
from oracle import exact as E
from oracle import oracle as O


def annulus(n1, n2, R1=1.0, R2=2.0, CR=0.0, Q=21):
    return O.Grid(Q, n1, n2, O.POLAR, edges=I.polar_edges(R1, R2, n1, CR))


def node_r(edges):
    return 0.5 * (edges[:-1] + edges[1:])


def contravariant_of(g, ux, uy):
    """Contravariant components of a physical velocity given per row at the
    column-1 node (the co-tangent vectors of that node project it)."""
    U1 = np.empty(g.n1)
    U2 = np.empty(g.n1)
    for i in range(1, g.n1 + 1):
        geo = g.node_geometry(i, 1)
        U1[i - 1] = ux[i - 1] * geo["G1"][0] + uy[i - 1] * geo["G1"][1]
        U2[i - 1] = ux[i - 1] * geo["G2"][0] + uy[i - 1] * geo["G2"][1]
    return np.repeat(U1[:, None], g.n2, 1), np.repeat(U2[:, None], g.n2, 1)


def column1_positions(edges, n2):
    r = node_r(edges)
    th = 0.5 * 2.0 * math.pi / n2
    return r * math.cos(th), r * math.sin(th)


def test_rigid_rotation_angular_momentum_is_twice_energy_over_omega():
    n1, n2, Om = 16, 64, 3e-3
    e = I.polar_edges(1.0, 2.0, n1, 0.35)
    g = annulus(n1, n2, CR=0.35)
    x, y = column1_positions(e, n2)
    U1, U2 = contravariant_of(g, -Om * y, Om * x)
    rho = 1.0 + 0.2 * I.white_field((n1, n2), seed=5)
    d = g.flow_diagnostics(rho, U1, U2)
    assert d["am"] > 0.0
    assert d["am"] == pytest.approx(2.0 * d["ke"] / Om, rel=1e-13)
    assert d["umax"] == pytest.approx(Om * node_r(e)[-1], rel=1e-13)
    assert d["res"] == math.inf


def test_radial_flow_carries_no_angular_momentum():
    n1, n2, s = 16, 64, 1e-2
    e = I.polar_edges(1.0, 2.0, n1)
    g = annulus(n1, n2)
    x, y = column1_positions(e, n2)
    r2 = x * x + y * y
    U1, U2 = contravariant_of(g, s * x / r2, s * y / r2)
    d = g.flow_diagnostics(np.ones((n1, n2)), U1, U2)
    assert abs(d["am"]) <= 1e-14 * d["ke"] / s * 2.0
    assert d["umax"] == pytest.approx(s / node_r(e)[0], rel=1e-13)


def couette_integrals(R1, R2, U1):
    """KE, angular momentum and the residual norms of the exact circular
    Couette profile over the annulus, per unit density (continuous)."""
    A = E.Annulus.couette(R1, R2, U1 / R1)
    a, b = A.a, A.b

    def I2(r0, r1):  # integral of u^2 r dr
        F = lambda r: a * a * r ** 4 / 4.0 + a * b * r * r + b * b * math.log(r)
        return F(r1) - F(r0)

    ke = math.pi * I2(R1, R2)
    am = 2.0 * math.pi * (a * (R2 ** 4 - R1 ** 4) / 4.0 + b * (R2 ** 2 - R1 ** 2) / 2.0)
    return A, ke, am, I2


def test_couette_totals_converge_to_the_closed_form_integrals():
    """Uniform annulus R1 = 1, R2 = 2, exact Couette profile with the inner
    wall at 0.01: the J-weighted sums (cell volumes in units of Delta x^2)
    converge to the integrals over the annulus at second order."""
    R1, R2, U1 = 1.0, 2.0, 0.01
    A, ke_c, am_c, I2 = couette_integrals(R1, R2, U1)
    errs = []
    for n1 in (8, 16, 32):
        n2 = 4 * n1
        e = I.polar_edges(R1, R2, n1)
        dx = (R2 - R1) / n1
        g = annulus(n1, n2)
        x, y = column1_positions(e, n2)
        r = np.sqrt(x * x + y * y)
        u = A.u(r)
        U1f, U2f = contravariant_of(g, -u * y / r, u * x / r)
        d = g.flow_diagnostics(np.ones((n1, n2)), U1f, U2f)
        ke = d["ke"] * dx * dx
        am = d["am"] * dx * dx
        errs.append((abs(ke / ke_c - 1.0), abs(am / am_c - 1.0)))
        assert d["umax"] == pytest.approx(A.u(node_r(e)[0]), rel=1e-13)
        assert d["uu"] * dx * dx == pytest.approx(2.0 * ke, rel=1e-13)
        # residual against a field that differs in the inner half only
        prev1, prev2 = U1f.copy(), U2f.copy()
        inner = node_r(e) < 0.5 * (R1 + R2)
        prev1[inner] = 0.0
        prev2[inner] = 0.0
        dt = 7
        res = g.flow_diagnostics(np.ones((n1, n2)), U1f, U2f, (prev1, prev2), dt)["res"]
        expect = math.sqrt(I2(R1, 0.5 * (R1 + R2)) / I2(R1, R2)) / dt
        errs[-1] = errs[-1] + (abs(res / expect - 1.0),)
    errs = np.array(errs)
    assert (errs[-1] < 2e-3).all(), errs
    ratios = errs[:-1] / errs[1:]
    assert (ratios > 3.5).all() and (ratios < 4.6).all(), ratios


def test_uniform_flow_on_the_planar_couette_cells():
    """n1 = 16 rows by n2 = 32 columns of cells twice as long along q^2
    (Delta x = 1, step2 = 2): Ut^2 = U moves 2 U per step, the channel's area
    is 2 n1 n2, no angular momentum is reported on planar grids."""
    n1, n2, U = 16, 32, 3e-3
    g = O.Grid(9, n1, n2, O.PLANAR, edges=I.uniform_edges(n1), step2=2.0)
    rho0 = 1.1
    d = g.flow_diagnostics(np.full((n1, n2), rho0), np.zeros((n1, n2)), np.full((n1, n2), U))
    assert d["umax"] == pytest.approx(2.0 * U, rel=1e-14)
    assert d["ke"] == pytest.approx(0.5 * rho0 * (2.0 * n1 * n2) * (2.0 * U) ** 2, rel=1e-13)
    assert d["am"] == 0.0


def test_general_path_gives_the_polar_diagnostics():
    """j-dependent random fields on the uniform annulus: the general path
    (every column's own node and tangents) against the polar kind (column 1
    turned about the origin)."""
    n1, n2 = 8, 40
    R1, R2 = 1.0, 2.0
    dr = (R2 - R1) / n1
    th = 2.0 * math.pi / n2
    P = I.mapped_nodes(lambda q1, q2: ((R1 + q1 * dr) * np.cos(q2 * th),
                                       (R1 + q1 * dr) * np.sin(q2 * th)), n1, n2, "extend")
    a = annulus(n1, n2, Q=9)
    b = O.Grid(9, n1, n2, O.GENERAL, nodes=P, dx=dr)
    rho = 1.0 + 0.1 * I.white_field((n1, n2), seed=2)
    U1 = 1e-2 * I.white_field((n1, n2), seed=3)
    U2 = 1e-2 * I.white_field((n1, n2), seed=4)
    prev = (U1 * 0.9 + 1e-3 * I.white_field((n1, n2), seed=6), U2 * 1.1)
    da = a.flow_diagnostics(rho, U1, U2, prev, 3)
    db = b.flow_diagnostics(rho, U1, U2, prev, 3)
    for k in ("res", "ke", "am", "umax", "uu"):
        assert db[k] == pytest.approx(da[k], rel=1e-12), k
    assert abs(da["am"]) > 0.0


def test_residual_special_cases():
    n1, n2 = 12, 48
    g = annulus(n1, n2, CR=0.35)
    rho = 1.0 + 0.1 * I.white_field((n1, n2), seed=8)
    U1 = 1e-3 * I.smooth_field((n1, n2), seed=9)
    U2 = 1e-2 * I.smooth_field((n1, n2), seed=10)
    assert g.flow_diagnostics(rho, U1, U2, (U1, U2), 5)["res"] == 0.0
    eps, dt = 0.03, 11
    r = g.flow_diagnostics(rho, U1, U2, ((1 - eps) * U1, (1 - eps) * U2), dt)["res"]
    assert r == pytest.approx(eps / dt, rel=1e-12)
    assert g.flow_diagnostics(rho, U1, U2, None, 5)["res"] == math.inf
    assert g.flow_diagnostics(rho, U1, U2, (U1, U2), 0)["res"] == math.inf
    z = np.zeros((n1, n2))
    assert g.flow_diagnostics(rho, z, z, (z, z), 5)["res"] == 0.0


def test_diagnostics_of_a_run_follow_the_state():
    """diagnostics() of a circular Couette run from rest: mass from the
    state's totals stays fixed, the residual falls to the rounding floor as
    the flow settles, and KE and angular momentum then stop changing (the
    criterion of Sec. 3.1)."""
    n1, n2 = 8, 50
    e = I.polar_edges(1.0, 2.0, n1)
    g = O.Grid(21, n1, n2, O.POLAR, edges=e, bc_lo=O.MOVING, bc_hi=O.NOSLIP)
    th = 2.0 * math.pi / n2
    g.set_case(0.8, 1.0, 0.01 * (1.0 / n1) / (1.0 * math.sin(th)), 0.0)
    g.init_rest()
    g.step(100)
    hist = [g.diagnostics()]
    for _ in range(6):
        g.step(200)
        p = hist[-1]
        hist.append(g.diagnostics((p["Ut1"], p["Ut2"]), 200))
    res = [d["res"] for d in hist]
    assert res[0] == math.inf and all(math.isfinite(r) for r in res[1:])
    assert res[1] > res[2] > res[3] and res[-1] < 1e-14
    assert hist[-1]["am"] > 0.0
    assert hist[-1]["ke"] == pytest.approx(hist[-2]["ke"], rel=1e-13)
    assert hist[-1]["am"] == pytest.approx(hist[-2]["am"], rel=1e-13)
    for d in hist:
        assert d["totals"][0] == pytest.approx(hist[0]["totals"][0], rel=1e-13)
