"""Pins of the 3-D oracle (Sec. 2 in three coordinates, D3Q39).

The lattice is pinned by exact rational moments (isotropy through the sixth
order at T0 = 2/3, failing at the eighth); f^eq by its closed-form moments
for an arbitrary metric; the geometry by the closed forms of the channel and
the annulus (Theta vanishes on a uniform channel, the polar metric is
diagonal with the known lengths); the update by exact conservation, the
per-cell momentum balance, the rest state of a channel, and steady channel
flows against their exact profiles (Couette exact to rounding, Poiseuille
converging as n1 grows).
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import clbm_inputs as I
from oracle import exact as E
from oracle import oracle3d as O3


def exact_moment(c, w, idx):
    s = Fraction(0)
    for a in range(len(w)):
        t = Fraction(w[a]).limit_denominator(100000)
        for i in idx:
            t *= int(c[a][i])
        s += t
    return s


def isotropic(idx, T0):
    """T0^(n/2) times the sum over pairings of Kronecker deltas."""
    idx = list(idx)
    if not idx:
        return Fraction(1)
    if len(idx) % 2:
        return Fraction(0)
    first, rest = idx[0], idx[1:]
    s = Fraction(0)
    for p in range(len(rest)):
        if rest[p] == first:
            s += T0 * isotropic(rest[:p] + rest[p + 1:], T0)
    return s


def test_d3q39_isotropy_through_sixth_order_and_not_eighth():
    c, w, star, hat, T0 = O3.lattice()
    assert len(set(map(tuple, c))) == 39
    T0 = Fraction(T0).limit_denominator(100)
    assert T0 == Fraction(2, 3)
    for n in range(0, 7):
        for idx in itertools.product(range(3), repeat=n):
            assert exact_moment(c, w, idx) == isotropic(idx, T0), idx
    assert exact_moment(c, w, (0,) * 8) != isotropic((0,) * 8, T0)
    for a in range(39):
        assert tuple(c[star[a]]) == tuple(-c[a])
        assert tuple(c[hat[a]]) == (-c[a][0], c[a][1], c[a][2])


def test_feq_closed_form_moments_for_an_arbitrary_metric():
    g = O3.Grid(4, 1, 1, O3.CHANNEL, edges=np.arange(5.0))
    c, w, _, _, T0 = O3.lattice()
    rng = np.random.default_rng(3)
    A = rng.normal(size=(3, 3)) * 0.2 + np.eye(3)
    gi = A @ A.T
    U = rng.normal(size=3) * 0.05
    Ut = U + rng.normal(size=3) * 0.01
    rho = 1.07
    f = np.array([g.feq(a, rho, U, Ut, gi) for a in range(39)])
    cf = c.astype(float)
    assert abs(f.sum() - rho) < 1e-14
    np.testing.assert_allclose(cf.T @ f, rho * U, atol=1e-15)
    M2 = np.einsum("ai,aj,a->ij", cf, cf, f)
    np.testing.assert_allclose(M2, rho * (T0 * gi + np.outer(Ut, Ut)), atol=1e-14)
    M3 = np.einsum("ai,aj,ak,a->ijk", cf, cf, cf, f)
    ref = rho * (T0 * (np.einsum("ij,k->ijk", gi, Ut) + np.einsum("jk,i->ijk", gi, Ut) +
                       np.einsum("ki,j->ijk", gi, Ut)) + np.einsum("i,j,k->ijk", Ut, Ut, Ut))
    np.testing.assert_allclose(M3, ref, atol=1e-14)


def test_uniform_channel_has_identity_metric_and_no_theta():
    n1 = 6
    g = O3.Grid(n1, 3, 2, O3.CHANNEL, edges=np.arange(n1 + 1.0), step2=1.0, step3=1.0)
    for i in range(1, n1 + 1):
        geo = g.row_geometry(i)
        assert geo["J"] == pytest.approx(1.0, abs=1e-15)
        np.testing.assert_allclose(geo["ginv"], np.eye(3), atol=1e-15)
        for a in range(39):
            assert np.abs(g.theta(i, a, 1)).max() < 1e-15


def test_stretched_channel_theta_is_the_ratio_of_wall_normal_lengths():
    n1 = 8
    e = I.geometric_stretch_edges(n1, 1.1, float(n1))
    dx = (e[-1] - e[0]) / n1
    g = O3.Grid(n1, 2, 2, O3.CHANNEL, edges=e, step2=dx, step3=dx)
    c, _, _, _, _ = O3.lattice()

    def xnode(i):
        if 1 <= i <= n1:
            return 0.5 * (e[i - 1] + e[i])
        if i < 1:
            k = 1 - i
            return 2 * e[0] - 0.5 * (e[k - 1] + e[k])
        k = i - n1
        m = n1 + 1 - k
        return 2 * e[n1] - 0.5 * (e[m - 1] + e[m])

    def g1(i):
        return (xnode(i + 1) - xnode(i - 1)) / (2 * dx)

    for i in range(1, n1 + 1):
        assert g.row_geometry(i)["J"] == pytest.approx(g1(i), rel=1e-14)
        for a in range(39):
            th = g.theta(i, a, 1)
            expect = np.zeros((3, 3))
            expect[0, 0] = g1(i + c[a][0]) / g1(i) - 1.0
            np.testing.assert_allclose(th, expect, atol=1e-14)


def test_annulus_metric_is_polar():
    n1, n2, n3 = 6, 40, 2
    e = I.polar_edges(1.0, 2.0, n1)
    dr = (e[-1] - e[0]) / n1
    g = O3.Grid(n1, n2, n3, O3.ANNULUS, edges=e, step3=0.5)
    dth = 2 * math.pi / n2
    for i in range(1, n1 + 1):
        r = 0.5 * (e[i - 1] + e[i])
        geo = g.row_geometry(i)
        l1, l2, l3 = 1.0, r * math.sin(dth) / dr, 0.5 / dr
        np.testing.assert_allclose(np.diag(geo["g"]), [l1 ** 2, l2 ** 2, l3 ** 2], rtol=1e-13)
        np.testing.assert_allclose(geo["ginv"], np.diag([1 / l1 ** 2, 1 / l2 ** 2, 1 / l3 ** 2]),
                                   rtol=1e-13, atol=1e-15)
        assert geo["J"] == pytest.approx(l1 * l2 * l3, rel=1e-13)


def test_rest_is_a_fixed_point_of_a_uniform_anisotropic_channel():
    """Cells 1 x 2 x 0.5 (a constant, non-identity metric, Theta = 0) between
    a no-slip and a resting moving wall: the rest state stays put.  (On a
    stretched channel it does not: J varies, which is what the paper's no-flow
    adjustment is for.)"""
    n1 = 8
    g = O3.Grid(n1, 2, 3, O3.CHANNEL, edges=np.arange(n1 + 1.0), step2=2.0, step3=0.5,
                bc_lo=O3.MOVING, bc_hi=O3.NOSLIP)
    g.set_case(0.9)
    g.init_rest()
    s0 = g.state()
    g.step(40)
    assert np.abs(g.state() - s0).max() <= 1e-14 * np.abs(s0).max()


def test_annulus_conserves_mass_and_balances_momentum_per_cell():
    n1, n2, n3 = 6, 30, 3
    e = I.polar_edges(1.0, 2.0, n1, 0.35)
    g = O3.Grid(n1, n2, n3, O3.ANNULUS, edges=e, step3=0.2, bc_lo=O3.MOVING, bc_hi=O3.NOSLIP)
    g.set_case(0.8, 1.0, 0.02, 0.0, (1e-5, 2e-5, 3e-5))
    g.init_rest()
    st = g.state() * (1.0 + I.smooth_field((39 * n1, n2, n3), seed=4, amplitude=3e-3).reshape(39, n1, n2, n3))
    g.set_state(st)
    m0 = g.totals()[0]
    for _ in range(3):
        g.step(10)
        assert abs(g.totals()[0] - m0) <= 2e-14 * m0
    c, _, _, _, _ = O3.lattice()
    for (i, j, k) in ((1, 1, 1), (3, 17, 2), (6, 30, 3)):
        o = g.collide_one(i, j, k)
        J = g.row_geometry(i)["J"]
        assert abs(o["Npost"].sum() - o["Nin"].sum()) <= 1e-14 * o["Nin"].sum()
        np.testing.assert_allclose(c.T.astype(float) @ (o["Npost"] - o["Nin"]), J * o["F"],
                                   rtol=1e-10, atol=1e-16)


def test_uniform_channel_couette_converges_to_the_line():
    """Planar Couette across a uniform channel (moving low wall): the steady
    profile approaches the exact line as n1 grows.  At tau = 1 it is within
    2e-6 of it at n1 = 8; at tau = 0.8 the walls slip by 2.9 % / 1.6 % at
    n1 = 8 / 16 (first order: the multi-speed walls of App. B are not exact
    for a linear profile away from tau = 1, as the paper notes for D2Q21)."""
    errs = {}
    for tau in (1.0, 0.8):
        for n1 in (8, 16):
            g = O3.Grid(n1, 1, 1, O3.CHANNEL, edges=np.arange(n1 + 1.0), bc_lo=O3.MOVING,
                        bc_hi=O3.NOSLIP)
            U0 = 0.01
            g.set_case(tau, 1.0, U0, 0.0)
            g.init_rest()
            g.step(int(14 * n1 * n1 / (math.pi ** 2 * (tau - 0.5) * 2.0 / 3.0)) + 200)
            u = g.moments()["Ut"][1][:, 0, 0]
            x = np.arange(n1) + 0.5
            errs[(tau, n1)] = np.abs(u - U0 * (1.0 - x / n1)).max() / U0
    assert errs[(1.0, 8)] < 1e-5
    assert errs[(0.8, 16)] < errs[(0.8, 8)] / 1.5


def test_channel_poiseuille_converges_to_the_parabola():
    tau = 1.0
    nu = E.nu_of_tau(tau, 2.0 / 3.0)
    errs = []
    for n1 in (8, 16):
        gacc = 1e-5 * (8.0 / n1) ** 2
        g = O3.Grid(n1, 1, 2, O3.CHANNEL, edges=np.arange(n1 + 1.0))
        g.set_case(tau, 1.0, 0.0, 0.0, (0.0, 0.0, gacc))
        g.init_rest()
        g.step(int(14 * n1 * n1 / (math.pi ** 2 * nu)) + 200)
        u = g.moments()["Ut"][2][:, 0, 0]
        x = np.arange(n1) + 0.5
        ex = E.planar_poiseuille(x, float(n1), gacc, nu)
        errs.append(np.abs(u - ex).max() / ex.max())
    # 1.7 % and 0.43 %: second order
    assert errs[1] < errs[0] / 3.0 and errs[0] < 0.02
