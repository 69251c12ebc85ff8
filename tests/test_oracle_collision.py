"""Pins of the oracle's collision step (Sec. 2, Eqs. 6-19)."""
import math

import numpy as np
import pytest

import clbm_inputs as I
from oracle import oracle as O


def _spd(rng):
    a = rng.uniform(0.3, 2.0)
    b = rng.uniform(0.3, 2.0)
    c = rng.uniform(-0.3, 0.3) * math.sqrt(a * b)
    return np.array([[a, c], [c, b]])


def _grid(Q=21):
    return O.Grid(Q, 8, 4, O.PLANAR, edges=I.uniform_edges(8), step2=1.0)


@pytest.mark.parametrize("seed", range(5))
def test_equilibrium_moments_d2q21(seed):
    """Eq. 19 on D2Q21: sum f = rho, sum c f = rho U,
    sum cc f = rho (T0 g^ij + Ut^i Ut^j),
    sum ccc f = rho [T0 (g^ij Ut^k + g^jk Ut^i + g^ki Ut^j) + Ut^i Ut^j Ut^k]."""
    rng = np.random.default_rng(seed)
    g = _grid(21)
    c, w, _, _, T0 = O.lattice(21)
    gi = _spd(rng)
    rho = rng.uniform(0.8, 1.2)
    U = rng.uniform(-0.1, 0.1, 2)
    Ut = U + rng.uniform(-0.05, 0.05, 2)
    f = np.array([g.feq(a, rho, U, Ut, gi) for a in range(21)])
    cf = c.astype(float)
    assert abs(f.sum() - rho) < 1e-14
    np.testing.assert_allclose(cf.T @ f, rho * U, atol=1e-15)
    M2 = np.einsum("a,ai,aj->ij", f, cf, cf)
    np.testing.assert_allclose(M2, rho * (T0 * gi + np.outer(Ut, Ut)), atol=1e-14)
    M3 = np.einsum("a,ai,aj,ak->ijk", f, cf, cf, cf)
    want = np.zeros((2, 2, 2))
    for i in range(2):
        for j in range(2):
            for k in range(2):
                want[i, j, k] = rho * (T0 * (gi[i, j] * Ut[k] + gi[j, k] * Ut[i] + gi[k, i] * Ut[j])
                                       + Ut[i] * Ut[j] * Ut[k])
    np.testing.assert_allclose(M3, want, atol=1e-14)


def test_equilibrium_third_moment_fails_on_d2q9():
    """D2Q9 lacks 6th-order isotropy, so its third equilibrium moment is wrong."""
    rng = np.random.default_rng(7)
    g = _grid(9)
    c, w, _, _, T0 = O.lattice(9)
    gi = _spd(rng)
    U = np.array([0.05, 0.03])
    f = np.array([g.feq(a, 1.0, U, U, gi) for a in range(9)])
    cf = c.astype(float)
    M3 = np.einsum("a,ai,aj,ak->ijk", f, cf, cf, cf)
    want = T0 * 3 * gi[0, 0] * U[0] + U[0] ** 3
    assert abs(M3[0, 0, 0] - want) > 1e-3


def test_identity_metric_equilibrium_is_textbook_hermite():
    """g = delta, U = Ut: the third-order Hermite equilibrium of Cartesian LBM,
    w rho [1 + cu/T + ((cu)^2 - T u^2)/2T^2 + ((cu)^3 - 3 T (cu) u^2)/6T^3]."""
    for Q in (9, 21):
        g = _grid(Q)
        c, w, _, _, T = O.lattice(Q)
        u = np.array([0.07, -0.04])
        for a in range(Q):
            cu = c[a] @ u
            uu = u @ u
            want = w[a] * 1.1 * (1 + cu / T + (cu ** 2 - T * uu) / (2 * T ** 2)
                                 + (cu ** 3 - 3 * T * cu * uu) / (6 * T ** 3))
            assert abs(g.feq(a, 1.1, u, u, np.eye(2)) - want) < 1e-15


def _perturbed_grid(Q, kind, bc_lo, bc_hi, seed, amp=2e-3, gext=(0.0, 0.0)):
    if kind == O.POLAR:
        n1, n2 = 12, 50
        g = O.Grid(Q, n1, n2, O.POLAR, edges=I.polar_edges(1.0, 2.0, n1, 0.3), bc_lo=bc_lo, bc_hi=bc_hi)
    else:
        n1, n2 = 12, 9
        g = O.Grid(Q, n1, n2, O.PLANAR, edges=I.linear_contraction_edges(n1, 0.35, 12.0),
                   step2=1.3, bc_lo=bc_lo, bc_hi=bc_hi)
    g.set_case(0.8, 1.0, 0.02, -0.01, gext)
    g.init_rest()
    st = g.state()
    g.set_state(st * (1 + I.white_field(st.shape, seed=seed, amplitude=amp)))
    g.step(3)
    return g


@pytest.mark.parametrize("Q", [9, 21])
@pytest.mark.parametrize("kind", [O.PLANAR, O.POLAR])
def test_cell_conserves_mass_and_adds_JF(Q, kind):
    """Per cell: sum_a (N' - N) = 0 and sum_a c_a (N' - N) = J F (Eqs. 6, 11, 17)."""
    g = _perturbed_grid(Q, kind, O.MOVING, O.NOSLIP, seed=3, gext=(1e-4, -2e-4))
    c, w, _, _, T0 = O.lattice(Q)
    J = g.volume()
    for (i, j) in [(1, 1), (2, 5), (6, 3), (g.n1, 2), (g.n1 - 1, g.n2)]:
        o = g.collide_one(i, j)
        d = o["Npost"] - o["Nin"]
        assert abs(d.sum()) < 1e-14
        np.testing.assert_allclose(c.T.astype(float) @ d, J[i - 1, j - 1] * o["F"], atol=1e-14)
        # the source term alone: sum dN = 0, sum c dN = J F, sum cc dN = 2 J sym(dPi)
        dN = o["dN"]
        cf = c.astype(float)
        assert abs(dN.sum()) < 1e-15
        np.testing.assert_allclose(cf.T @ dN, J[i - 1, j - 1] * o["F"], atol=1e-15)
        M2 = np.einsum("a,ai,aj->ij", dN, cf, cf)
        np.testing.assert_allclose(M2, J[i - 1, j - 1] * (o["dPi"] + o["dPi"].T), atol=1e-15)


def test_force_vanishes_on_identity_metric_without_body_force():
    g = O.Grid(21, 10, 6, O.PLANAR, edges=I.uniform_edges(10), step2=1.0, bc_lo=O.NOSLIP, bc_hi=O.NOSLIP)
    g.set_case(0.9)
    g.init_rest()
    st = g.state()
    g.set_state(st * (1 + I.white_field(st.shape, seed=1, amplitude=1e-2)))
    for (i, j) in [(1, 1), (5, 3), (10, 6)]:
        o = g.collide_one(i, j)
        assert np.abs(o["F"]).max() < 1e-16
        assert np.abs(o["dPi"]).max() < 1e-16
        assert np.abs(o["dN"]).max() < 1e-16


def test_body_force_enters_force_and_velocity():
    """Reading R5: F^k gets rho g^k, and Ut = U + F/(2 rho) (Eq. 18)."""
    g = O.Grid(9, 8, 4, O.PLANAR, edges=I.uniform_edges(8), step2=1.0)
    g.set_case(1.0, 1.0, 0.0, 0.0, (0.0, 3e-3))
    g.init_rest()
    o = g.collide_one(4, 2)
    assert abs(o["F"][1] - 3e-3 * o["rho"]) < 1e-17
    assert abs(o["Ut"][1] - 1.5e-3) < 1e-17


def test_christoffel_force_is_outward_at_rest_in_polar_cells():
    """At rest the azimuthal populations push outward (centrifugal sign)."""
    g = O.Grid(21, 16, 60, O.POLAR, edges=I.polar_edges(1.0, 2.0, 16))
    g.set_case(1.0)
    g.init_rest()
    assert g.collide_one(8, 1)["F"][0] > 0
