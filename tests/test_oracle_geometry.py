"""Pins of the oracle's geometry (Sec. 2, Eqs. 1-5; App. C; App. D)."""
import math

import numpy as np
import pytest

import clbm_inputs as I
from conftest import golden
from oracle import oracle as O


def _rot(phi):
    return np.array([[math.cos(phi), -math.sin(phi)], [math.sin(phi), math.cos(phi)]])


def _node_r(e, i):
    """Node coordinate of 1-based row i with mirrored ghosts (independent retype
    of the half-spaced lattice: nodes at edge midpoints, walls at the edges)."""
    n = len(e) - 1
    mid = lambda k: 0.5 * (e[k - 1] + e[k])
    if 1 <= i <= n:
        return mid(i)
    if i < 1:
        return 2 * e[0] - mid(1 - i)
    return 2 * e[n] - mid(2 * n + 1 - i)


@pytest.mark.parametrize("CR", [0.0, 0.35])
def test_polar_basis_app_d(CR):
    R1, R2, Nr, Nt = 1.0, 2.0, 16, 60
    e = I.polar_edges(R1, R2, Nr, CR)
    g = O.Grid(21, Nr, Nt, O.POLAR, edges=e)
    dbar = (R2 - R1) / Nr
    dth = 2 * math.pi / Nt
    for i in [-2, 0, 1, 5, Nr, Nr + 3]:
        for j in [-2, 1, 3]:
            geo = g.node_geometry(i, j)
            th = (j - 0.5) * dth
            rhat = np.array([math.cos(th), math.sin(th)])
            that = np.array([-math.sin(th), math.cos(th)])
            r = _node_r(e, i)
            s = (_node_r(e, i + 1) - _node_r(e, i - 1)) / (2 * dbar)
            g2n = math.sin(dth) / dbar * r
            np.testing.assert_allclose(geo["g1"], s * rhat, rtol=0, atol=1e-13)
            np.testing.assert_allclose(geo["g2"], g2n * that, rtol=0, atol=1e-12)
            assert abs(geo["J"] - s * g2n) < 1e-12 * s * g2n
            np.testing.assert_allclose(geo["ginv"], [[1 / s ** 2, 0], [0, 1 / g2n ** 2]],
                                       rtol=1e-12, atol=1e-15)
            # co-tangent vectors are dual to the tangent vectors (Eq. 3)
            G = np.array([geo["G1"], geo["G2"]])
            T = np.array([geo["g1"], geo["g2"]])
            np.testing.assert_allclose(G @ T.T, np.eye(2), atol=1e-13)


def test_polar_theta_closed_form():
    """Theta^k_m(q + c, q) from the rotated polar basis:
    g_1(i', th+phi) = s' rhat(th+phi), g_2(i', th+phi) = |g_2|' that(th+phi)."""
    R1, R2, Nr, Nt = 1.0, 3.0, 12, 40
    e = I.polar_edges(R1, R2, Nr, 0.2)
    g = O.Grid(21, Nr, Nt, O.POLAR, edges=e)
    c, *_ = O.lattice(21)
    dbar = (R2 - R1) / Nr
    dth = 2 * math.pi / Nt
    s = lambda i: (_node_r(e, i + 1) - _node_r(e, i - 1)) / (2 * dbar)
    gn = lambda i: math.sin(dth) / dbar * _node_r(e, i)
    for i in [1, 2, 3, 7, Nr - 1, Nr]:
        for a in range(21):
            for sg in (+1, -1):
                ip, phi = i + sg * c[a][0], sg * c[a][1] * dth
                want = np.array([
                    [(s(ip) * math.cos(phi) - s(i)) / s(i), -gn(ip) * math.sin(phi) / s(i)],
                    [s(ip) * math.sin(phi) / gn(i), (gn(ip) * math.cos(phi) - gn(i)) / gn(i)],
                ])
                got = g.theta(i, 5, a, sg)
                np.testing.assert_allclose(got, want, rtol=0, atol=2e-12)


def test_identity_metric_and_zero_christoffel():
    n1 = 10
    g = O.Grid(21, n1, 7, O.PLANAR, edges=I.uniform_edges(n1, 0.3), step2=0.3)
    for i in range(-2, n1 + 4):
        geo = g.node_geometry(i, 1)
        assert abs(geo["J"] - 1) < 1e-14
        np.testing.assert_allclose(geo["ginv"], np.eye(2), atol=1e-14)
    for a in range(21):
        for sg in (1, -1):
            assert np.abs(g.theta(2, 4, a, sg)).max() < 1e-14


def test_non_equilateral_uniform_cells():
    """dx/dy = 2 cells with Delta x = dy: J = 2, g^22 = 1/4, Theta = 0."""
    n1 = 16
    g = O.Grid(9, n1, 32, O.PLANAR, edges=I.uniform_edges(n1, 1.0), step2=2.0)
    geo = g.node_geometry(3, 1)
    assert abs(geo["J"] - 2) < 1e-14
    np.testing.assert_allclose(geo["ginv"], [[1, 0], [0, 0.25]], atol=1e-15)
    for a in range(9):
        assert np.abs(g.theta(1, 1, a, 1)).max() < 1e-14


def test_stretched_planar_theta():
    """Only g_1 varies (with i): Theta^1_1(q+c) = s(i+c1)/s(i) - 1, rest 0."""
    N = 16
    e = I.linear_contraction_edges(N, 0.4, 1.0)
    g = O.Grid(21, N, 5, O.PLANAR, edges=e, step2=1.0 / N)
    dbar = 1.0 / N
    s = lambda i: (_node_r(e, i + 1) - _node_r(e, i - 1)) / (2 * dbar)
    c, *_ = O.lattice(21)
    for i in [1, 2, 3, 8, 15, 16]:
        for a in range(21):
            th = g.theta(i, 2, a, 1)
            want = np.zeros((2, 2))
            want[0, 0] = s(i + c[a][0]) / s(i) - 1
            np.testing.assert_allclose(th, want, atol=1e-13)


def test_mirror_ghost_geometry_is_symmetric():
    """Ghost rows mirror the fluid rows through the wall (App. B)."""
    N = 12
    e = I.linear_contraction_edges(N, 0.3, 2.0)
    g = O.Grid(21, N, 4, O.PLANAR, edges=e, step2=1.0)
    for k in (1, 2, 3):
        lo_g, lo_f = g.node_geometry(1 - k, 1), g.node_geometry(k, 1)
        assert abs(lo_g["J"] - lo_f["J"]) < 1e-13
        hi_g, hi_f = g.node_geometry(N + k, 1), g.node_geometry(N + 1 - k, 1)
        assert abs(hi_g["J"] - hi_f["J"]) < 1e-13


def test_contraction_worked_example():
    vals = {}
    for line in open(golden("contraction_example.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    CR = vals["CR"]
    for N in (8, 16, 32, 64, 128):
        e = I.linear_contraction_edges(N, CR, 1.0)
        d = np.diff(e)
        dbar = 1.0 / N
        assert abs(d[0] / dbar - vals["first_over_avg"]) < 1e-12
        assert abs(d[N // 2 - 1] / d[0] - vals["middle_over_first"]) < 5e-3
        assert abs(d[0] / d[N // 2 - 1] - (1 - CR) / (1 + CR)) < 1e-12
        # boundary values and symmetry of App. C
        assert abs(e[0]) < 1e-15 and abs(e[N // 2] - 0.5) < 1e-14 and abs(e[N] - 1.0) < 1e-14
        np.testing.assert_allclose(d, d[::-1], atol=1e-14)
        # the step law of App. C on both halves
        a = 2 * CR / (N / 2 - 1)
        for i in range(1, N + 1):
            want = (1 + a * (i - N / 4 - 0.5)) if i <= N // 2 else (1 - a * (i - 3 * N / 4 - 0.5))
            assert abs(d[i - 1] / dbar - want) < 1e-12


def test_polar_rejects_ghosts_through_origin():
    with pytest.raises(ValueError):
        O.Grid(21, 16, 40, O.POLAR, edges=I.polar_edges(1.0, 11.0, 16))
