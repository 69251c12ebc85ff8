"""Equilibrium start from macroscopic fields on the GPU (clbm_set_equilibrium):
N'(q,-1) = J f^eq(rho, U, Ut = U; g^{ij}(q)) of Eq. 19, against the oracle's
own f^eq cell by cell, against the moments the equilibrium must carry, and
through the steps that follow (moving walls read the start's moments)."""
import math

import numpy as np
import pytest

import clbm_inputs as I
from oracle import exact as E
from oracle import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _clbm():
    from paper_2301_01868_gb300 import clbm
    return clbm


def fields(n1, n2, seed):
    rho = 1.0 + I.smooth_field((n1, n2), seed=seed, amplitude=0.02)
    U1 = I.smooth_field((n1, n2), seed=seed + 1, amplitude=0.01)
    U2 = I.smooth_field((n1, n2), seed=seed + 2, amplitude=0.01)
    return rho, U1, U2


def oracle_equilibrium(o, rho, U1, U2):
    """J f^eq per cell from the oracle's f^eq; the annulus's geometry is that
    of column 1 in every column (the oracle keeps one column)."""
    N = np.empty((o.Q, o.n1, o.n2))
    for i in range(o.n1):
        geo = o.node_geometry(i + 1, 1)
        for j in range(o.n2):
            U = np.array([U1[i, j], U2[i, j]])
            for a in range(o.Q):
                N[a, i, j] = geo["J"] * o.feq(a, rho[i, j], U, U, geo["ginv"])
    return N


def annulus_pair(Q, prec, n1=8, n2=40):
    c = _clbm()
    e = I.polar_edges(1.0, 2.0, n1, 0.35)
    o = O.Grid(Q, n1, n2, O.POLAR, edges=e, bc_lo=O.MOVING, bc_hi=O.NOSLIP)
    g = c.Grid(Q, n1, n2, e, kind=c.POLAR, precision=prec, bc_lo=c.MOVING, bc_hi=c.NOSLIP)
    return o, g


@pytest.mark.parametrize("Q", [9, 21])
def test_equilibrium_matches_oracle_feq_and_carries_its_moments(Q):
    o, g = annulus_pair(Q, 0)
    o.set_case(0.8, 1.0, 0.01, 0.0)
    g.set_case(0.8, 1.0, 0.01, 0.0)
    rho, U1, U2 = fields(o.n1, o.n2, 31)
    g.set_equilibrium(rho, U1, U2)
    N = g.state()
    ref = oracle_equilibrium(o, rho, U1, U2)
    assert np.abs(N - ref).max() <= 1e-14 * np.abs(ref).max()
    # sum N = J rho and sum c N = J rho U (Eqs. 7, 8), whatever computed them
    cvec, _, _, _, _ = O.lattice(Q)
    J = o.volume()
    assert np.abs(N.sum(0) - J * rho).max() <= 1e-14 * np.abs(J * rho).max()
    mom = np.tensordot(cvec.T.astype(float), N, axes=(1, 0))
    np.testing.assert_allclose(mom[0], J * rho * U1, rtol=0, atol=1e-14 * np.abs(J).max())
    np.testing.assert_allclose(mom[1], J * rho * U2, rtol=0, atol=1e-14 * np.abs(J).max())
    assert g.t == 0


@pytest.mark.parametrize("Q", [9, 21])
def test_steps_after_an_equilibrium_start_match_the_oracle(Q):
    """The moving wall reads rho and Ut^2 of the last collision: the start
    supplies (rho, U^2), which the oracle is given explicitly."""
    o, g = annulus_pair(Q, 0)
    U0 = 0.01 * (1.0 / 8) / math.sin(2.0 * math.pi / 40)
    o.set_case(0.8, 1.0, U0, 0.0)
    g.set_case(0.8, 1.0, U0, 0.0)
    # a j-invariant start: D2Q21 amplifies j-dependent modes on anisotropic
    # cells, which would make a long comparison measure that growth
    rho, U1, U2 = fields(o.n1, o.n2, 41)
    U1[...] = 0.0
    rho = np.repeat(rho[:, :1], o.n2, axis=1)
    U2 = np.repeat(U2[:, :1], o.n2, axis=1)
    g.set_equilibrium(rho, U1, U2)
    o.set_state(oracle_equilibrium(o, rho, U1, U2), rho, U2)
    o.step(60)
    g.step(60)
    so = o.state()
    assert np.sqrt(((g.state() - so) ** 2).sum() / (so ** 2).sum()) <= 1e-13


def test_device_fields_and_profiles_broadcast():
    c = _clbm()
    o, g = annulus_pair(21, 1)
    g.set_case(0.8)
    rho, U1, U2 = fields(o.n1, o.n2, 5)
    prof = U2[:, :1].copy()
    g.set_equilibrium(None, None, prof)              # (n1, 1) profile, host
    a = g.state()
    d = torch.tensor(prof, device=g.device)
    g.set_equilibrium(None, None, d)                 # the same on the device
    assert np.array_equal(g.state(), a)
    with pytest.raises(ValueError):
        g.set_equilibrium(torch.tensor(rho, device=g.device), U1, None)
    with pytest.raises(c.ClbmError):
        c.Grid(21, 8, 40, I.polar_edges(1.0, 2.0, 8), kind=c.POLAR).set_equilibrium(None, None, prof)


@pytest.mark.parametrize("prec,tol", [(1, 1e-6), (2, 1e-3), (3, 1e-2)])
def test_lower_precision_equilibrium_start(prec, tol):
    """Stored as deviations from the rest state in the grid's precision."""
    o, g64 = annulus_pair(21, 0)
    _, g = annulus_pair(21, prec)
    rho, U1, U2 = fields(o.n1, o.n2, 17)
    for x in (g64, g):
        x.set_case(0.8)
    rest = g64.state()
    for x in (g64, g):
        x.set_equilibrium(rho, U1, U2)
    a, b = g64.state(), g.state()
    assert np.abs(b - a).max() <= tol * np.abs(a - rest).max()


def test_exact_couette_start_is_closer_early_and_ends_in_the_same_state():
    """Circular Couette D2Q21 at N_r = 32: started from the equilibrium of
    the exact profile the velocity is far closer to the steady one after 1000
    steps than when started from rest, and both runs end in the same steady
    state (it is unique).  (The number of steps to a residual of 1e-10 is
    about the same either way: the last decade is set by the slow density
    oscillation, not by the velocity start.)"""
    c = _clbm()
    R1, R2, uw, tau, Nr = 1.0, 2.0, 0.01, 0.8, 32
    Nt = I.n_theta(Nr, R1, R2)
    e = I.polar_edges(R1, R2, Nr)
    dx = (R2 - R1) / Nr
    M = R1 / dx
    r_lat = 0.5 * (e[:-1] + e[1:]) / dx
    ex = E.Annulus.couette(M, M + Nr, uw / M).u(r_lat)
    Ut2 = ex / (math.sin(2.0 * math.pi / Nt) * r_lat)          # u_theta = Ut^2 |g_2|
    out = {}
    for start in ("rest", "exact"):
        g = c.Grid(21, Nr, Nt, e, kind=c.POLAR, precision="fp64", bc_lo=c.MOVING, bc_hi=c.NOSLIP)
        g.set_case(tau, 1.0, c.wall_speed_polar(uw, R1, Nt, dx), 0.0)
        if start == "exact":
            g.set_equilibrium(None, None, Ut2[:, None])
        g.step(1000)
        early = g.moments(names=("Ut2",))["Ut2"][:, 0]
        g.residual()
        steps, res = 1000, math.inf
        while steps < 200000 and res > 1e-10:
            g.step(500)
            steps += 500
            res, _ = g.residual()
        out[start] = (steps, early, g.moments(names=("Ut2",))["Ut2"][:, 0])
        g.close()
    final = out["rest"][2]
    gap = {k: np.abs(v[1] - final).max() / np.abs(final).max() for k, v in out.items()}
    for k in out:
        print("\nEQSTART circular Couette D2Q21 32x%d from %s: %d steps to residual 1e-10, "
              "distance to the steady profile after 1000 steps %.2e" % (Nt, k, out[k][0], gap[k]))
    assert gap["exact"] < gap["rest"] / 5.0
    assert np.abs(out["exact"][2] - final).max() <= 1e-5 * np.abs(final).max()
