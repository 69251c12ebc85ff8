"""Resolution ladders on the GPU, run to a steady state, against the exact
profiles of the paper's flows (Sec. 3):

* planar Poiseuille (Eqs. 24-25) on the geometrically stretched channel of
  the planar configuration, D2Q21, tau = 1, stretch 1.02^(64 / n1) per cell
  and g = 1e-6 (64 / n1)^2 (the same total stretch and peak speed on every
  rung), n1 x n2 = 64 x 16, 128 x 32, 256 x 64 (and 512 x 128 in FP64): FP64
  to a residual of 1e-10,
  FP32 for a fixed 20 decay times of the slowest mode (a residual threshold
  near FP32's floor would stop it early, with a start-up remnant that grows
  as n1^2);
* circular Couette (Eq. 27) in the annulus 1 <= r <= 2, uniform radial grid,
  N_theta = round(2 pi N_r), tau = 0.8, inner wall at 0.01, D2Q21 at
  N_r = 32, 64, 128, each to a residual of 1e-10; D2Q9 at 32 beside it, run
  6000 steps (6 of its diffusion times): its inner-wall radial mode keeps growing
  slowly, with the lag or with an implicit force pass, and ends the run
  unstable long before a residual of 1e-10.  The paper finds D2Q9 converging
  to something other than the exact profile and D2Q21 converging to it,
  slowly (Sec. 3, Sec. 4); here D2Q21 halves its error per doubling.

Run with -s to see the tables (lines starting LADDER).
"""
import math

import numpy as np
import pytest

import clbm_inputs as I
from oracle import exact as E

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _clbm():
    from paper_2301_01868_gb300 import clbm
    return clbm


def run_to_steady(g, tol, chunk, max_steps):
    g.residual()
    steps = 0
    res = math.inf
    while steps < max_steps:
        g.step(chunk)
        steps += chunk
        res, _ = g.residual()
        if res <= tol:
            break
    return steps, res


def l2rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


RUNGS = ((64, 16), (128, 32), (256, 64))
RUNGS_FP64 = RUNGS + ((512, 128),)


def poiseuille(c, n1, n2, tau, prec):
    e = I.geometric_stretch_edges(n1, 1.02 ** (64.0 / n1), float(n1))
    gacc = 1e-6 * (64.0 / n1) ** 2
    g = c.Grid(21, n1, n2, e, kind=c.PLANAR, step2=1.0, precision=prec)
    g.set_case(tau, 1.0, 0.0, 0.0, (0.0, gacc))
    return g, e, gacc


def poiseuille_exact(e, n1, gacc, nu):
    x = 0.5 * (e[:-1] + e[1:])
    return E.planar_poiseuille(x, float(n1), gacc, nu)


def test_planar_poiseuille_ladder_fp64_converges_at_second_order():
    c = _clbm()
    tau, T0 = 1.0, 2.0 / 3.0
    nu = E.nu_of_tau(tau, T0)
    errs = []
    for n1, n2 in RUNGS_FP64:
        g, e, gacc = poiseuille(c, n1, n2, tau, "fp64")
        steps, res = run_to_steady(g, 1e-10, 2000, 2000000)
        err = l2rel(g.moments(names=("Ut2",))["Ut2"][:, 0], poiseuille_exact(e, n1, gacc, nu))
        errs.append(err)
        print("\nLADDER planar Poiseuille D2Q21 fp64 %dx%d stretch %.4f: %d steps, residual %.1e, "
              "L2 error vs exact %.3e" % (n1, n2, 1.02 ** (64.0 / n1), steps, res, err))
        g.close()
        assert res <= 1e-10
    # ratios 3.37, 3.27, 2.90: close to second order, easing at 512 as the
    # error nears the walls' share
    assert all(errs[k + 1] < errs[k] / 2.5 for k in range(3))


def test_planar_poiseuille_fp32_reaches_its_rounding_floor():
    """FP32 runs 20 decay times of the slowest mode (n1^2 / (pi^2 nu)) per
    rung.  At 64 x 16 it matches FP64's discretisation error; on the finer
    rungs the per-step body force (g = 6e-8 at n1 = 256) sits a few FP32
    roundings above the stored deviations' resolution and the error settles
    at a floor of a few 1e-4 instead of falling further."""
    c = _clbm()
    tau, T0 = 1.0, 2.0 / 3.0
    nu = E.nu_of_tau(tau, T0)
    errs = []
    for n1, n2 in RUNGS:
        g, e, gacc = poiseuille(c, n1, n2, tau, "fp32")
        steps = int(math.ceil(20.0 * n1 * n1 / (math.pi ** 2 * nu) / 1000.0)) * 1000
        g.step(steps - 1000)
        g.residual()
        g.step(1000)
        res, _ = g.residual()             # mean change per step over the last 1000
        err = l2rel(g.moments(names=("Ut2",))["Ut2"][:, 0], poiseuille_exact(e, n1, gacc, nu))
        errs.append(err)
        print("\nLADDER planar Poiseuille D2Q21 fp32 %dx%d stretch %.4f: %d steps, residual %.1e, "
              "L2 error vs exact %.3e" % (n1, n2, 1.02 ** (64.0 / n1), steps, res, err))
        g.close()
        assert res <= 1e-7              # FP32's floor of the per-step change
    assert errs[0] < 1e-3
    assert max(errs) < 1e-3


def test_circular_couette_ladder_d2q21_converges_and_beats_d2q9():
    c = _clbm()
    R1, R2, uw, tau = 1.0, 2.0, 0.01, 0.8
    errs = {}
    for Q, rungs in ((21, (32, 64, 128)), (9, (32,))):
        for Nr in rungs:
            Nt = I.n_theta(Nr, R1, R2)
            e = I.polar_edges(R1, R2, Nr)
            dx = (R2 - R1) / Nr
            M = R1 / dx
            g = c.Grid(Q, Nr, Nt, e, kind=c.POLAR, precision="fp64", bc_lo=c.MOVING, bc_hi=c.NOSLIP)
            g.set_case(tau, 1.0, c.wall_speed_polar(uw, R1, Nt, dx), 0.0)
            if Q == 21:
                steps, res = run_to_steady(g, 1e-10, 1000, 400000)
            else:
                # D2Q9's inner-wall radial mode outgrows the flow before a tight
                # residual; 6000 steps are 6 diffusion times, before it shows
                steps = 6000
                g.residual()
                g.step(steps - 1000)
                g.residual()
                g.step(1000)
                res, _ = g.residual()
            r_lat = 0.5 * (e[:-1] + e[1:]) / dx
            u = g.moments(names=("Ut2",))["Ut2"][:, 0] * math.sin(2.0 * math.pi / Nt) * r_lat
            ex = E.Annulus.couette(M, M + Nr, uw / M).u(r_lat)
            errs[(Q, Nr)] = l2rel(u, ex)
            print("\nLADDER circular Couette D2Q%d fp64 %dx%d: %d steps, residual %.1e, "
                  "L2 error vs exact %.3e" % (Q, Nr, Nt, steps, res, errs[(Q, Nr)]))
            g.close()
    assert errs[(21, 64)] < errs[(21, 32)] / 1.6 and errs[(21, 128)] < errs[(21, 64)] / 1.6
    assert errs[(21, 32)] < errs[(9, 32)] / 2.0


def test_precision_ladder_on_the_contracted_annulus_at_128():
    """Circular Couette on the bench's radial grid (App. C contraction
    CR = 0.35) at N_r = 128, N_theta = 804, tau = 0.8, 14 diffusion times from
    rest: every storage precision against FP64 and against Eq. 27."""
    c = _clbm()
    R1, R2, uw, tau, Nr = 1.0, 2.0, 0.01, 0.8, 128
    Nt = I.n_theta(Nr, R1, R2)
    e = I.polar_edges(R1, R2, Nr, 0.35)
    dx = (R2 - R1) / Nr
    M = R1 / dx
    nu = (tau - 0.5) * 2.0 / 3.0
    steps = int(math.ceil(14 * Nr * Nr / (math.pi ** 2 * nu) / 1000.0)) * 1000
    r_lat = 0.5 * (e[:-1] + e[1:]) / dx
    ex = E.Annulus.couette(M, M + Nr, uw / M).u(r_lat)
    u = {}
    for prec in ("fp64", "fp32", "fp16", "bf16"):
        g = c.Grid(21, Nr, Nt, e, kind=c.POLAR, precision=prec, bc_lo=c.MOVING, bc_hi=c.NOSLIP)
        g.set_case(tau, 1.0, c.wall_speed_polar(uw, R1, Nt, dx), 0.0)
        g.step(steps)
        u[prec] = g.moments(names=("Ut2",))["Ut2"][:, 0] * math.sin(2.0 * math.pi / Nt) * r_lat
        g.close()
    for prec in u:
        print("\nLADDER precision D2Q21 %s 128x804 CR 0.35 (%d steps): vs FP64 %.2e, vs exact %.3e"
              % (prec, steps, l2rel(u[prec], u["fp64"]), l2rel(u[prec], ex)))
    assert l2rel(u["fp64"], ex) < 0.02
    assert l2rel(u["fp32"], u["fp64"]) < 1e-4
    assert l2rel(u["fp16"], u["fp64"]) < 2e-2
    assert l2rel(u["bf16"], u["fp64"]) < 2e-1           # 8 mantissa bits: 1.2e-1



def test_circular_poiseuille_ladder_d2q21_converges():
    """The fourth flow of Sec. 3: the annulus 1 <= r <= 2 with both walls at
    rest, driven by a constant contravariant azimuthal force g^2 (the
    physical acceleration g^2 r sin(dtheta) grows with r; R10, R5), peak
    speed about 0.01, tau = 0.8, uniform radial grids.  D2Q21 approaches
    the exact profile (A/8)(r^2 - R1^2)(R2^2 - r^2)/r at second order as N_r
    grows (the no-slip walls are second order; circular Couette's first order
    comes from its moving wall); D2Q9 at N_r = 32 (6000 steps) is 40 % off."""
    c = _clbm()
    R1, R2, tau, target = 1.0, 2.0, 0.8, 0.01
    errs = {}
    for Q, rungs in ((21, (32, 64, 128)), (9, (32,))):
        T0 = 2.0 / 3.0 if Q == 21 else 1.0 / 3.0
        nu = T0 * (tau - 0.5)
        for Nr in rungs:
            Nt = I.n_theta(Nr, R1, R2)
            e = I.polar_edges(R1, R2, Nr)
            dx = (R2 - R1) / Nr
            M = R1 / dx
            alpha = math.sin(2.0 * math.pi / Nt)
            r_lat = 0.5 * (e[:-1] + e[1:]) / dx
            peak = np.abs(E.Annulus.poiseuille(M, M + Nr, 1.0).u(np.linspace(M, M + Nr, 2001))).max()
            g2 = nu * target / (alpha * peak)          # A = alpha g2 / nu gives the peak
            ex = E.Annulus.poiseuille(M, M + Nr, alpha * g2 / nu).u(r_lat)
            g = c.Grid(Q, Nr, Nt, e, kind=c.POLAR, precision="fp64", bc_lo=c.NOSLIP, bc_hi=c.NOSLIP)
            g.set_case(tau, 1.0, 0.0, 0.0, (0.0, g2))
            if Q == 21:
                steps, res = run_to_steady(g, 1e-10, 1000, 400000)
            else:
                steps = 6000
                g.step(steps)
                res = float("nan")
            u = g.moments(names=("Ut2",))["Ut2"][:, 0] * alpha * r_lat
            errs[(Q, Nr)] = l2rel(u, ex)
            print("\nLADDER circular Poiseuille D2Q%d fp64 %dx%d: %d steps, residual %.1e, "
                  "L2 error vs exact %.3e" % (Q, Nr, Nt, steps, res, errs[(Q, Nr)]))
            g.close()
    # measured 2.33e-3 / 6.36e-4 / 1.67e-4 (second order), D2Q9 4.0e-1
    assert errs[(21, 64)] < errs[(21, 32)] / 3.0 and errs[(21, 128)] < errs[(21, 64)] / 3.0
    assert errs[(21, 32)] < errs[(9, 32)] / 10.0
