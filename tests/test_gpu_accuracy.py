"""Precision ladder at steady state: circular Couette flow (Sec. 3.3) in the
annulus 1 <= r <= 2, uniform radial grid N_r = 32, N_theta = 201 (near-square
cells at the inner wall), tau = 0.8, inner wall at u_theta = 0.01, outer wall
at rest, 6000 steps from rest (about 11 diffusion times N_r^2 / (pi^2 nu)).

Every precision reports its L2 velocity error against the FP64 oracle after
the same steps and against the exact profile u = a r + b / r (Eq. 27) at the
node radii; D2Q21 and D2Q9 side by side.  Run with -s to see the table.
"""
import math

import numpy as np
import pytest

import clbm_inputs as I
from oracle import exact as E
from oracle import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

R1, R2, UW, NR, TAU, STEPS = 1.0, 2.0, 0.01, 32, 0.8, 6000
NT = I.n_theta(NR, R1, R2)
DBAR = (R2 - R1) / NR
DTH = 2.0 * math.pi / NT
M = R1 / DBAR
EDGES = I.polar_edges(R1, R2, NR)
R_LAT = 0.5 * (EDGES[:-1] + EDGES[1:]) / DBAR      # node radii in lattice units
U0 = UW / (math.sin(DTH) * M)                        # contravariant wall speed
EXACT = E.Annulus.couette(M, M + NR, UW / M).u(R_LAT)

_oracle_cache = {}


def u_theta(ut2):
    """Physical azimuthal velocity of the j-invariant profile: Ut^2 |g_2|."""
    return np.asarray(ut2)[:, 0] * math.sin(DTH) * R_LAT


def oracle_profile(Q):
    if Q not in _oracle_cache:
        o = O.Grid(Q, NR, NT, O.POLAR, edges=EDGES, bc_lo=O.MOVING, bc_hi=O.NOSLIP)
        o.set_case(TAU, 1.0, U0, 0.0)
        o.init_rest()
        o.step(STEPS)
        _oracle_cache[Q] = u_theta(o.moments()["Ut2"])
    return _oracle_cache[Q]


def l2rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# FP16: six units of its roundoff (6 x 2^-11): the stored deviations are
# rounded every step and which way each goes depends on the FP32 arithmetic
# order (the one- and two-cells-per-thread kernels measure 1.7e-3 and 2.0e-3)
LADDER = [(21, "fp64", 1e-12, 0.04), (21, "fp32", 1e-5, 0.04), (21, "fp16", 3e-3, 0.04),
          (21, "bf16", 5e-2, 0.1), (9, "fp64", 1e-12, 0.15), (9, "fp32", 1e-5, 0.15)]


@pytest.mark.parametrize("Q,prec,tol_oracle,tol_exact", LADDER)
def test_precision_ladder_circular_couette(Q, prec, tol_oracle, tol_exact):
    from paper_2301_01868_gb300 import clbm
    g = clbm.Grid(Q, NR, NT, EDGES, kind=clbm.POLAR, precision=prec, bc_lo=clbm.MOVING,
                  bc_hi=clbm.NOSLIP)
    g.set_case(TAU, 1.0, U0, 0.0)
    g.step(STEPS)
    u = u_theta(g.moments(names=("Ut2",))["Ut2"])
    g.close()
    e_orc = l2rel(u, oracle_profile(Q))
    e_ex = l2rel(u, EXACT)
    e_orc_ex = l2rel(oracle_profile(Q), EXACT)
    print("\nACCURACY D2Q%d %s N_r=%d N_theta=%d tau=%g steps=%d: L2 vs oracle %.3e, "
          "vs exact %.4e (oracle vs exact %.4e)" % (Q, prec, NR, NT, TAU, STEPS, e_orc, e_ex, e_orc_ex))
    assert e_orc <= tol_oracle
    assert e_ex <= tol_exact


def test_d2q21_closer_to_exact_than_d2q9_on_curved_cells():
    """The paper's argument for D2Q21 on curved grids (Sec. 3.3)."""
    assert l2rel(oracle_profile(21), EXACT) < 0.5 * l2rel(oracle_profile(9), EXACT)
