"""Write ``steady_profiles.txt``: the FP64 oracle's circular Couette profile
on the annulus 1 <= r <= 2 (Sec. 3.3, Eq. 27) after a fixed number of steps
from rest, for D2Q21 and D2Q9, with the exact profile at the same radii.

The bench compares the CUDA library's profile after the same steps with
these values (its L2 velocity error against the oracle and against the exact
solution) without running the oracle itself.  This script calls only the
oracle (``oracle/``) and the seedless grid builders of ``clbm_inputs``;
rerun it after any change to the oracle's arithmetic:

    python tests/golden/make_steady_profiles.py
"""
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import clbm_inputs as I  # noqa: E402
from oracle import exact as E  # noqa: E402
from oracle import oracle as O  # noqa: E402

R1, R2, UW, NR, TAU, STEPS = 1.0, 2.0, 0.01, 32, 0.8, 6000
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "steady_profiles.txt")


def main():
    nt = I.n_theta(NR, R1, R2)
    edges = I.polar_edges(R1, R2, NR)
    dbar = (R2 - R1) / NR
    dth = 2.0 * math.pi / nt
    M = R1 / dbar
    r_lat = 0.5 * (edges[:-1] + edges[1:]) / dbar
    U0 = UW / (math.sin(dth) * M)
    exact = E.Annulus.couette(M, M + NR, UW / M).u(r_lat)
    lines = ["# FP64 oracle: circular Couette in the annulus 1 <= r <= 2 (Sec. 3.3),",
             "# uniform radial grid N_r = %d, N_theta = %d, tau = %g, inner wall at" % (NR, nt, TAU),
             "# u_theta = %g, outer wall at rest, %d steps from rest (N'(q,-1) = J f^eq" % (UW, STEPS),
             "# of rho0 = 1 at rest).  Columns: node radius in lattice units r / Delta_r,",
             "# exact u_theta of Eq. 27, oracle u_theta = Ut^2 |g_2| for D2Q21 and D2Q9.",
             "# Written by tests/golden/make_steady_profiles.py (calls only the oracle).",
             "NR %d" % NR, "NTHETA %d" % nt, "TAU %r" % TAU, "UWALL %r" % UW, "STEPS %d" % STEPS]
    prof = {}
    for Q in (21, 9):
        o = O.Grid(Q, NR, nt, O.POLAR, edges=edges, bc_lo=O.MOVING, bc_hi=O.NOSLIP)
        o.set_case(TAU, 1.0, U0, 0.0)
        o.init_rest()
        o.step(STEPS)
        prof[Q] = o.moments()["Ut2"][:, 0] * math.sin(dth) * r_lat
    lines.append("# r_lat exact d2q21 d2q9")
    for k in range(NR):
        lines.append("%.17g %.17g %.17g %.17g" % (r_lat[k], exact[k], prof[21][k], prof[9][k]))
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(OUT)


if __name__ == "__main__":
    main()
