"""The committed oracle profile the bench compares against
(tests/golden/steady_profiles.txt): its exact column is Eq. 27 at the node
radii, its oracle columns stay within the accuracy the paper reports for the
two lattices on curved cells (D2Q21 much closer to the exact profile than
D2Q9, Sec. 3.3)."""
import math

import numpy as np

import clbm_inputs as I
from conftest import golden
from oracle import exact as E


def load():
    hdr, rows = {}, []
    for ln in open(golden("steady_profiles.txt")):
        if ln.startswith("#") or not ln.strip():
            continue
        p = ln.split()
        if p[0].isalpha():
            hdr[p[0]] = float(p[1])
        else:
            rows.append([float(x) for x in p])
    return hdr, np.array(rows)


def test_exact_column_is_the_closed_form():
    hdr, rows = load()
    nr = int(hdr["NR"])
    assert int(hdr["NTHETA"]) == I.n_theta(nr, 1.0, 2.0)
    edges = I.polar_edges(1.0, 2.0, nr)
    dbar = 1.0 / nr
    r_lat = 0.5 * (edges[:-1] + edges[1:]) / dbar
    np.testing.assert_allclose(rows[:, 0], r_lat, rtol=1e-15)
    M = 1.0 / dbar
    ex = E.Annulus.couette(M, M + nr, hdr["UWALL"] / M).u(r_lat)
    np.testing.assert_allclose(rows[:, 1], ex, rtol=1e-14)
    # the inner wall moves at UWALL, the outer one rests: the profile falls across the gap
    assert rows[0, 1] < hdr["UWALL"] and rows[-1, 1] > 0 and (np.diff(rows[:, 1]) < 0).all()


def test_oracle_columns_match_the_reported_accuracy():
    _, rows = load()
    ex = rows[:, 1]
    e21 = np.linalg.norm(rows[:, 2] - ex) / np.linalg.norm(ex)
    e9 = np.linalg.norm(rows[:, 3] - ex) / np.linalg.norm(ex)
    assert 0.02 < e21 < 0.04
    assert e9 > 2.0 * e21
