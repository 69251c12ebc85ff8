"""Pins of the oracle's lattice tables against App. A and App. B.

The printed D2Q21 weights of the two outer shells (7/432, 7/1620) break the
normalisation of App. A; the oracle uses 1/432 and 1/1620 (reading R1), which
satisfy every isotropy condition of App. A exactly.  The velocity order is
inferred from the App. B index maps (reading R2)."""
from fractions import Fraction

import numpy as np
import pytest

from conftest import golden
from oracle import oracle as O


def _sections(path):
    out, cur = {}, None
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("["):
            cur = line.strip("[]")
            out[cur] = []
        else:
            out[cur].append(line.split())
    return out


TABLES = _sections(golden("lattice_tables.txt"))


def _moment(w, c, p, q):
    return sum(wa * Fraction(int(ca[0])) ** p * Fraction(int(ca[1])) ** q for wa, ca in zip(w, c))


def _frac_weights(Q):
    c, w, _, _, T0 = O.lattice(Q)
    fw = [Fraction(x).limit_denominator(100000) for x in w]
    for x, f in zip(w, fw):
        assert abs(float(f) - x) < 1e-16
    return c, fw, Fraction(T0).limit_denominator(100)


def test_printed_d2q21_weights_are_not_normalised():
    w = [Fraction(r[1]) for r in TABLES["D2Q21 weights as printed"]]
    c, _, _ = _frac_weights(21)
    assert sum(w) == Fraction(289, 270)
    assert _moment(w, c, 2, 0) != Fraction(2, 3)


def test_oracle_d2q21_weights_match_print_except_outer_shells():
    printed = [Fraction(r[1]) for r in TABLES["D2Q21 weights as printed"]]
    _, fw, _ = _frac_weights(21)
    for a in range(21):
        if 13 <= a <= 20:
            assert fw[a] == printed[a] / 7
        else:
            assert fw[a] == printed[a]


def test_d2q9_weights_match_print():
    printed = [Fraction(r[1]) for r in TABLES["D2Q9 weights"]]
    _, fw, T0 = _frac_weights(9)
    assert fw == printed and T0 == Fraction(1, 3)


@pytest.mark.parametrize("Q", [9, 21])
def test_isotropy_app_a(Q):
    c, w, T0 = _frac_weights(Q)
    assert sum(w) == 1
    # odd moments vanish
    for p in range(0, 6):
        for q in range(0, 6 - p):
            if (p + q) % 2 == 1:
                assert _moment(w, c, p, q) == 0
    assert _moment(w, c, 2, 0) == T0 and _moment(w, c, 1, 1) == 0
    assert _moment(w, c, 4, 0) == 3 * T0 ** 2 and _moment(w, c, 2, 2) == T0 ** 2
    six = (_moment(w, c, 6, 0) == 15 * T0 ** 3 and _moment(w, c, 4, 2) == 3 * T0 ** 3
           and _moment(w, c, 2, 4) == 3 * T0 ** 3)
    # App. A: only D2Q21 is isotropic to 6th order
    assert six == (Q == 21)


def test_velocity_order_against_index_maps():
    c, _, star, hat, _ = O.lattice(21)
    bb = {int(a): int(b) for a, b in TABLES["bounce-back"]}
    sp = {int(a): int(b) for a, b in TABLES["specular"]}
    assert bb == {a: int(star[a]) for a in bb}
    assert sp == {a: int(hat[a]) for a in sp}
    for a, b in bb.items():
        assert tuple(c[b]) == (-c[a][0], -c[a][1])
    for a, b in sp.items():
        assert tuple(c[b]) == (-c[a][0], c[a][1])
    excluded = sorted(int(x) for x in TABLES[
        "directions with no wall-normal component, excluded from the wall maps"][0])
    assert excluded == [a for a in range(21) if c[a][0] == 0]
    # the maps cover exactly the wall-crossing directions
    assert sorted(bb) == [a for a in range(21) if c[a][0] != 0]


def test_d2q9_is_prefix_of_d2q21():
    c9, _, s9, h9, _ = O.lattice(9)
    c21, _, s21, h21, _ = O.lattice(21)
    assert np.array_equal(c9, c21[:9])
    assert np.array_equal(s9, s21[:9]) and np.array_equal(h9, h21[:9])
    assert len({tuple(x) for x in c21}) == 21
