"""The batched record's lattice selection (host logic of bench.py, no GPU):
the seeded configuration is reproducible, its first n lattices are a prefix
of the 512, and the "smallest" selection holds the n smallest of the 512 by
cell count, the circular lattices with n1 = round(n2 / 2 pi)."""
import math
import sys

import pytest

from conftest import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _key(r):
    return (r.case, r.n1, r.n2, r.tau)


def test_first_n_is_a_prefix_of_the_configuration():
    full = bench.batch_requests(512)
    assert [_key(r) for r in bench.batch_selection(40)] == [_key(r) for r in full[:40]]
    assert [_key(r) for r in bench.batch_requests(512)] == [_key(r) for r in full]


def test_smallest_selection_holds_the_smallest_lattices():
    full = bench.batch_requests(512)
    small = bench.batch_selection(150, "smallest")
    assert len(small) == 150
    cut = max(r.n1 * r.n2 for r in small)
    assert sum(r.n1 * r.n2 < cut for r in full) <= 150
    assert all(r.n1 * r.n2 <= cut for r in small)
    assert len({r.rid for r in small}) == 150


def test_shapes_follow_the_configuration():
    for r in bench.batch_requests(512):
        assert r.lattice == 21 and 0.55 <= r.tau <= 1.0
        if r.case.startswith("circular"):
            assert r.n1 == max(8, int(round(r.n2 / (2.0 * math.pi))))
        else:
            assert 32 <= r.n1 <= 1024 and 32 <= r.n2 <= 2048


def test_unknown_selection_is_refused():
    with pytest.raises(ValueError):
        bench.batch_selection(10, "largest")
