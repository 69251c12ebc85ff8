"""Failure detection on the GPU without a fault: the bounded wait that every
spin of the pipelined kernels goes through gives up on a barrier nothing
completes, reports CLBM_ETIMEOUT, and leaves the context usable; a lattice
driven unstable is reported (CLBM_EUNSTABLE) and can be restarted."""
import math

import numpy as np
import pytest

import clbm_inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _clbm():
    from paper_2301_01868_gb300 import clbm
    return clbm


def small_annulus(c, prec=1):
    n1, n2 = 32, 201
    e = I.polar_edges(1.0, 2.0, n1)
    g = c.Grid(21, n1, n2, e, kind=c.POLAR, precision=prec, bc_lo=c.MOVING, bc_hi=c.NOSLIP)
    g.set_case(0.8, 1.0, c.wall_speed_polar(0.01, 1.0, n2, 1.0 / n1), 0.0)
    return g


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    c = _clbm()
    st, ms_small = c.selftest_bounded_wait(1 << 12)
    assert st == 5, c.lib().clbm_last_error()           # CLBM_ETIMEOUT
    st, ms_large = c.selftest_bounded_wait(1 << 16)
    assert st == 5
    # the update's waits poll 2^18 times: their time-out, from the measured
    # rate, should be about a second
    full_s = ms_large / (1 << 16) * (1 << 18) / 1e3
    print("\nBOUNDED_WAIT %.3f ms for 2^12 polls, %.3f ms for 2^16: 2^18 polls ~ %.2f s"
          % (ms_small, ms_large, full_s))
    assert 0.01 < full_s < 5.0
    g = small_annulus(c)
    g.step(20)
    res, cons = g.residual()
    g.step(20)
    res, cons = g.residual()
    assert math.isfinite(res) and cons[0] > 0
    g.close()


def test_unstable_lattice_is_reported_and_restarts():
    c = _clbm()
    g = small_annulus(c, prec=0)
    st = g.state()
    st[:, 5, 7] = np.nan
    g.set_state(st)
    g.step(2)
    with pytest.raises(c.UnstableError):
        g.residual()
    g.set_case(0.8, 1.0, 0.0, 0.0)           # a new case restarts from rest
    g.step(10)
    res, cons = g.residual()
    assert np.isfinite(cons).all()
    g.close()


def test_selftest_rejects_bad_poll_counts():
    c = _clbm()
    assert c.selftest_bounded_wait(0)[0] == 1
    assert c.selftest_bounded_wait((1 << 22) + 1)[0] == 1
