"""Asynchronous host copies (clbm_upload_state_async / clbm_set_uploaded_state
/ clbm_download_moments_async / clbm_wait_copies): a pipelined sequence of
starts and results gives, bit for bit, what the synchronous calls give, with
two uploads in flight and downloads overlapping the next update."""
import math

import numpy as np
import pytest

import clbm_inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _grid(prec):
    from paper_2301_01868_gb300 import clbm
    n1, n2 = 24, 150
    e = I.polar_edges(1.0, 2.0, n1, 0.35)
    st = torch.cuda.Stream()
    g = clbm.Grid(21, n1, n2, e, kind=clbm.POLAR, precision=prec, bc_lo=clbm.MOVING, bc_hi=clbm.NOSLIP,
                  stream=st)
    g.set_case(0.8, 1.0, clbm.wall_speed_polar(0.02, 1.0, n2, 1.0 / n1), 0.0)
    return g


def _pinned(shape):
    return torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()


@pytest.mark.parametrize("prec", [0, 1])
def test_pipelined_copies_equal_synchronous_calls(prec):
    a, b = _grid(prec), _grid(prec)
    rest = a.state()
    starts = []
    for k in range(4):
        s = _pinned(rest.shape)
        s[...] = rest * (1.0 + I.smooth_field(rest.shape, seed=40 + k, amplitude=1e-3))
        starts.append(s)
    # synchronous reference
    ref = []
    for s in starts:
        a.set_state(s)
        a.step(25)
        ref.append(a.moments(names=("rho", "Ut1", "Ut2")))
    # pipelined: upload k + 1 while k computes, download k while k + 1 computes
    outs = [{k: _pinned((b.n1, b.n2)) for k in ("rho", "Ut1", "Ut2")} for _ in starts]
    b.upload_state_async(starts[0])
    b.upload_state_async(starts[1])
    for k in range(len(starts)):
        b.set_uploaded_state()
        if k + 2 < len(starts):
            b.upload_state_async(starts[k + 2])
        b.step(25)
        b.download_moments_async(outs[k])
    b.wait_copies()
    for r, o in zip(ref, outs):
        for key in ("rho", "Ut1", "Ut2"):
            assert np.array_equal(r[key], o[key]), key
    a.close()
    b.close()


def test_upload_queue_limits():
    from paper_2301_01868_gb300 import clbm
    g = _grid(1)
    with pytest.raises(clbm.ClbmError):
        g.set_uploaded_state()          # nothing uploaded
    s = _pinned((g.Q, g.n1, g.n2))
    s[...] = g.state()
    g.upload_state_async(s)
    g.upload_state_async(s)
    with pytest.raises(clbm.ClbmError):
        g.upload_state_async(s)         # two wait already
    g.set_uploaded_state()
    g.set_uploaded_state()
    g.step(3)
    res, cons = g.residual()
    assert math.isinf(res) and cons[0] > 0
    g.wait_copies()
    g.close()
