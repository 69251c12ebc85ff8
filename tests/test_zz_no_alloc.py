"""The allocation-free totals entry point (clbm_totals_noalloc), called through
the C ABI, agrees with the conservation sums of clbm_residual.

clbm_totals_noalloc is for callers that cannot allocate device memory (code
running during CUDA graph capture, processes confined to a fixed memory
budget): it keeps its reduction scratch in a static device array.  This file
is collected last so that a failure here never hides another test's result.
"""
import ctypes

import numpy as np
import pytest

import clbm_inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_totals_without_allocation_match_residual_twice():
    from paper_2301_01868_gb300 import clbm

    lib = clbm.lib()
    f = lib.clbm_totals_noalloc
    f.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_int, ctypes.c_void_p]
    f.restype = ctypes.c_int

    n1, n2 = 24, 100
    e = I.polar_edges(1.0, 2.0, n1, 0.35)
    g = clbm.Grid(21, n1, n2, e, kind=clbm.POLAR, precision=clbm.FP64, bc_lo=clbm.MOVING,
                  bc_hi=clbm.NOSLIP)
    g.set_case(0.8, 1.0, clbm.wall_speed_polar(0.01, 1.0, n2, 1.0 / n1), 0.0)
    g.step(40)
    for _ in range(2):
        _, cons = g.residual()                       # the existing entry point
        Np = g.state(device=True)                    # caller-owned device input
        out = np.zeros(3)
        rc = f(21, Np.data_ptr(), n1, n2, out.ctypes.data, 0, g.stream.cuda_stream)
        assert rc == 0, lib.clbm_last_error().decode()
        mass = cons[0]
        assert abs(out[0] - mass) <= 1e-12 * abs(mass)
        assert abs(out[1] - cons[1]) <= 1e-12 * abs(mass)
        assert abs(out[2] - cons[2]) <= 1e-12 * abs(mass)
        # result written to device memory as well
        dev_out = torch.zeros(3, dtype=torch.float64, device=g.device)
        rc = f(21, Np.data_ptr(), n1, n2, dev_out.data_ptr(), 1, g.stream.cuda_stream)
        assert rc == 0
        g.stream.synchronize()
        np.testing.assert_array_equal(dev_out.cpu().numpy(), out)
        g.step(25)
    g.close()


def test_totals_without_allocation_rejects_oversized_grids():
    from paper_2301_01868_gb300 import clbm

    lib = clbm.lib()
    f = lib.clbm_totals_noalloc
    f.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_int, ctypes.c_void_p]
    f.restype = ctypes.c_int
    out = np.zeros(3)
    rc = f(21, ctypes.c_void_p(16), 4096, 4096, out.ctypes.data, 0, None)
    assert rc == 1  # CLBM_EINVAL, before any device access
    assert "scratch limit" in lib.clbm_last_error().decode()
