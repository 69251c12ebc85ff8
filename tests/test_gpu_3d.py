"""The three-dimensional update (D3Q39, clbm3.h) on the GPU against the 3-D
FP64 oracle: state, moments and totals on channel and annulus grids, both
wall conditions, body force, ragged block tails, degenerate periodic sizes,
FP32; plus conservation and run-to-run identity."""
import math

import numpy as np
import pytest

import clbm_inputs as I
from oracle import oracle3d as O3

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _clbm():
    from paper_2301_01868_gb300 import clbm
    return clbm


class Case3:
    def __init__(self, n1, n2, n3, kind=0, edges=None, step2=1.0, step3=1.0, bc=(0, 0), tau=0.8,
                 U0=(0.0, 0.0), g=(0.0, 0.0, 0.0)):
        self.n1, self.n2, self.n3, self.kind = n1, n2, n3, kind
        self.edges = np.arange(n1 + 1.0) if edges is None else edges
        self.step2, self.step3, self.bc, self.tau, self.U0, self.g = step2, step3, bc, tau, U0, g

    def oracle(self):
        o = O3.Grid(self.n1, self.n2, self.n3, self.kind, edges=self.edges, step2=self.step2,
                    step3=self.step3, bc_lo=self.bc[0], bc_hi=self.bc[1])
        o.set_case(self.tau, 1.0, self.U0[0], self.U0[1], self.g)
        o.init_rest()
        return o

    def gpu(self, prec=0):
        c = _clbm()
        g = c.Grid3(self.n1, self.n2, self.n3, self.edges, kind=self.kind, step2=self.step2,
                    step3=self.step3, precision=prec, bc_lo=self.bc[0], bc_hi=self.bc[1])
        g.set_case(self.tau, 1.0, self.U0[0], self.U0[1], self.g)
        return g


def perturbed(o, seed, amp):
    st = o.state()
    Q, n1, n2, n3 = st.shape
    f = I.smooth_field((Q * n1, n2, n3), seed=seed, amplitude=amp).reshape(st.shape)
    return st * (1.0 + f)


def run_pair(case, steps, prec=0, seed=5, amp=2e-3):
    o = case.oracle()
    g = case.gpu(prec)
    if amp:
        st = perturbed(o, seed, amp)
        o.set_state(st)
        g.set_state(st)
    o.step(steps)
    g.step(steps)
    return o, g


def rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def stretched_channel(n1=10, n2=6, n3=5, **kw):
    e = I.geometric_stretch_edges(n1, 1.06, float(n1))
    dx = (e[-1] - e[0]) / n1
    return Case3(n1, n2, n3, 0, edges=e, step2=dx, step3=dx, **kw)


def test_fp64_channel_state_matches_oracle():
    """Stretched channel, moving low wall, body force along q^3, a start
    that depends on all three coordinates."""
    case = stretched_channel(bc=(1, 0), U0=(0.02, 0.0), g=(0.0, 1e-6, 2e-6))
    o, g = run_pair(case, 100)
    assert rel(g.state(), o.state()) <= 1e-13
    mo, mg = o.moments(), g.moments()
    assert np.abs(mg["rho"] - mo["rho"]).max() <= 1e-13
    assert rel(mg["Ut"], mo["Ut"]) <= 1e-11


def test_fp64_annulus_matches_oracle():
    e = I.polar_edges(1.0, 2.0, 8, 0.35)
    case = Case3(8, 50, 3, 1, edges=e, step3=0.15, bc=(1, 0), U0=(0.05, 0.0), g=(0.0, 0.0, 1e-6))
    o, g = run_pair(case, 100, amp=1e-3)
    assert rel(g.state(), o.state()) <= 1e-13
    mo, mg = o.moments(), g.moments()
    assert rel(mg["Ut"], mo["Ut"]) <= 1e-11


def test_fp64_no_slip_walls_ragged_blocks():
    """Rows of 13 x 11 = 143 cells: two blocks, the second ragged."""
    case = stretched_channel(n1=6, n2=13, n3=11, g=(0.0, 2e-6, 0.0))
    o, g = run_pair(case, 60, seed=9)
    assert rel(g.state(), o.state()) <= 1e-13


def test_fp64_degenerate_periodic_sizes():
    """n2 = n3 = 1: every neighbour along q^2 and q^3 is the cell itself."""
    case = Case3(8, 1, 1, 0, bc=(1, 0), U0=(0.03, 0.0), g=(0.0, 0.0, 1e-5))
    o, g = run_pair(case, 300, amp=0.0)
    assert rel(g.state(), o.state()) <= 1e-13


def test_fp32_channel_velocity_matches_oracle():
    case = stretched_channel(bc=(1, 0), U0=(0.02, 0.0), g=(0.0, 1e-6, 2e-6))
    o, g = run_pair(case, 200, prec=1)
    assert rel(g.moments()["Ut"], o.moments()["Ut"]) <= 1e-5


@pytest.mark.parametrize("prec,tol", [(2, 3e-3), (3, 3e-2)])
def test_16bit_storage_channel_velocity_near_oracle(prec, tol):
    """FP32 compute with FP16 / BF16 storage of the deviations."""
    case = stretched_channel(bc=(1, 0), U0=(0.02, 0.0), g=(0.0, 1e-6, 2e-6))
    o, g = run_pair(case, 200, prec=prec, amp=0.0)
    assert rel(g.moments()["Ut"], o.moments()["Ut"]) <= tol


def test_totals_conserve_mass_and_match_oracle():
    case = stretched_channel(bc=(0, 0), g=(0.0, 0.0, 0.0))
    o, g = run_pair(case, 0)
    t0 = g.totals()
    np.testing.assert_allclose(t0, o.totals(), rtol=1e-13, atol=1e-13)
    o.step(150)
    g.step(150)
    t1 = g.totals()
    assert abs(t1[0] - t0[0]) <= 1e-13 * abs(t0[0])
    np.testing.assert_allclose(t1, o.totals(), rtol=1e-12, atol=1e-12)


def test_two_runs_are_bitwise_identical():
    case = stretched_channel(n1=12, n2=20, n3=16, bc=(1, 0), U0=(0.02, 0.0))
    out = []
    for _ in range(2):
        o = case.oracle()
        g = case.gpu(1)
        g.set_state(perturbed(o, 3, 1e-3))
        g.step(50)
        out.append(g.state())
        g.close()
    assert np.array_equal(out[0], out[1])


def test_grid_rejects_bad_descriptions():
    c = _clbm()
    with pytest.raises(c.ClbmError):
        c.Grid3(3, 4, 4, np.arange(4.0))
    with pytest.raises(c.ClbmError):
        c.Grid3(6, 4, 4, np.array([0, 1, 2, 2, 3, 4, 5.0]))
    with pytest.raises(c.ClbmError):
        c.Grid3(6, 4, 4, np.arange(7.0), precision=4)
    g = c.Grid3(6, 4, 4, np.arange(7.0))
    with pytest.raises(c.ClbmError):
        g.step(1)                 # no case yet
    with pytest.raises(c.ClbmError):
        g.set_case(0.5)


def test_circular_couette_converges_in_three_dimensions():
    """The extruded annulus (1 <= r <= 2, N_theta = round(2 pi N_r), two axial
    nodes, tau = 0.8, inner wall at 0.01): the steady D3Q39 profile approaches
    the exact circular Couette profile (Eq. 27) as N_r grows, about halving
    its error per doubling as D2Q21 does in 2-D, and stays axially uniform."""
    from oracle import exact as E
    c = _clbm()
    R1, R2, uw, tau = 1.0, 2.0, 0.01, 0.8
    nu = (tau - 0.5) * 2.0 / 3.0
    errs = []
    for Nr in (16, 32, 64):
        Nt = I.n_theta(Nr, R1, R2)
        e = I.polar_edges(R1, R2, Nr)
        dx = (R2 - R1) / Nr
        g = c.Grid3(Nr, Nt, 2, e, kind=c.ANNULUS3, step3=dx, precision="fp64", bc_lo=c.MOVING,
                    bc_hi=c.NOSLIP)
        g.set_case(tau, 1.0, c.wall_speed_polar(uw, R1, Nt, dx), 0.0)
        g.step(int(20 * Nr * Nr / (math.pi ** 2 * nu)))
        ut = g.moments()["Ut"][1]
        assert np.abs(ut - ut[:, :1, :1]).max() <= 1e-12 * np.abs(ut).max()
        r_lat = 0.5 * (e[:-1] + e[1:]) / dx
        u = ut[:, 0, 0] * math.sin(2.0 * math.pi / Nt) * r_lat
        M = R1 / dx
        ex = E.Annulus.couette(M, M + Nr, uw / M).u(r_lat)
        errs.append(float(np.linalg.norm(u - ex) / np.linalg.norm(ex)))
        print("\nLADDER3D circular Couette D3Q39 fp64 %dx%dx2: L2 error vs exact %.3e" % (Nr, Nt, errs[-1]))
        g.close()
    assert errs[1] < errs[0] / 1.6 and errs[2] < errs[1] / 1.6
    assert errs[1] < 0.05


def test_3d_equilibrium_start_matches_oracle_feq():
    """J f^eq of given fields (Eq. 19) against the 3-D oracle's f^eq, cell by
    cell; then 40 steps from that start against the oracle (the walls read
    the start's moments)."""
    e = I.polar_edges(1.0, 2.0, 6, 0.35)
    case = Case3(6, 30, 3, 1, edges=e, step3=0.2, bc=(1, 0), U0=(0.04, 0.0))
    o = case.oracle()
    g = case.gpu(0)
    sh = (6, 30, 3)
    rho = 1.0 + I.smooth_field((6, 30, 3), seed=21, amplitude=0.02)
    U = I.smooth_field((18, 30, 3), seed=22, amplitude=0.01).reshape((3,) + sh)
    g.set_equilibrium(rho, U)
    N = g.state()
    ref = np.empty_like(N)
    for i in range(6):
        geo = o.row_geometry(i + 1)
        for j in range(30):
            for k in range(3):
                u = U[:, i, j, k]
                for a in range(39):
                    ref[a, i, j, k] = geo["J"] * o.feq(a, rho[i, j, k], u, u, geo["ginv"])
    assert np.abs(N - ref).max() <= 1e-14 * np.abs(ref).max()
    o.set_state(ref, rho, U[1], U[2])
    o.step(40)
    g.step(40)
    assert rel(g.state(), o.state()) <= 1e-13


@pytest.mark.parametrize("prec", [0, 1])
def test_3d_restore_continues_bit_for_bit(prec):
    case = stretched_channel(n1=8, n2=12, n3=10, bc=(1, 0), U0=(0.02, 0.0), g=(0.0, 1e-6, 1e-6))
    a = case.gpu(prec)
    a.step(30)
    blob = a.checkpoint()
    a.step(40)
    sa = a.state()
    c = _clbm()
    b = c.Grid3(case.n1, case.n2, case.n3, case.edges, kind=case.kind, step2=case.step2, step3=case.step3,
                precision=prec, bc_lo=1, bc_hi=0)
    b.restore(blob)
    assert b.t == 30
    b.step(40)
    assert np.array_equal(b.state(), sa)
    other = c.Grid3(case.n1, case.n2, case.n3 + 1, np.asarray(case.edges), kind=case.kind,
                    step2=case.step2, step3=case.step3, precision=prec)
    with pytest.raises(c.ClbmError):
        other.restore(blob)



# the two forms of the FP32-compute update: pulled pairs kept in registers
# (kernel 1) or in shared memory (kernel 2, more blocks per SM); the same
# arithmetic in the same order, so the same bits
def _gpu_kernel(case, prec, kernel):
    g = case.gpu(prec)
    g.set_kernel(kernel)
    return g


@pytest.mark.parametrize("kernel", [1, 2])
@pytest.mark.parametrize("n2,n3", [(13, 11), (1, 5), (7, 1)])
def test_fp32_kernels_ragged_and_degenerate_columns(kernel, n2, n3):
    """Ragged block tails, n2 = 1 (every q^2 neighbour is the cell itself),
    n3 = 1."""
    case = stretched_channel(n1=6, n2=n2, n3=n3, bc=(1, 0), U0=(0.02, 0.0), g=(0.0, 2e-6, 1e-6))
    o = case.oracle()
    g = _gpu_kernel(case, 1, kernel)
    st = perturbed(o, 9, 2e-3)
    o.set_state(st)
    g.set_state(st)
    o.step(60)
    g.step(60)
    rest = case.oracle().state()
    assert rel(g.state() - rest, o.state() - rest) <= 1e-5
    assert rel(g.moments()["Ut"], o.moments()["Ut"]) <= 1e-5


@pytest.mark.parametrize("prec,tol", [(2, 3e-3), (3, 3e-2)])
@pytest.mark.parametrize("kernel", [1, 2])
def test_16bit_storage_kernels_near_oracle(prec, tol, kernel):
    case = stretched_channel(n2=7, bc=(1, 0), U0=(0.02, 0.0), g=(0.0, 1e-6, 2e-6))
    o = case.oracle()
    g = _gpu_kernel(case, prec, kernel)
    o.step(200)
    g.step(200)
    assert rel(g.moments()["Ut"], o.moments()["Ut"]) <= tol


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_kernels_give_the_same_bits_and_fp64_keeps_registers(prec):
    """The contracted annulus (CR = 0.35, moving inner wall), a perturbed
    start, 80 steps (captured-graph replays included): both kernels write
    identical states."""
    e = I.polar_edges(1.0, 2.0, 8, 0.35)
    case = Case3(8, 50, 3, 1, edges=e, step3=0.15, bc=(1, 0), U0=(0.05, 0.0), g=(0.0, 0.0, 1e-6))
    st = perturbed(case.oracle(), 5, 1e-3)
    out = []
    for kernel in (1, 2):
        g = _gpu_kernel(case, prec, kernel)
        g.set_state(st)
        g.step(80)
        out.append(g.state())
        g.close()
    for o in out[1:]:
        assert np.array_equal(out[0], o)
    c = _clbm()
    g = case.gpu(0)
    g.set_kernel(1)
    with pytest.raises(c.ClbmError):
        g.set_kernel(2)
    g.close()
