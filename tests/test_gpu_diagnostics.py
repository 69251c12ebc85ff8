"""Parity of the convergence and conservation diagnostics (Sec. 3.1: the
steady state is judged by the kinetic energy and angular momentum no longer
changing, with the mass conserved) against the oracle's.

clbm_residual gives res = ||u(t) - u(t')||_J / ((t - t') ||u(t)||_J) and
cons = mass, momentum (2), kinetic energy, angular momentum, max |u|; the
oracle computes the same from its own moments (orc_flow_diagnostics,
orc_totals) on the same seeded inputs.  Every kernel that forms them is
covered: the per-cell k_residual (FP64; FP32 when the per-cell update is
chosen; iterated force; general grids), the pipelined k_residual_ws (FP32,
FP16 and BF16 storage, D2Q21 and D2Q9, polar and planar), the batched
reduction (every tile variant), and the full 1024 x 4096 bench grid.

Tolerances (relative): FP64 1e-12; FP32 1e-5 for the velocity-linear
quantities (angular momentum, max |u|, residual) and 2e-5 for the kinetic
energy (quadratic in u, so twice the velocity's relative error); 16-bit
storage six units of the storage type's roundoff (FP16 6 x 2^-11 = 3e-3,
BF16 5e-2), doubled for the kinetic energy: the stored deviations are
rounded every step, and which way each rounding goes depends on the FP32
arithmetic order, so kernels equal to FP32 rounding (one and two cells per
thread) give FP16 errors of 1.7e-3 and 2.0e-3 on the same run.  Mass is compared at 1e-12 (FP64) / 1e-6
(FP32 sums of rounded deviations: the rest part is exact, the deviations
carry the storage rounding).  Momentum, which vanishes at rest, is compared
absolutely, relative to the mass.
"""
import math

import numpy as np
import pytest

import clbm_inputs as I
from conftest import storage_rounded
from oracle import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _clbm():
    from paper_2301_01868_gb300 import clbm
    return clbm


PREC = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3}
# (velocity-linear, kinetic energy, mass) tolerances per precision
TOL = {"fp64": (1e-12, 1e-12, 1e-12), "fp32": (1e-5, 2e-5, 1e-6),
       "fp16": (3e-3, 6e-3, 1e-4), "bf16": (5e-2, 1e-1, 1e-3)}


class Setup:
    """A grid described once, built on both sides."""

    def __init__(self, Q, n1, n2, kind, edges=None, step2=1.0, nodes=None, dx=0.0, bc=(0, 0),
                 tau=0.8, U0=(0.0, 0.0), g=(0.0, 0.0), iters=0):
        self.__dict__.update(locals())
        del self.__dict__["self"]

    def oracle(self):
        o = O.Grid(self.Q, self.n1, self.n2, self.kind, edges=self.edges, step2=self.step2,
                   nodes=self.nodes, dx=self.dx, bc_lo=self.bc[0], bc_hi=self.bc[1])
        o.set_case(self.tau, 1.0, self.U0[0], self.U0[1], self.g)
        o.set_force_iterations(self.iters)
        o.init_rest()
        return o

    def gpu(self, prec, kernel=0):
        c = _clbm()
        g = c.Grid(self.Q, self.n1, self.n2, self.edges, kind=self.kind, step2=self.step2,
                   nodes=self.nodes, dx=self.dx, precision=PREC[prec], bc_lo=self.bc[0],
                   bc_hi=self.bc[1])
        g.set_case(self.tau, 1.0, self.U0[0], self.U0[1], self.g, self.iters)
        if kernel:
            g.set_kernel(kernel)
        return g


def polar(Q, n1=24, n2=100, CR=0.35, uw=0.02, **kw):
    R1, R2 = 1.0, 2.0
    U0 = _clbm().wall_speed_polar(uw, R1, n2, (R2 - R1) / n1)
    return Setup(Q, n1, n2, O.POLAR, edges=I.polar_edges(R1, R2, n1, CR), bc=(1, 0),
                 U0=(U0, 0.0), **kw)


def stretched(Q, n1=37, n2=45, tau=0.6, umax=0.05):
    e = I.geometric_stretch_edges(n1, 1.02 ** (64.0 / n1), float(n1))
    nu = (1 / 3 if Q == 9 else 2 / 3) * (tau - 0.5)
    return Setup(Q, n1, n2, O.PLANAR, edges=e, bc=(0, 1), tau=tau, U0=(0.0, 0.004),
                 g=(0.0, 8 * nu * umax / n1 ** 2))


def wavy(Q, n1=14, n2=22):
    P = I.mapped_nodes(I.wavy_channel(n1, n2, amp=0.15), n1, n2, "extend")
    return Setup(Q, n1, n2, O.GENERAL, nodes=P, dx=1.0, g=(0.0, 1e-5))


def check(cons, res, d, prec, what):
    tl, tk, tm = TOL[prec]
    mass = d["totals"][0]
    assert abs(cons[0] - mass) <= tm * abs(mass), (what, "mass", cons[0], mass)
    for k in (1, 2):
        assert abs(cons[k] - d["totals"][k]) <= tm * abs(mass), (what, "momentum", k)
    assert cons[3] == pytest.approx(d["ke"], rel=tk), (what, "kinetic energy")
    assert cons[4] == pytest.approx(d["am"], rel=tl, abs=1e-300), (what, "angular momentum")
    assert cons[5] == pytest.approx(d["umax"], rel=tl), (what, "max |u|")
    if math.isinf(d["res"]):
        assert math.isinf(res), what
    else:
        assert res == pytest.approx(d["res"], rel=tl), (what, "residual", res, d["res"])


def run_and_compare(setup, prec, kernel=0, t1=60, dt=90, perturb=0.0, seed=3):
    """Both sides from the same start: t1 steps, a residual call (the
    snapshot), dt more steps, a second call; each call's diagnostics against
    the oracle's of the same state."""
    o = setup.oracle()
    g = setup.gpu(prec, kernel)
    if perturb:
        rest = o.state()
        st = rest * (1.0 + I.smooth_field(rest.shape, seed=seed, amplitude=perturb))
        g.set_state(st)
        o.set_state(storage_rounded(rest, st, prec))
    o.step(t1)
    g.step(t1)
    r0, c0 = g.residual()
    d0 = o.diagnostics()
    check(c0, r0, d0, prec, "first call")
    o.step(dt)
    g.step(dt)
    r1, c1 = g.residual()
    d1 = o.diagnostics((d0["Ut1"], d0["Ut2"]), dt)
    check(c1, r1, d1, prec, "second call")
    assert math.isfinite(r1) and r1 > 0.0
    g.close()
    return d1


# per-cell residual kernel (FP64 runs the per-cell update and residual)
@pytest.mark.parametrize("Q", [21, 9])
def test_fp64_polar_per_cell_residual(Q):
    s = polar(Q, CR=0.35 if Q == 21 else 0.0)
    d = run_and_compare(s, "fp64")
    assert d["am"] > 0.0


def test_fp64_stretched_planar_with_body_force():
    run_and_compare(stretched(21), "fp64")


def test_fp64_iterated_force():
    run_and_compare(polar(21, iters=2), "fp64")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_general_grid(prec):
    d = run_and_compare(wavy(21), prec, perturb=2e-3)
    assert d["am"] != 0.0


# the pipelined residual (k_residual_ws) wherever the update is pipelined
@pytest.mark.parametrize("Q", [21, 9])
@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
def test_pipelined_residual_polar(Q, prec):
    run_and_compare(polar(Q, CR=0.35 if Q == 21 else 0.0), prec)


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_pipelined_residual_planar(prec):
    run_and_compare(stretched(21), prec)


def test_fp32_per_cell_residual():
    run_and_compare(polar(21), "fp32", kernel=1)


@pytest.mark.parametrize("kernel", [1, 3])
def test_fp32_ragged_tiles_random_start(kernel):
    """Row and column counts that leave partial tiles; a j-dependent start
    on near-square cells."""
    run_and_compare(polar(21, n1=19, n2=131, CR=0.0), "fp32", kernel=kernel, t1=20, dt=40,
                    perturb=2e-3, seed=9)


def test_residual_without_steps_between_calls_is_infinite():
    """Two calls without a step in between: t - t' = 0 gives +inf, as the
    oracle's definition does."""
    s = polar(21)
    g = s.gpu("fp64")
    g.step(40)
    g.residual()
    r, _ = g.residual()
    assert math.isinf(r)
    g.close()


# batched reduction against the oracle
def test_batch_residual_matches_oracle_for_every_variant():
    c = _clbm()
    setups = [polar(21, n1=12, n2=50), stretched(21, n1=9, n2=33), polar(21, n1=20, n2=130),
              stretched(21, n1=17, n2=257)]
    for variant in range(5):
        stream = torch.cuda.Stream()
        grids = []
        for s in setups:
            g = c.Grid(s.Q, s.n1, s.n2, s.edges, kind=s.kind, step2=s.step2, precision=1,
                       bc_lo=s.bc[0], bc_hi=s.bc[1], stream=stream)
            g.set_case(s.tau, 1.0, s.U0[0], s.U0[1], s.g)
            grids.append(g)
        ors = [s.oracle() for s in setups]
        b = c.Batch(grids)
        b.set_variant(variant)
        b.step(50)
        for o in ors:
            o.step(50)
        r0, c0 = b.residual()
        d0 = [o.diagnostics() for o in ors]
        b.step(70)
        for o in ors:
            o.step(70)
        r1, c1 = b.residual()
        d1 = [o.diagnostics((d["Ut1"], d["Ut2"]), 70) for o, d in zip(ors, d0)]
        for k in range(len(setups)):
            check(c0[k], r0[k], d0[k], "fp32", "variant %d grid %d first" % (variant, k))
            check(c1[k], r1[k], d1[k], "fp32", "variant %d grid %d second" % (variant, k))
        b.close()
        for g in grids:
            g.close()


# the full bench grid
@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_fullsize_bench_grid_diagnostics(prec):
    """The annulus 1024 x 4096 of the bench (D2Q21, CR = 0.35, inner wall at
    0.01, tau = 0.8) from a seeded j-dependent start: the diagnostics of the
    start and, one step later, the residual over that step, against the
    oracle on the whole grid."""
    n1, n2, R1, R2 = 1024, 4096, 1.0, 2.0
    e = I.polar_edges(R1, R2, n1, 0.35)
    U0 = _clbm().wall_speed_polar(0.01, R1, n2, (R2 - R1) / n1)
    s = Setup(21, n1, n2, O.POLAR, edges=e, bc=(1, 0), tau=0.8, U0=(U0, 0.0))
    run_and_compare(s, prec, t1=0, dt=1, perturb=2e-3, seed=5)
