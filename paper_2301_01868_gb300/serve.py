"""Continuous-batching solve server on one GPU.

A request asks for the steady solution of one of the paper's four flows
(planar Couette / Poiseuille, circular Couette / Poiseuille, Sec. 3) on a
given lattice and resolution.  The server keeps every admitted lattice
resident on the device, admits queued requests as soon as their arrival time
has passed and their workspace fits the HBM budget, advances all admitted
lattices together through ``clbm.Batch`` (one persistent launch per phase,
grouped by lattice type), checks every lattice's residual after each chunk
of steps, and retires a lattice when its residual meets the request's
tolerance or its step cap is reached, which frees room for the next ones.
Requests that arrive while others run join the next chunk.

D2Q9 lattices of the circular flows iterate the force once per step (the
implicit form Sec. 2 allows).  On these polar grids D2Q9 grows a radial
velocity in the row next to the inner wall; the lagged force lets it grow
about three times faster than one implicit pass, which lets most D2Q9
circular requests converge first.  Requests whose lattice diverges anyway
end with status "diverged" (D2Q21 and the planar flows stay stable with the
lagged force).  Every result carries its status: converged, capped (step cap
reached) or diverged (non-finite residual).
"""
import math
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np

from . import clbm

CASES = ("planar_couette", "planar_poiseuille", "circular_couette", "circular_poiseuille")


@dataclass
class Request:
    case: str
    lattice: int            # 9 or 21
    n1: int                 # wall-normal cells
    n2: int                 # periodic cells
    tau: float
    speed: float            # wall speed, or target peak velocity of a forced flow
    tol: float = 1e-8       # residual tolerance (clbm_residual)
    arrival: float = 0.0    # seconds after the server starts
    max_steps: int = 200000
    force_iterations: int = -1  # implicit-force passes; -1 picks by lattice and case
    rid: int = 0
    future: Future = field(default=None, repr=False)


def _annulus_peak(M, N):
    """max over r in [M, M+N] of (r^2 - M^2)((M+N)^2 - r^2)/r."""
    r = np.linspace(M, M + N, 2001)
    return float(((r ** 2 - M ** 2) * ((M + N) ** 2 - r ** 2) / r).max())


def force_iterations(req):
    """Implicit-force passes of a request: as asked, else one for D2Q9 on the
    polar grids of the circular flows and none otherwise."""
    if req.force_iterations >= 0:
        return int(req.force_iterations)
    return 1 if req.lattice == 9 and req.case.startswith("circular") else 0


def build_grid(req, precision, stream, device=0):
    """The Grid and case of a request (lattice units, Delta x = 1)."""
    Q, n1, n2 = req.lattice, req.n1, req.n2
    T0 = 1.0 / 3.0 if Q == 9 else 2.0 / 3.0
    it = force_iterations(req)
    nu = T0 * (req.tau - 0.5)
    if req.case.startswith("planar"):
        edges = np.arange(n1 + 1, dtype=np.float64)
        if req.case == "planar_couette":
            g = clbm.Grid(Q, n1, n2, edges, kind=clbm.PLANAR, step2=1.0, precision=precision,
                          bc_lo=clbm.NOSLIP, bc_hi=clbm.MOVING, device=device, stream=stream)
            g.set_case(req.tau, 1.0, 0.0, req.speed, force_iterations=it)
        else:
            g = clbm.Grid(Q, n1, n2, edges, kind=clbm.PLANAR, step2=1.0, precision=precision,
                          bc_lo=clbm.NOSLIP, bc_hi=clbm.NOSLIP, device=device, stream=stream)
            g.set_case(req.tau, 1.0, 0.0, 0.0, (0.0, 8.0 * nu * req.speed / n1 ** 2), force_iterations=it)
        return g
    R1, R2 = 1.0, 2.0
    dx = (R2 - R1) / n1
    edges = R1 + dx * np.arange(n1 + 1, dtype=np.float64)
    if req.case == "circular_couette":
        g = clbm.Grid(Q, n1, n2, edges, kind=clbm.POLAR, precision=precision, bc_lo=clbm.MOVING,
                      bc_hi=clbm.NOSLIP, device=device, stream=stream)
        g.set_case(req.tau, 1.0, clbm.wall_speed_polar(req.speed, R1, n2, dx), 0.0, force_iterations=it)
    else:
        M = R1 / dx
        alpha = math.sin(2.0 * math.pi / n2)
        g2 = 8.0 * nu * req.speed / (alpha * _annulus_peak(M, n1))
        g = clbm.Grid(Q, n1, n2, edges, kind=clbm.POLAR, precision=precision, bc_lo=clbm.NOSLIP,
                      bc_hi=clbm.NOSLIP, device=device, stream=stream)
        g.set_case(req.tau, 1.0, 0.0, 0.0, (0.0, g2), force_iterations=it)
    return g


class Server:
    """Admits requests by HBM footprint and advances them in continuous batches.

    precision : storage / compute of every lattice (clbm precision code or name)
    hbm_budget : bytes of lattice workspace allowed on the device at once
    chunk : time steps between residual checks
    """

    def __init__(self, precision="fp32", hbm_budget=150e9, chunk=100, device=0, tune=True):
        import torch

        self.torch = torch
        self.precision = clbm.PRECISIONS[precision] if isinstance(precision, str) else precision
        self.budget = float(hbm_budget)
        self.chunk = int(chunk)
        self.device = device
        self.tune = tune
        self.stream = torch.cuda.Stream(device=device)
        self.queue = []
        self.active = []          # dicts: req, grid, bytes, steps, t_admit
        self.done = []
        self.used = 0.0
        self._batches = {}
        self._retired = []        # grids of retired lattices, freed once no batch lists them
        self._dirty = True
        self.t0 = None
        self._next_id = 0
        self.tunes = 0            # autotuner runs (a shape class is timed once per process)
        self.deferred = 0         # admission checks that found the head of the queue over budget
        self.peak_bytes = 0.0     # most workspace bytes held at once

    # ------------------------------------------------------------ requests
    def submit(self, req):
        """Queue a request; its Future resolves to a result dict."""
        req.future = Future()
        req.rid = self._next_id
        self._next_id += 1
        need = clbm.workspace_bytes(req.lattice, self.precision, req.n1, req.n2)
        if need > self.budget:
            req.future.set_exception(ValueError("request needs %d bytes, over the budget" % need))
            return req.future
        self.queue.append(req)
        self.queue.sort(key=lambda r: r.arrival)
        return req.future

    def _now(self):
        return time.perf_counter() - self.t0

    def _admit(self):
        now = self._now()
        while self.queue and self.queue[0].arrival <= now:
            req = self.queue[0]
            need = clbm.workspace_bytes(req.lattice, self.precision, req.n1, req.n2)
            if self.used + need > self.budget:
                self.deferred += 1
                break
            self.queue.pop(0)
            g = build_grid(req, self.precision, self.stream, self.device)
            self.active.append(dict(req=req, grid=g, bytes=need, steps=0, t_admit=now, checks=0))
            self.used += need
            self.peak_bytes = max(self.peak_bytes, self.used)
            self._dirty = True

    def _close_batches(self):
        """Destroy every batch, then the grids of retired lattices (a batch
        holds its lattices' handles until it is destroyed)."""
        for b, _ in self._batches.values():
            b.close()
        self._batches = {}
        for g, nbytes in self._retired:
            g.close()
            self.used -= nbytes
        self._retired = []

    def _rebuild(self):
        self._close_batches()
        groups = {}
        for a in self.active:
            groups.setdefault(a["req"].lattice, []).append(a)
        for Q, members in groups.items():
            b = clbm.Batch([a["grid"] for a in members])
            self._batches[Q] = (b, members)
        self._dirty = False

    def _retire(self, a, res, converged):
        req = a["req"]
        g = a["grid"]
        m = g.moments(names=("rho", "Ut1", "Ut2"))
        t_done = self._now()
        out = dict(rid=req.rid, case=req.case, lattice=req.lattice, n1=req.n1, n2=req.n2,
                   steps=g.t, residual=res, converged=converged,
                   status=_status(converged, res),
                   latency=t_done - req.arrival, t_admit=a["t_admit"], t_done=t_done,
                   Ut2_profile=m["Ut2"][:, 0].copy(), rho_profile=m["rho"][:, 0].copy())
        # the grid's memory is released (and leaves the budget) with the
        # batch that still lists it
        self._retired.append((g, a["bytes"]))
        self.done.append(out)
        req.future.set_result(out)
        self._dirty = True

    # -------------------------------------------------------------- loop
    def run(self):
        """Serve until the queue is empty and every admitted lattice retired."""
        self.t0 = time.perf_counter()
        while self.queue or self.active:
            if self._retired:          # free retired lattices before admitting more
                self._close_batches()
                self._dirty = True
            self._admit()
            if not self.active:
                wait = self.queue[0].arrival - self._now()
                if wait > 0:
                    time.sleep(min(wait, 0.05))
                continue
            if self._dirty:
                self._rebuild()
                if self.tune:
                    # time the variants only for a shape class not timed yet in
                    # this process; tuning advances every member (steps + 1 per
                    # usable variant), which the grids' own time counters record
                    for b, _ in self._batches.values():
                        if not b.variant()[1]:
                            b.tune(steps=2)
                            self.tunes += 1
            for b, members in self._batches.values():
                b.step(self.chunk)
            for Q, (b, members) in list(self._batches.items()):
                res, _ = b.residual()   # NaN marks a lattice that went unstable
                for a, r in zip(members, res):
                    a["checks"] += 1
                    a["steps"] = a["grid"].t
                    conv = a["checks"] > 1 and np.isfinite(r) and r <= a["req"].tol
                    if conv or a["steps"] >= a["req"].max_steps or not np.isfinite(r) and a["checks"] > 1:
                        self.active.remove(a)
                        self._retire(a, float(r), bool(conv))
        self._close_batches()
        return self.stats()

    def stats(self):
        out = _stats(self.done)
        out.update(deferred_admissions=self.deferred, peak_workspace_bytes=self.peak_bytes,
                   budget_bytes=self.budget, tuner_runs=self.tunes)
        return out


def serve_serial(requests, precision="fp32", chunk=100, device=0):
    """Baseline: the same requests solved one after another, each on its own
    lattice with single-lattice launches (clbm_step, clbm_residual)."""
    import torch

    stream = torch.cuda.Stream(device=device)
    prec = clbm.PRECISIONS[precision] if isinstance(precision, str) else precision
    t0 = time.perf_counter()
    done = []
    for req in sorted(requests, key=lambda r: r.arrival):
        now = time.perf_counter() - t0
        if req.arrival > now:
            time.sleep(req.arrival - now)
        g = build_grid(req, prec, stream, device)
        steps, checks, r = 0, 0, float("inf")
        conv = False
        while True:
            g.step(chunk)
            steps += chunk
            try:
                r, _ = g.residual()
            except clbm.UnstableError:
                r = float("nan")
            checks += 1
            conv = checks > 1 and np.isfinite(r) and r <= req.tol
            if conv or steps >= req.max_steps or (not np.isfinite(r) and checks > 1):
                break
        m = g.moments(names=("rho", "Ut1", "Ut2"))
        t_done = time.perf_counter() - t0
        done.append(dict(rid=req.rid, steps=steps, residual=r, converged=bool(conv),
                         status=_status(conv, r), latency=t_done - req.arrival, t_done=t_done,
                         service=t_done - max(req.arrival, now),
                         Ut2_profile=m["Ut2"][:, 0].copy(), rho_profile=m["rho"][:, 0].copy()))
        g.close()
    return done, _stats(done)


def _status(converged, res):
    if converged:
        return "converged"
    return "capped" if np.isfinite(res) else "diverged"


def _stats(done):
    """Solves/s and time-to-converged percentiles; every solve counts in the
    throughput, only converged ones in the latency percentiles."""
    if not done:
        return dict(solves=0)
    span = max(d["t_done"] for d in done)
    lat = np.array([d["latency"] for d in done if d["status"] == "converged"])
    n = {k: sum(d["status"] == k for d in done) for k in ("converged", "capped", "diverged")}
    out = dict(solves=len(done), converged=n["converged"], capped=n["capped"],
               diverged=n["diverged"], wall_s=span, solves_per_s=len(done) / span,
               converged_per_s=n["converged"] / span)
    if len(lat):
        out.update(p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)))
    return out


def poisson_requests(n, rate, seed=20230105, n1_range=(16, 64), n2_range=(16, 128),
                     tau_range=(0.55, 1.0), speed_range=(1e-3, 1e-2), tol=1e-8, max_steps=100000,
                     lattices=(9, 21)):
    """Seeded request stream: Poisson arrivals at `rate` per second (0: all at
    once), case and lattice uniform, sizes log-uniform, tau and target speed
    uniform; one seed gives the same requests at every rate.  The
    circular flows (annulus 1 <= r <= 2) take the azimuthal size from the
    radial one so that cells are near-square at the inner wall, as the paper's
    polar grids are (Sec. 3.3); an independent n2 gives cells of aspect ratio
    up to n1 2 pi / n2, on which the curvilinear equilibrium loses stability."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(n):
        # the gap is drawn at every rate (0: everything at t = 0), so streams
        # of one seed hold the same requests at any rate
        gap = rng.exponential(1.0)
        t += gap / rate if rate > 0 else 0.0
        n1 = int(round(math.exp(rng.uniform(math.log(n1_range[0]), math.log(n1_range[1])))))
        n2 = int(round(math.exp(rng.uniform(math.log(n2_range[0]), math.log(n2_range[1])))))
        case = CASES[rng.integers(len(CASES))]
        n1 = max(n1, 8)
        n2 = int(round(n1 * 2.0 * math.pi)) if case.startswith("circular") else max(n2, 4)
        out.append(Request(case=case, lattice=int(rng.choice(lattices)),
                           n1=n1, n2=n2, tau=float(rng.uniform(*tau_range)),
                           speed=float(rng.uniform(*speed_range)), tol=tol, arrival=t,
                           max_steps=max_steps, rid=k))
    return out
