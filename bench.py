"""Throughput of the fused curvilinear LBM update on GB300.

Workload (default): circular Couette flow in the annulus 1 <= r <= 2 with the
App. C contracted radial grid (CR = 0.35), D2Q21, FP32 compute and storage,
N_r x N_theta = 1024 x 4096, inner wall at u_theta = 0.01, outer wall at rest,
tau = 0.8, from rest.  One bench step = `--chunk` time steps of the whole hot
path (boundary fill + fused stream-collide-force per time step) followed by
one residual / conservation reduction.  Metric: million lattice-cell updates
per second (MLUPS), whole job over all ranks.

The state (2 x 352 MB) is larger than the 129 MB L2, so no flush is needed
between steps.  Under torchrun every rank advances its own replica (weak
scaling, no data-path collective).

--impl reference times the FP64 CPU oracle instead (the only reference this
paper has): each of its steps is one oracle time step of the same annulus at
a bounded size.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import clbm_inputs as I  # noqa: E402

WORKLOADS = {
    # name: (Q, precision, n1, n2, R1, R2, CR, tau, u_wall)
    "circular_couette_d2q21_fp32_1024x4096": (21, "fp32", 1024, 4096, 1.0, 2.0, 0.35, 0.8, 0.01),
    "circular_couette_d2q21_f16_1024x4096": (21, "fp16", 1024, 4096, 1.0, 2.0, 0.35, 0.8, 0.01),
    "circular_couette_d2q21_bf16_1024x4096": (21, "bf16", 1024, 4096, 1.0, 2.0, 0.35, 0.8, 0.01),
    "circular_couette_d2q21_fp64_1024x4096": (21, "fp64", 1024, 4096, 1.0, 2.0, 0.35, 0.8, 0.01),
    "circular_couette_d2q9_fp32_1024x4096": (9, "fp32", 1024, 4096, 1.0, 2.0, 0.35, 0.8, 0.01),
    "circular_couette_d2q21_fp32_128x512": (21, "fp32", 128, 512, 1.0, 2.0, 0.35, 0.8, 0.01),
    # half the bench grid: the case ncu's full captures run on (state 2 x 176 MB, above L2)
    "circular_couette_d2q21_fp32_512x4096": (21, "fp32", 512, 4096, 1.0, 2.0, 0.35, 0.8, 0.01),
    "circular_couette_d2q21_f16_512x4096": (21, "fp16", 512, 4096, 1.0, 2.0, 0.35, 0.8, 0.01),
}
# general (non-separable) grids: name -> (Q, precision, n1, n2, amplitude, tau, u_wall)
GENERAL_WORKLOADS = {
    "wavy_channel_d2q21_fp32_1024x4096": (21, "fp32", 1024, 4096, 0.15, 0.8, 0.01),
}
TABLE_VALUES_PER_CELL = {21: 73, 9: 37}   # per-cell table entries of general grids
# three-dimensional workloads (D3Q39): name -> (precision, n1, n2, n3, R1, R2, CR, tau, u_wall)
THREE_D_WORKLOADS = {
    "annulus3d_d3q39_fp32_128x804x32": ("fp32", 128, 804, 32, 1.0, 2.0, 0.35, 0.8, 0.01),
    "annulus3d_d3q39_fp64_128x804x32": ("fp64", 128, 804, 32, 1.0, 2.0, 0.35, 0.8, 0.01),
    "annulus3d_d3q39_f16_128x804x32": ("fp16", 128, 804, 32, 1.0, 2.0, 0.35, 0.8, 0.01),
    "annulus3d_d3q39_bf16_128x804x32": ("bf16", 128, 804, 32, 1.0, 2.0, 0.35, 0.8, 0.01),
}
DEFAULT = "circular_couette_d2q21_fp32_1024x4096"
METRIC = "D2Q21 curvilinear MLUPS and % HBM roofline; served solves/s, p99 latency"
STORAGE_BYTES = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}
KERNEL_SOURCES = ["paper_2301_01868_gb300/csrc/k_step.cu",
                  "paper_2301_01868_gb300/csrc/k_step_tma.cu",
                  "paper_2301_01868_gb300/csrc/clbm_cell.cuh",
                  "paper_2301_01868_gb300/csrc/clbm_f2.cuh",
                  "paper_2301_01868_gb300/csrc/clbm_internal.cuh",
                  "paper_2301_01868_gb300/csrc/clbm_lattice.cuh",
                  "paper_2301_01868_gb300/csrc/clbm_sync.cuh"]


def kernel_hash():
    """Hash of the update kernels' code (comments and blank space left out, so
    that only a change of the code makes a captured traffic figure stale)."""
    import re
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p)) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def traffic_for(workload, kernel):
    """Per-launch DRAM bytes of the timed update kernel from the committed ncu
    summary, only if it was taken on the current kernel source (kernel 1: the
    per-cell kernel; 0 and 3: the pipelined TMA kernel, the automatic choice
    for 16/32-bit storage; 2: not captured)."""
    p = os.path.join(ROOT, "profiles", "fused_step_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(workload)
    if not e or e.get("kernel_hash") != kernel_hash():
        return None
    if kernel == 2:
        return None
    return e.get("bytes_per_launch_per_cell_kernel" if kernel == 1 else "bytes_per_launch")


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.idx)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


_T0 = time.perf_counter()


def progress(what):
    """One line on stderr per finished part of the run (the JSON line goes to stdout)."""
    print("[bench %.0f s] %s done" % (time.perf_counter() - _T0, what), file=sys.stderr, flush=True)


def max_over_ranks(x, dist, device):
    """Largest value of x over all ranks (x itself without a process group)."""
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    if dist is not None and dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(cells, chunk, steps, world, ms_max):
    """Cell updates of every rank's replica per second of the slowest rank, in millions."""
    return cells * chunk * steps * world / (ms_max * 1e-3) / 1e6


def smi_index(local):
    """nvidia-smi index (or UUID) of this rank's GPU."""
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if not vis:
        return local
    return vis.split(",")[local].strip()


def wavy(wl):
    """Wavy channel between straight walls (general grid), low wall moving."""
    Q, prec, n1, n2, amp, tau, uw = GENERAL_WORKLOADS[wl]
    nodes = I.mapped_nodes(I.wavy_channel(n1, n2, amp=amp), n1, n2, "extend")
    return Q, prec, n1, n2, nodes, tau, uw


def annulus(wl):
    Q, prec, n1, n2, R1, R2, CR, tau, uw = WORKLOADS[wl]
    e = I.polar_edges(R1, R2, n1, CR)
    dx = (R2 - R1) / n1
    U0 = uw * dx / (R1 * math.sin(2.0 * math.pi / n2))
    return Q, prec, n1, n2, e, tau, U0


def cpu_baseline(wl, target_s=12.0, max_steps=50, parity=True):
    """The FP64 oracle as it stands on this host's cores: MLUPS on the full
    workload grid, as many whole time steps as fit in about target_s.  With
    parity, the same grid is then advanced on the GPU for as many steps from
    rest and its velocity compared with the oracle's (normwise L2 over every
    cell: the full-size parity of the timed configuration)."""
    from oracle import oracle as O
    Q, prec, n1, n2, e, tau, U0 = annulus(wl)
    o = O.Grid(Q, n1, n2, O.POLAR, edges=e, bc_lo=O.MOVING, bc_hi=O.NOSLIP)
    o.set_case(tau, 1.0, U0, 0.0)
    o.init_rest()
    t0 = time.perf_counter()
    o.step(1)
    t1 = time.perf_counter() - t0
    n = max(1, min(max_steps, int(target_s / max(t1, 1e-9)) - 1))
    t0 = time.perf_counter()
    o.step(n)
    dt = time.perf_counter() - t0
    out = {"value": n1 * n2 * n / dt / 1e6, "unit": "MLUPS", "cores": O.threads(),
           "kind": "oracle",
           "sample": "%d time steps of the full %dx%d D2Q%d FP64 oracle grid (%.1f s), "
                     "after one untimed step" % (n, n1, n2, Q, dt)}
    if parity:
        from paper_2301_01868_gb300 import clbm
        ref = o.moments()
        g = clbm.Grid(Q, n1, n2, e, kind=clbm.POLAR, precision=prec, bc_lo=clbm.MOVING,
                      bc_hi=clbm.NOSLIP)
        g.set_case(tau, 1.0, U0, 0.0)
        g.step(1 + n)
        m = g.moments(names=("Ut1", "Ut2"))
        g.close()
        num = ((m["Ut1"] - ref["Ut1"]) ** 2 + (m["Ut2"] - ref["Ut2"]) ** 2).sum()
        den = (ref["Ut1"] ** 2 + ref["Ut2"] ** 2).sum()
        out["parity"] = {"steps": 1 + n, "velocity_l2_vs_oracle": float(math.sqrt(num / den)),
                         "what": "whole %dx%d grid from rest, GPU (%s, automatic kernel) against "
                                 "the oracle after the same steps" % (n1, n2, prec)}
    return out


def steady_accuracy():
    """L2 velocity errors of the precision ladder at a steady state against
    the FP64 oracle and the exact profile (Eq. 27): circular Couette on the
    annulus at N_r = 32, N_theta = 201, tau = 0.8, 6000 steps from rest; the
    oracle's profile is the committed fixture tests/golden/steady_profiles.txt
    (written by the oracle; the bench does not run it)."""
    from paper_2301_01868_gb300 import clbm
    path = os.path.join(ROOT, "tests", "golden", "steady_profiles.txt")
    hdr, rows = {}, []
    with open(path) as f:
        for ln in f:
            if ln.startswith("#") or not ln.strip():
                continue
            p = ln.split()
            if p[0].isalpha():
                hdr[p[0]] = float(p[1])
            else:
                rows.append([float(x) for x in p])
    rows = np.array(rows)
    nr, nt, tau, uw, steps = (int(hdr["NR"]), int(hdr["NTHETA"]), hdr["TAU"], hdr["UWALL"],
                              int(hdr["STEPS"]))
    r_lat, exact, orc = rows[:, 0], rows[:, 1], {21: rows[:, 2], 9: rows[:, 3]}
    edges = I.polar_edges(1.0, 2.0, nr)
    sn = math.sin(2.0 * math.pi / nt)
    U0 = uw / (sn * (1.0 / ((2.0 - 1.0) / nr)))
    out = []
    for Q, prec in ((21, "fp64"), (21, "fp32"), (21, "fp16"), (21, "bf16"), (9, "fp64"), (9, "fp32")):
        g = clbm.Grid(Q, nr, nt, edges, kind=clbm.POLAR, precision=prec, bc_lo=clbm.MOVING,
                      bc_hi=clbm.NOSLIP)
        g.set_case(tau, 1.0, U0, 0.0)
        g.step(steps)
        u = g.moments(names=("Ut2",))["Ut2"][:, 0] * sn * r_lat
        g.close()
        out.append({"lattice": "D2Q%d" % Q, "storage": prec,
                    "l2_vs_oracle": float(np.linalg.norm(u - orc[Q]) / np.linalg.norm(orc[Q])),
                    "l2_vs_exact": float(np.linalg.norm(u - exact) / np.linalg.norm(exact)),
                    "oracle_l2_vs_exact": float(np.linalg.norm(orc[Q] - exact) / np.linalg.norm(exact))})
    return {"case": "circular Couette, annulus 1 <= r <= 2, N_r=%d, N_theta=%d, tau=%g, "
                    "%d steps from rest" % (nr, nt, tau, steps), "ladder": out}


def _timed_steps(g, torch, stream, steps):
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    g.step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1)


def precision_records(steps=300):
    """The other storage types and lattices on the bench grid (annulus
    1024 x 4096, CR = 0.35): average update launch from CUDA events (graph
    replays of 10 launches), MLUPS, and the fraction of the measured HBM
    peak at 2 Q s bytes per cell update."""
    import torch
    from paper_2301_01868_gb300 import clbm
    peak, _ = peaks()
    out = []
    for wl in ("circular_couette_d2q21_f16_1024x4096", "circular_couette_d2q21_bf16_1024x4096",
               "circular_couette_d2q9_fp32_1024x4096", "circular_couette_d2q21_fp64_1024x4096"):
        Q, prec, n1, n2, e, tau, U0 = annulus(wl)
        stream = torch.cuda.Stream()
        g = clbm.Grid(Q, n1, n2, e, kind=clbm.POLAR, precision=prec, bc_lo=clbm.MOVING,
                      bc_hi=clbm.NOSLIP, stream=stream)
        g.set_case(tau, 1.0, U0, 0.0)
        n = steps if prec != "fp64" else 60
        g.step(n)
        g.set_profiling(True, period=10)
        ms = _timed_steps(g, torch, stream, n)
        kms, kl = g.kernel_time()
        g.set_profiling(False)
        g.close()
        alg = 2 * Q * STORAGE_BYTES[prec] * n1 * n2
        k_avg = kms / kl if kl else ms / n
        out.append({"workload": wl, "mlups": n1 * n2 * n / (ms * 1e-3) / 1e6, "kernel_ms_avg": k_avg,
                    "algorithmic_bytes_per_launch": alg,
                    "hbm_frac": alg / (k_avg * 1e-3) / 1e9 / peak,
                    "bound": "FP64 pipe (HBM fraction for reference)" if prec == "fp64" else "hbm"})
    return out


def config_records():
    """The small configurations, GPU beside the oracle on the same grid:
    planar Couette (D2Q9 FP64, 16 x 32 cells twice as long as wide, top wall
    at 0.01, tau = 1, 20000 steps: MLUPS and the L2 error of the final
    profile against the linear exact one) and the stretched planar
    Poiseuille ladder (D2Q21 FP64 and FP32, 64x16 .. 512x128, stretch
    1.02^(64/n1) per cell, g = 1e-6 (64/n1)^2, tau = 0.6: MLUPS over 2000
    steps).  The oracle is timed on the host cores over a bounded number of
    steps, and the GPU's velocity after those steps is compared with the
    oracle's."""
    import torch
    from oracle import oracle as O
    from paper_2301_01868_gb300 import clbm
    stream = torch.cuda.Stream()
    out = {}
    # planar Couette
    n1, n2 = 16, 32
    e = I.uniform_edges(n1)
    g = clbm.Grid(9, n1, n2, e, kind=clbm.PLANAR, step2=2.0, precision="fp64", bc_lo=clbm.NOSLIP,
                  bc_hi=clbm.MOVING, stream=stream)
    g.set_case(1.0, 1.0, 0.0, 0.005)
    ms = _timed_steps(g, torch, stream, 20000)
    u = 2.0 * g.moments(names=("Ut2",))["Ut2"][:, 0]
    g.close()
    ex = 0.01 * (np.arange(n1) + 0.5) / n1
    o = O.Grid(9, n1, n2, O.PLANAR, edges=e, step2=2.0, bc_lo=O.NOSLIP, bc_hi=O.MOVING)
    o.set_case(1.0, 1.0, 0.0, 0.005)
    o.init_rest()
    t0 = time.perf_counter()
    o.step(2000)
    dto = time.perf_counter() - t0
    g2 = clbm.Grid(9, n1, n2, e, kind=clbm.PLANAR, step2=2.0, precision="fp64", bc_lo=clbm.NOSLIP,
                   bc_hi=clbm.MOVING, stream=stream)
    g2.set_case(1.0, 1.0, 0.0, 0.005)
    g2.step(2000)
    ug, uo = g2.moments(names=("Ut2",))["Ut2"], o.moments()["Ut2"]
    g2.close()
    out["planar_couette_d2q9_fp64_16x32"] = {
        "gpu_mlups": n1 * n2 * 20000 / (ms * 1e-3) / 1e6, "steps": 20000,
        "l2_vs_exact": float(np.linalg.norm(u - ex) / np.linalg.norm(ex)),
        "oracle_mlups": n1 * n2 * 2000 / dto / 1e6, "oracle_cores": O.threads(), "oracle_steps": 2000,
        "l2_vs_oracle_at_oracle_steps": float(np.linalg.norm(ug - uo) / np.linalg.norm(uo))}
    # stretched planar Poiseuille ladder
    tau = 0.6
    nu = (2.0 / 3.0) * (tau - 0.5)
    for (n1, n2) in ((64, 16), (128, 32), (256, 64), (512, 128)):
        e = I.geometric_stretch_edges(n1, 1.02 ** (64.0 / n1), float(n1))
        gacc = 1e-6 * (64.0 / n1) ** 2
        rec = {"stretch_per_cell": 1.02 ** (64.0 / n1), "g": gacc}
        osteps = 2000 if n1 <= 128 else 200
        o = O.Grid(21, n1, n2, O.PLANAR, edges=e, step2=1.0)
        o.set_case(tau, 1.0, 0.0, 0.0, (0.0, gacc))
        o.init_rest()
        t0 = time.perf_counter()
        o.step(osteps)
        dto = time.perf_counter() - t0
        uo = o.moments()["Ut2"]
        rec.update(oracle_mlups=n1 * n2 * osteps / dto / 1e6, oracle_cores=O.threads(), oracle_steps=osteps)
        for prec in ("fp64", "fp32"):
            g = clbm.Grid(21, n1, n2, e, kind=clbm.PLANAR, step2=1.0, precision=prec, stream=stream)
            g.set_case(tau, 1.0, 0.0, 0.0, (0.0, gacc))
            g.step(osteps)
            ug = g.moments(names=("Ut2",))["Ut2"]
            ms = _timed_steps(g, torch, stream, 2000)
            g.close()
            rec[prec] = {"gpu_mlups": n1 * n2 * 2000 / (ms * 1e-3) / 1e6,
                         "l2_vs_oracle_at_oracle_steps": float(np.linalg.norm(ug - uo) / np.linalg.norm(uo))}
        out["planar_poiseuille_d2q21_%dx%d" % (n1, n2)] = rec
    return out


def run_reference(args):
    """--impl reference: the oracle, each step one time step of the same
    annulus at 128 x 512 (a bounded sample of the workload)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    wl = args.workload
    Q, prec, _, _, R1, R2, CR, tau, uw = WORKLOADS[wl]
    n1, n2 = 128, 512
    e = I.polar_edges(R1, R2, n1, CR)
    U0 = uw * ((R2 - R1) / n1) / (R1 * math.sin(2.0 * math.pi / n2))
    o = O.Grid(Q, n1, n2, O.POLAR, edges=e, bc_lo=O.MOVING, bc_hi=O.NOSLIP)
    o.set_case(tau, 1.0, U0, 0.0)
    o.init_rest()
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    v = n1 * n2 * args.steps / dt / 1e6
    cfg = config_of(wl, args)
    cfg.update(n1=n1, n2=n2, sample_of="%dx%d" % WORKLOADS[wl][2:4],
               l2="oracle on the host (no GPU)")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": cfg,
           "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": O.threads(), "kind": "oracle",
                            "sample": "%d oracle time steps of the same annulus at %dx%d"
                                      % (args.steps, n1, n2)},
           "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def config_of(wl, args):
    if wl in GENERAL_WORKLOADS:
        Q, prec, n1, n2, amp, tau, uw = GENERAL_WORKLOADS[wl]
        geom = "wavy channel (general grid, per-cell tables), amplitude %g" % amp
    else:
        Q, prec, n1, n2, R1, R2, CR, tau, uw = WORKLOADS[wl]
        geom = "annulus R2/R1=%g, radial CR=%g" % (R2 / R1, CR)
    return {"workload": wl, "lattice": "D2Q%d" % Q, "n1": n1, "n2": n2, "geometry": geom,
            "tau": tau, "u_wall": uw,
            "storage": prec, "chunk": args.chunk,
            "kernel": {0: "auto", 1: "per-cell", 2: "tma-tiles", 3: "tma-pipeline",
                       4: "tma-pipeline, two cells per thread",
                       5: "tma-pipeline, multi-step launches",
                       6: "tma-pipeline, two cells per thread, multi-step launches"}[args.kernel],
            "l2": "inputs larger than L2 (state %d MB)" % (2 * Q * n1 * n2 * STORAGE_BYTES[prec] >> 20),
            "parallelism": "replicas" if args.gpus > 1 else "single"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--chunk", type=int, default=100, help="time steps per bench step")
    ap.add_argument("--impl", default="clbm", choices=["clbm", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS) + sorted(GENERAL_WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-inputs", choices=("state", "state_serial", "fields"), default="state",
                    help="what the e2e leg uploads each step: the FP64 state with the copies overlapping "
                         "the previous step (default), the same copies in series, or the macroscopic fields")
    ap.add_argument("--kernel", type=int, default=0,
                    help="0 automatic, 1 one thread per cell, 2 TMA-staged tiles, "
                         "3 TMA-staged warp-specialised pipeline, 4 the same with two cells per "
                         "thread in packed arithmetic, 5 / 6 kernels 3 / 4 with many time steps "
                         "per launch")
    ap.add_argument("--serve", action="store_true",
                    help="only the serving comparison (continuous batching vs serial solves)")
    ap.add_argument("--serve-requests", type=int, default=48)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="leave out the accuracy, precision, batch and small-configuration records")
    ap.add_argument("--batch", action="store_true",
                    help="only the batched form against per-lattice launches (512 lattices)")
    ap.add_argument("--batch-lattices", type=int, default=512)
    ap.add_argument("--batch-select", default="first", choices=["first", "smallest"],
                    help="--batch: the first --batch-lattices lattices of the configured 512, "
                         "or the smallest")
    ap.add_argument("--slab", action="store_true",
                    help="with N ranks, split the one lattice into N slabs along q^2 (strong "
                         "scaling, a halo exchange every time step) instead of N replicas")
    ap.add_argument("--three-d", default=None, choices=sorted(THREE_D_WORKLOADS),
                    help="only the three-dimensional (D3Q39) update on this workload")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.batch:
        return run_batch(args)
    if args.three_d:
        return run_3d(args)
    if args.serve:
        print(json.dumps(run_serving(args.serve_requests, verbose=True)))
        return
    if args.slab:
        return run_slab(args)

    import torch
    from paper_2301_01868_gb300 import clbm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    wl = args.workload
    stream = torch.cuda.Stream()
    general = wl in GENERAL_WORKLOADS
    if general:
        Q, prec, n1, n2, nodes, tau, U0 = wavy(wl)
        g = clbm.Grid(Q, n1, n2, None, kind=clbm.GENERAL, nodes=nodes, dx=1.0, precision=prec,
                      bc_lo=clbm.MOVING, bc_hi=clbm.NOSLIP, device=local, stream=stream)
    else:
        Q, prec, n1, n2, e, tau, U0 = annulus(wl)
        g = clbm.Grid(Q, n1, n2, e, kind=clbm.POLAR, precision=prec, bc_lo=clbm.MOVING,
                      bc_hi=clbm.NOSLIP, device=local, stream=stream)
    g.set_case(tau, 1.0, U0, 0.0)
    if args.kernel:
        g.set_kernel(args.kernel)

    def bench_step():
        g.step(args.chunk)
        return g.residual()

    for _ in range(args.warmup):
        bench_step()
    clocks = Clocks(smi_index(local))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # graph replays of 10 back-to-back update launches are timed as a whole
    # (plain launches: every 10th, the events cost ~2 us each)
    g.set_profiling(True, period=10)
    launches0 = g.launch_count()
    barrier()
    clocks.start()
    time.sleep(0.3)
    ev0.record(stream)
    last = None
    for _ in range(args.steps):
        last = bench_step()
    ev1.record(stream)
    barrier()
    ck = clocks.stop()
    launches = g.launch_count() - launches0
    ms = ev0.elapsed_time(ev1)
    kms, kl = g.kernel_time()
    g.set_profiling(False)
    ms_max = max_over_ranks(ms, dist, "cuda")
    cells = n1 * n2
    value = whole_job_mlups(cells, args.chunk, args.steps, world, ms_max)
    sb = STORAGE_BYTES[prec]
    bytes_per_launch = 2 * Q * sb * cells
    if general:   # the per-cell tables are read once per update as well
        bytes_per_launch += TABLE_VALUES_PER_CELL[Q] * (8 if prec == "fp64" else 4) * cells
    achieved = bytes_per_launch / (kms / kl * 1e-3) / 1e9 if kl else None
    peak, peak_src = peaks()
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None, "traffic": traffic_for(wl, args.kernel) if prec != "fp64" else None,
            "peak_source": peak_src + " (hbm_gbs)", "algorithmic_bytes_per_launch": bytes_per_launch,
            "kernel_ms_avg": kms / kl if kl else None}

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(g, args, torch, stream, world, dist, cells, Q, args.e2e_inputs)

    out = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": {"fp64": "f64", "fp32": "f32", "fp16": "f32 compute, f16 storage",
                     "bf16": "f32 compute, bf16 storage"}[prec],
           "data": "synthetic", "config": config_of(wl, args), "roofline": roof,
           "gpu_launches": launches, "clocks": ck, "e2e": e2e,
           "residual_last": last[0] if last else None}
    g.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not general:
        out["cpu_baseline"] = cpu_baseline(wl)
        progress("cpu baseline")
    if rank == 0 and world == 1 and not args.no_extras:
        out["accuracy"] = steady_accuracy()
        if "cpu_baseline" in out:
            out["accuracy"]["full_grid"] = out["cpu_baseline"].get("parity")
        progress("accuracy")
        if wl == DEFAULT:
            out["precisions"] = precision_records()
            progress("precisions")
            out["batch"] = batch_record()
            progress("batch")
            out["three_d"] = [three_d_record(w, 10, 3, 100)
                              for w in ("annulus3d_d3q39_fp32_128x804x32", "annulus3d_d3q39_f16_128x804x32")]
            progress("3-D")
            if not args.no_cpu_baseline:
                out["configs"] = config_records()
                progress("configs")
    if rank == 0 and world == 1 and not args.no_serve:
        out["serving"] = run_serving(args.serve_requests)
        progress("serving")
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


def run_slab(args):
    """--slab: the workload's lattice split into one slab per rank along the
    periodic direction (paper_2301_01868_gb300.slab), each step followed by
    the halo exchange of the crossing populations with both neighbours
    (NCCL point-to-point between GPUs) and the residual reduced over the
    ranks.  value = the whole lattice's cell updates per second of the
    slowest rank (strong scaling: the work is fixed as N grows)."""
    import torch
    from paper_2301_01868_gb300 import clbm, slab
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    Q, prec, n1, n2, e, tau, U0 = annulus(args.workload)
    stream = torch.cuda.Stream()
    s = slab.Slab(Q, n1, n2, e, kind=clbm.POLAR, precision=prec, bc_lo=clbm.MOVING, bc_hi=clbm.NOSLIP,
                  device=local, stream=stream, rank=rank, world=world)
    s.set_case(tau, 1.0, U0, 0.0)

    def bench_step():
        s.step(args.chunk)
        return s.residual()

    for _ in range(args.warmup):
        bench_step()
    clocks = Clocks(smi_index(local))
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    launches0 = s.grid.launch_count()
    last = None
    for _ in range(args.steps):
        last = bench_step()
    ev1.record(stream)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
    value = n1 * n2 * args.chunk * args.steps / (ms * 1e-3) / 1e6
    out = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "strong", "vs_baseline": None,
           "dtype": {"fp64": "f64", "fp32": "f32", "fp16": "f32 compute, f16 storage",
                     "bf16": "f32 compute, bf16 storage"}[prec],
           "data": "synthetic",
           "config": dict(config_of(args.workload, args), parallelism="slabs along q^2 (%d)" % world,
                          slab_columns=[s.j0, s.j1]),
           "gpu_launches": s.grid.launch_count() - launches0, "clocks": ck,
           "residual_last": last[0] if last else None, "roofline": None, "e2e": None}
    if rank == 0:
        print(json.dumps(out))
    s.close()
    if dist is not None:
        dist.destroy_process_group()


def annulus3d(wl):
    prec, n1, n2, n3, R1, R2, CR, tau, uw = THREE_D_WORKLOADS[wl]
    e = I.polar_edges(R1, R2, n1, CR)
    dx = (R2 - R1) / n1
    U0 = uw * dx / (R1 * math.sin(2.0 * math.pi / n2))
    return prec, n1, n2, n3, e, dx, tau, U0


def cpu_baseline_3d(wl, target_s=10.0):
    """The FP64 3-D oracle on this host: MLUPS on a bounded sample of the
    workload (the same annulus at n1 / 8 x n2 / 8 x 4 cells)."""
    from oracle import oracle3d as O3
    prec, n1, n2, n3, e, dx, tau, U0 = annulus3d(wl)
    m1, m2, m3 = n1 // 8, n2 // 8, 4
    R1, R2 = e[0], e[-1]
    es = I.polar_edges(R1, R2, m1, THREE_D_WORKLOADS[wl][6])
    o = O3.Grid(m1, m2, m3, O3.ANNULUS, edges=es, step3=(R2 - R1) / m1, bc_lo=O3.MOVING, bc_hi=O3.NOSLIP)
    o.set_case(tau, 1.0, U0, 0.0)
    o.init_rest()
    t0 = time.perf_counter()
    o.step(1)
    t1 = time.perf_counter() - t0
    n = max(1, min(50, int(target_s / max(t1, 1e-9)) - 1))
    t0 = time.perf_counter()
    o.step(n)
    dt = time.perf_counter() - t0
    return {"value": m1 * m2 * m3 * n / dt / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": "%d time steps of the same annulus at %dx%dx%d, D3Q39 FP64 oracle (%.1f s)"
                      % (n, m1, m2, m3, dt)}


def three_d_record(wl, steps, warmup, chunk, kernel=0, cpu=False):
    """The D3Q39 update on an extruded annulus, timed like the main line
    (chunk time steps per bench step, CUDA events on the grid's stream);
    roofline on the whole step (one update launch, ghost rows included)."""
    import torch
    from paper_2301_01868_gb300 import clbm
    prec, n1, n2, n3, e, dx, tau, U0 = annulus3d(wl)
    stream = torch.cuda.Stream()
    g = clbm.Grid3(n1, n2, n3, e, kind=clbm.ANNULUS3, step3=dx, precision=prec, bc_lo=clbm.MOVING,
                   bc_hi=clbm.NOSLIP, stream=stream)
    g.set_case(tau, 1.0, U0, 0.0)
    if kernel:
        g.set_kernel(kernel)
    for _ in range(warmup):
        g.step(chunk)
    torch.cuda.synchronize()
    clocks = Clocks(smi_index(0))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.start()
    time.sleep(0.3)
    ev0.record(stream)
    for _ in range(steps):
        g.step(chunk)
    ev1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    cells = n1 * n2 * n3
    nsteps = chunk * steps
    sb = STORAGE_BYTES[prec]
    bytes_per_step = 2 * 39 * sb * cells
    achieved = bytes_per_step / (ms * 1e-3 / nsteps) / 1e9
    peak, peak_src = peaks()
    tot = g.totals()
    out = {"metric": "D3Q39 curvilinear MLUPS and % HBM roofline", "value": cells * nsteps / (ms * 1e-3) / 1e6,
           "unit": "MLUPS", "n_gpus": 1, "steps": steps, "warmup": warmup,
           "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": {"fp64": "f64", "fp32": "f32", "fp16": "f32 compute, f16 storage",
                     "bf16": "f32 compute, bf16 storage"}[prec], "data": "synthetic",
           "config": {"workload": wl, "lattice": "D3Q39", "n1": n1, "n2": n2, "n3": n3,
                      "geometry": "annulus R2/R1=2 extruded along z, radial CR=%g" % THREE_D_WORKLOADS[wl][6],
                      "tau": tau, "u_wall": THREE_D_WORKLOADS[wl][8], "storage": prec, "chunk": chunk,
                      "l2": "inputs larger than L2 (state %d MB)" % (2 * 39 * cells * sb >> 20)},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": None, "peak_source": peak_src + " (hbm_gbs)",
                        "algorithmic_bytes_per_launch": bytes_per_step,
                        "kernel_ms_avg": ms / nsteps, "timed": "whole time step (the update, which also fills the next step's ghost rows)"},
           "gpu_launches": nsteps, "clocks": ck, "mass_after": tot[0]}
    g.close()
    if cpu:
        out["cpu_baseline"] = cpu_baseline_3d(wl)
    return out


def run_3d(args):
    """--three-d WL: only the 3-D record, one JSON line."""
    print(json.dumps(three_d_record(args.three_d, args.steps, args.warmup, args.chunk, args.kernel,
                                    cpu=not args.no_cpu_baseline)))


def _fifo_latencies(reqs, service):
    """Time-to-done of one FIFO server with the given service times at the
    requests' arrival times (the serial baseline at any arrival rate, from
    its service times measured once)."""
    t_free = 0.0
    out = []
    for r in sorted(reqs, key=lambda q: q.arrival):
        start = max(r.arrival, t_free)
        t_free = start + service[r.rid]
        out.append((r.rid, t_free - r.arrival, t_free))
    return out


def _pct(x, q):
    return float(np.percentile(np.asarray(x), q)) if len(x) else None


LADDER = dict(n1_range=(8, 256), n2_range=(8, 512), tol=1e-8, max_steps=30000)
LITERAL = dict(n1_range=(64, 2048), n2_range=(64, 4096), tol=1e-8, max_steps=500)


def run_serving(n=48, rates=(0.5, 0.8, 1.2), literal_n=64, verbose=False):
    """Served solves/s and time-to-converged (continuous batching against
    serial single-lattice solves), on seeded Poisson streams of solve
    requests: the four flows, D2Q9 / D2Q21 at random, tau in [0.55, 1],
    target speed in [1e-3, 1e-2], residual tolerance 1e-8, FP32 state with
    FP64 residuals.

    ladder: n1 log-uniform 8..256 (circular n2 = round(2 pi n1), planar n2
      log-uniform 8..512), a cap of 30,000 steps per request.  The serial
      path solves the stream once, back to back: its capacity C (solves/s)
      and each request's service time.  The server then takes the same
      requests at Poisson rates of 0.5, 0.8 and 1.2 C, with an HBM budget of
      30 % of the stream's total workspace so that admission binds; the
      serial latencies at each rate follow from its measured service times
      (one FIFO server at the same arrivals).
    literal: a sample of the configured distribution (n1 log-uniform
      64..2048, n2 64..4096, circular n2 from n1 as above) all queued at
      once under the configured 150 GB budget, each capped at 500 steps (a
      literal request needs up to ~3e7 steps to converge): the server's
      solves/s and the converged / capped / diverged counts."""
    from paper_2301_01868_gb300 import clbm, serve
    t_start = time.perf_counter()
    base = serve.poisson_requests(n, 0.0, **LADDER)
    done_serial, serial = serve.serve_serial(base, precision="fp32", chunk=100)
    service = {d["rid"]: d["service"] for d in done_serial}
    status_serial = {d["rid"]: d["status"] for d in done_serial}
    cap = n / sum(service.values())
    need = [clbm.workspace_bytes(r.lattice, clbm.FP32, r.n1, r.n2) for r in base]
    budget = 1.5 * max(need)      # two of the largest lattices never fit at once
    sweep = []
    for f in rates:
        reqs = serve.poisson_requests(n, f * cap, **LADDER)
        srv = serve.Server(precision="fp32", hbm_budget=budget, chunk=100)
        for r in reqs:
            srv.submit(r)
        st = srv.run()
        fifo = _fifo_latencies(reqs, service)
        conv_lat = [lat for rid, lat, _ in fifo if status_serial[rid] == "converged"]
        span = max(t for _, _, t in fifo)
        differ = sum(1 for d in srv.done if d["status"] != status_serial[d["rid"]])
        sweep.append({"rate_x_serial_capacity": f, "arrival_rate_per_s": f * cap,
                      "batched": st,
                      "serial": {"solves_per_s": n / span,
                                 "converged_per_s": sum(v == "converged" for v in status_serial.values()) / span,
                                 "p50_s": _pct(conv_lat, 50), "p99_s": _pct(conv_lat, 99)},
                      "status_differs": differ})
        if verbose:
            print(json.dumps(sweep[-1]), file=sys.stderr)
    lit = serve.poisson_requests(literal_n, 0.0, seed=20230106, **LITERAL)
    srv = serve.Server(precision="fp32", hbm_budget=150e9, chunk=100)
    for r in lit:
        srv.submit(r)
    literal = srv.run()
    literal["cells_per_request_mean"] = float(np.mean([r.n1 * r.n2 for r in lit]))
    mid = sweep[len(sweep) // 2]
    out = {"requests_per_rate": n,
           "ladder": "n1 8..256 log-uniform (circular n2 = round(2 pi n1), planar n2 8..512); "
                     "tol 1e-8; cap 30000 steps; HBM budget 1.5 x the largest request's workspace",
           "serial_capacity_solves_per_s": cap, "serial": serial, "budget_bytes": budget,
           "sweep": sweep,
           "speedup_solves_per_s_at_0.8": mid["batched"]["solves_per_s"] / mid["serial"]["solves_per_s"],
           "literal": dict(literal, requests=literal_n,
                           distribution="n1 64..2048, n2 64..4096 log-uniform (circular n2 = round(2 pi n1)); "
                                        "tol 1e-8; cap 500 steps; 150 GB budget; all queued at t = 0"),
           "wall_s": time.perf_counter() - t_start}
    return out


def batch_requests(n, seed=20230105):
    """The batched configuration: n lattices, case uniform over the four
    flows, D2Q21, tau uniform in [0.55, 1], speed 0.01.  Planar lattices draw
    n1 in 32..1024 and n2 in 32..2048; circular ones draw n2 in 32..2048 and
    take n1 = round(n2 / (2 pi)) (near-square cells at the inner wall, as the
    paper's polar grids)."""
    from paper_2301_01868_gb300 import serve
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        case = serve.CASES[rng.integers(4)]
        n1 = int(rng.integers(32, 1025))
        n2 = int(rng.integers(32, 2049))
        if case.startswith("circular"):
            n1 = max(8, int(round(n2 / (2.0 * math.pi))))
        out.append(serve.Request(case=case, lattice=21, n1=n1, n2=n2, tau=float(rng.uniform(0.55, 1.0)),
                                 speed=0.01, rid=k))
    return out


def batch_selection(n, select="first"):
    """The lattices of a batched record: the first n of the seeded
    configuration, or ("smallest") its n smallest of 512, to time and profile
    the small lattices' share."""
    if select == "smallest":
        return sorted(batch_requests(512), key=lambda r: r.n1 * r.n2)[:n]
    if select != "first":
        raise ValueError("select must be 'first' or 'smallest'")
    return batch_requests(n)


def batch_record(n_lattices=512, steps=5000, warmup=3, baseline_steps=20, verbose=False, select="first"):
    """The batched form against per-lattice launches on the same lattices:
    MLUPS over all lattices for `steps` timed steps after warm-up (the
    configured 5000 steps each by default), the batch's update variant from
    its autotuner, and the roofline of the batched update (168 B per cell
    update, D2Q21 FP32) from CUDA events around the timed steps (one launch
    per 4 GiB wave of lattices per time step, replayed two steps per CUDA
    graph); the per-lattice launches are timed over baseline_steps."""
    import torch
    from paper_2301_01868_gb300 import clbm, serve
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    reqs = batch_selection(n_lattices, select)
    t0 = time.perf_counter()
    grids = [serve.build_grid(r, clbm.FP32, stream) for r in reqs]
    setup_s = time.perf_counter() - t0
    cells = sum(r.n1 * r.n2 for r in reqs)
    ws = sum(clbm.workspace_bytes(21, clbm.FP32, r.n1, r.n2) for r in reqs)
    b = clbm.Batch(grids)
    best, ms = b.tune(steps=2)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b.step(warmup)
    torch.cuda.synchronize()
    l0 = b.launch_count()
    ev0.record(stream)
    b.step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_b = ev0.elapsed_time(ev1)
    l_b = b.launch_count() - l0
    b.close()
    for g in grids:
        g.step(warmup)
    torch.cuda.synchronize()
    ev0.record(stream)
    for g in grids:
        g.step(baseline_steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_l = ev0.elapsed_time(ev1)
    for g in grids:
        g.close()
    peak, peak_src = peaks()
    alg = 2 * 21 * 4 * cells
    achieved = alg / (t_b / steps * 1e-3) / 1e9
    return {"metric": "batched MLUPS (all lattices)", "unit": "MLUPS", "lattices": len(reqs),
            "cells": cells, "workspace_bytes": ws, "steps": steps, "warmup": warmup,
            "setup_s": setup_s, "tuned_variant": int(best),
            "variant_ms_per_step": list(map(float, ms)),
            "batched": {"value": cells * steps / (t_b * 1e-3) / 1e6, "ms": t_b, "launches": l_b},
            "per_lattice": {"value": cells * baseline_steps / (t_l * 1e-3) / 1e6, "ms": t_l,
                            "steps": baseline_steps, "launches": len(reqs) * baseline_steps},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_src + " (hbm_gbs)",
                         "algorithmic_bytes_per_step": alg,
                         "timed": "whole batched time step (graph replays of two steps)"},
            "config": {"workload": ("batched_%d_d2q21_fp32" if select == "first" else
                                    "batched_smallest_%d_d2q21_fp32") % len(reqs), "lattice": "D2Q21",
                       "storage": "fp32",
                       "shapes": "case uniform over the four flows; planar n1 32..1024 x n2 "
                                 "32..2048; circular n2 32..2048 with n1 = round(n2 / 2 pi) "
                                 "(near-square cells at the inner wall)",
                       "tau": "U[0.55, 1]", "steps_configured": 5000,
                       "steps_timed": steps, "waves": "one launch per 4 GiB of lattices per step"},
            "data": "synthetic"}


def run_batch(args):
    """--batch: only the batched record (args.steps timed steps), one JSON line."""
    print(json.dumps(batch_record(args.batch_lattices, args.steps, max(3, args.warmup),
                                  select=args.batch_select)))


def run_e2e(g, args, torch, stream, world, dist, cells, Q, inputs="state"):
    """Same metric through the public API with host buffers.  Every step
    uploads that step's inputs from pinned host memory, advances `chunk` time
    steps and reads the moments rho, Ut^1, Ut^2 back into pinned host memory.
    inputs "state" (the default): the full FP64 N' through the library's
    asynchronous host copies (clbm_upload_state_async / clbm_set_uploaded_state
    / clbm_download_moments_async / clbm_wait_copies): the library's copy
    stream uploads step k + 1's state and downloads step k - 1's moments
    while step k computes, so every copy stays inside the timed region but
    overlaps the update; "state_serial": the same copies one after another
    with the compute (clbm_set_state / clbm_moments with host buffers);
    "fields": the macroscopic start rho, U^1, U^2 (clbm_set_equilibrium, 3
    FP64 values per cell; fewer bytes, but the FP64 equilibrium on the device
    costs more than the saved transfer)."""
    n1, n2 = g.n1, g.n2
    names = ("rho", "Ut1", "Ut2")

    def pinned(shape):
        return torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()

    if inputs == "state":
        host_state = pinned((Q, n1, n2))
        host_state[...] = g.state()
        host_out = [{k: pinned((n1, n2)) for k in names} for _ in range(2)]

        def run(nsteps):
            g.upload_state_async(host_state)
            if nsteps > 1:
                g.upload_state_async(host_state)
            for k in range(nsteps):
                g.set_uploaded_state()
                if k + 2 < nsteps:
                    g.upload_state_async(host_state)     # overlaps this step's update
                g.step(args.chunk)
                g.download_moments_async(host_out[k % 2])   # overlaps the next update
            g.wait_copies()
        h2d = Q * cells * 8
    else:
        out = {k: pinned((n1, n2)) for k in names}
        if inputs == "state_serial":
            state_np = pinned((Q, n1, n2))
            state_np[...] = g.state()

            def upload():
                g.set_state(state_np)
            h2d = Q * cells * 8
        else:
            m = g.moments(names=("rho", "U1", "U2"))
            fields = []
            for k in ("rho", "U1", "U2"):
                f = pinned((n1, n2))
                f[...] = m[k]
                fields.append(f)

            def upload():
                g.set_equilibrium(*fields)
            h2d = 3 * cells * 8

        def run(nsteps):
            for _ in range(nsteps):
                upload()
                g.step(args.chunk)
                g.moments(names=names, out=out)

    run(1)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    run(args.steps)
    torch.cuda.synchronize()
    dt = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    what = {"state": "FP64 N' uploaded from pinned host memory by the library's copy stream while the "
                     "previous step computes (clbm_upload_state_async, clbm_set_uploaded_state)",
            "state_serial": "FP64 N' from pinned host memory through clbm_set_state, in series",
            "fields": "macroscopic start (FP64 rho, U^1, U^2 through clbm_set_equilibrium)"}[inputs]
    down = ("moments (FP64 rho, Ut^1, Ut^2) downloaded by the library's copy stream while the next "
            "step computes (clbm_download_moments_async, clbm_wait_copies)" if inputs == "state"
            else "moments (FP64 rho, Ut^1, Ut^2) through clbm_moments into pinned host memory")
    return {"value": cells * args.chunk * args.steps * world / dt / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 3 * cells * 8, "inputs": inputs,
            "note": "per step: %s, %d time steps, %s" % (what, args.chunk, down)}


if __name__ == "__main__":
    main()
