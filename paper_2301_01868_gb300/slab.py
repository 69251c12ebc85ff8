"""One lattice split into slabs along the periodic direction q^2, one slab
per rank (one GPU each), with a halo exchange after every time step.

The paper's update is local: a cell pulls each population from the cell
c_alpha behind it (Eq. 12), |c| <= 3 for D2Q21, and the wall conditions of
App. B act per column.  Cutting the periodic direction into runs of columns
therefore needs, per step and per side, only the populations that cross
the cut: D2Q21 7 at depth 1, 4 at depth 2 and 1 at depth 3 (12 strips of
the n1 + 2h stored rows), D2Q9 3.  Every slab is a grid of its own (the
geometry of planar and polar grids is the same for every column, so each
slab computes it alone: polar slabs take the ring's angular step); the
library packs and unpacks the strips (clbm_halo_pack / clbm_halo_unpack),
the ranks swap them with torch.distributed point-to-point messages (NCCL:
device buffers; gloo: through host memory), and the convergence and
conservation sums are reduced over the ranks.

Slabs whose ranks share one process (all on one GPU) exchange by device
copies instead (``SlabSet``); with one rank a slab exchanges with itself and
is the periodic grid.
"""
import math

import numpy as np

from . import clbm

_STORAGE_DTYPES = {0: "float64", 1: "float32", 2: "float16", 3: "bfloat16"}


def partition(n2, parts):
    """Column ranges [j0, j1) of `parts` slabs of n2 columns, as even as
    possible (the first n2 % parts slabs one column wider)."""
    if parts < 1 or n2 < parts:
        raise ValueError("need 1 <= parts <= n2")
    base, extra = divmod(n2, parts)
    out, j = [], 0
    for r in range(parts):
        w = base + (1 if r < extra else 0)
        out.append((j, j + w))
        j += w
    return out


def neighbours(rank, world):
    """(lower, upper) neighbour ranks on the ring of slabs."""
    return (rank - 1) % world, (rank + 1) % world


def exchange(send_lo, send_hi, recv_lo, recv_hi, rank, world, group=None):
    """Swap halo strips with the two neighbours: send_lo goes to the lower
    neighbour (its recv_hi), send_hi to the upper one (its recv_lo).  With
    one rank the slab is its own neighbour on both sides.  Buffers are
    tensors on the process group's device (CUDA for NCCL, CPU for gloo)."""
    if world == 1:
        recv_lo.copy_(send_hi)
        recv_hi.copy_(send_lo)
        return
    import torch.distributed as dist
    lo, hi = neighbours(rank, world)
    ops = [dist.P2POp(dist.isend, send_lo, lo, group), dist.P2POp(dist.irecv, recv_hi, hi, group),
           dist.P2POp(dist.isend, send_hi, hi, group), dist.P2POp(dist.irecv, recv_lo, lo, group)]
    for r in dist.batch_isend_irecv(ops):
        r.wait()


def combine_parts(parts, dt):
    """Residual and conservation values of a lattice from the summed parts
    of its slabs (clbm_residual_parts): parts = [sum J|du|^2, sum J|u|^2,
    mass, P1, P2, KE, L, max|u|, unstable cells] already reduced over the
    slabs.  Returns (res, cons[6]) as clbm_residual gives them."""
    dd, uu = parts[0], parts[1]
    if dt > 0:
        res = math.sqrt(dd) / (dt * math.sqrt(uu)) if uu > 0 else (math.inf if dd > 0 else 0.0)
    else:
        res = math.inf
    return res, np.array(parts[2:8], dtype=np.float64)


def reduce_parts(parts, rank, world, group=None, device="cpu"):
    """Sum the slabs' parts over the ranks (max for max |u|)."""
    parts = np.asarray(parts, dtype=np.float64).copy()
    if world == 1:
        return parts
    import torch
    import torch.distributed as dist
    s = torch.tensor(np.delete(parts, 7), dtype=torch.float64, device=device)
    m = torch.tensor([parts[7]], dtype=torch.float64, device=device)
    dist.all_reduce(s, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(m, op=dist.ReduceOp.MAX, group=group)
    s = s.cpu().numpy()
    return np.concatenate([s[:7], m.cpu().numpy(), s[7:]])


class Slab:
    """This rank's slab of a planar or polar lattice of n2 columns.

    Arguments as clbm.Grid, with n2 the whole lattice's column count; rank
    and world default to torch.distributed's (one rank without a process
    group).  The grid holds columns [j0, j1) of the lattice."""

    def __init__(self, lattice, n1, n2, edges, kind=clbm.PLANAR, step2=1.0, precision=clbm.FP64, dx=0.0,
                 bc_lo=clbm.NOSLIP, bc_hi=clbm.NOSLIP, device=0, stream=None, rank=None, world=None,
                 group=None):
        import torch
        import torch.distributed as dist
        if kind not in (clbm.PLANAR, clbm.POLAR):
            raise ValueError("slabs are built for planar and polar grids")
        if rank is None or world is None:
            on = dist.is_available() and dist.is_initialized()
            rank = dist.get_rank(group) if on else 0
            world = dist.get_world_size(group) if on else 1
        self.rank, self.world, self.group = rank, world, group
        self.n2_total = int(n2)
        self.j0, self.j1 = partition(self.n2_total, world)[rank]
        if isinstance(precision, str):
            precision = clbm.PRECISIONS[precision]
        self.grid = clbm.Grid(lattice, n1, self.j1 - self.j0, edges, kind=kind, step2=step2,
                              precision=precision, dx=dx, bc_lo=bc_lo, bc_hi=bc_hi, device=device,
                              stream=stream, n2_period=self.n2_total)
        g = self.grid
        n = g.halo_values()
        dt = getattr(torch, _STORAGE_DTYPES[g.precision])
        self.bufs = [torch.empty(n, dtype=dt, device=g.device) for _ in range(4)]
        self.torch = torch

    # ------------------------------------------------------------- exchange
    def _backend(self):
        """The process group's backend ("" with one rank and no group)."""
        if self.world == 1:
            return ""
        import torch.distributed as dist
        return dist.get_backend(self.group)

    def _host_staged(self):
        """Whether the strips travel through host memory (a gloo group)."""
        return self._backend() == "gloo"

    def _exchange(self):
        g, (s_lo, s_hi, r_lo, r_hi) = self.grid, self.bufs
        g.halo_pack(0, s_lo)
        g.halo_pack(1, s_hi)
        g.stream.synchronize()
        if self._host_staged():
            # bytes, whatever the storage type: the values move bit for bit
            h = [b.view(self.torch.uint8).cpu() for b in (s_lo, s_hi, r_lo, r_hi)]
            exchange(h[0], h[1], h[2], h[3], self.rank, self.world, self.group)
            r_lo.view(self.torch.uint8).copy_(h[2])
            r_hi.view(self.torch.uint8).copy_(h[3])
        else:
            exchange(s_lo, s_hi, r_lo, r_hi, self.rank, self.world, self.group)
        self.torch.cuda.current_stream(g.device).synchronize()
        g.halo_unpack(0, r_lo)
        g.halo_unpack(1, r_hi)

    def set_case(self, *args, **kw):
        self.grid.set_case(*args, **kw)
        self.grid.fill_ghosts()
        self._exchange()

    def set_state(self, Np_local, rho_prev=None, ut2_prev=None):
        """This slab's columns of N'(q, t-1), (Q, n1, j1 - j0)."""
        self.grid.set_state(Np_local, rho_prev, ut2_prev)
        self.grid.fill_ghosts()
        self._exchange()

    def step(self, n=1):
        for _ in range(int(n)):
            self.grid.step(1)
            self._exchange()

    # ---------------------------------------------------------- diagnostics
    def residual(self):
        """(res, cons) of the whole lattice (collective over the ranks)."""
        parts, dt = self.grid.residual_parts()
        # NCCL reduces device tensors, gloo host ones
        dev = self.grid.device if self._backend() == "nccl" else "cpu"
        tot = reduce_parts(parts, self.rank, self.world, self.group, device=dev)
        return combine_parts(tot, dt)

    def moments(self, **kw):
        """Moments of this slab's columns."""
        return self.grid.moments(**kw)

    def state(self):
        return self.grid.state()

    def close(self):
        self.grid.close()


class SlabSet:
    """Every slab of one lattice in this process, all on one device: the same
    slabs and strips, with the exchange done by device copies between the
    slabs' buffers.  A one-GPU check of the slab path (the kernels of the
    slabs never wait on each other: the host orders every launch)."""

    def __init__(self, parts, lattice, n1, n2, edges, **kw):
        import torch
        self.torch = torch
        stream = kw.pop("stream", None) or torch.cuda.Stream()
        self.slabs = [Slab(lattice, n1, n2, edges, rank=r, world=parts, stream=stream, **kw)
                      for r in range(parts)]
        self.stream = stream

    def _exchange(self):
        S = self.slabs
        for s in S:
            s.grid.halo_pack(0, s.bufs[0])
            s.grid.halo_pack(1, s.bufs[1])
        with self.torch.cuda.stream(self.stream):
            for r, s in enumerate(S):
                lo, hi = S[(r - 1) % len(S)], S[(r + 1) % len(S)]
                s.bufs[2].copy_(lo.bufs[1])      # from the lower neighbour's upper side
                s.bufs[3].copy_(hi.bufs[0])      # from the upper neighbour's lower side
        for s in S:
            s.grid.halo_unpack(0, s.bufs[2])
            s.grid.halo_unpack(1, s.bufs[3])

    def set_case(self, *args, **kw):
        for s in self.slabs:
            s.grid.set_case(*args, **kw)
            s.grid.fill_ghosts()
        self._exchange()

    def set_state(self, Np):
        """N'(q, t-1) of the whole lattice, (Q, n1, n2): each slab takes its columns."""
        for s in self.slabs:
            s.grid.set_state(np.ascontiguousarray(Np[:, :, s.j0:s.j1]))
            s.grid.fill_ghosts()
        self._exchange()

    def step(self, n=1):
        for _ in range(int(n)):
            for s in self.slabs:
                s.grid.step(1)
            self._exchange()

    def state(self):
        return np.concatenate([s.grid.state() for s in self.slabs], axis=2)

    def moments(self, names=("rho", "Ut1", "Ut2")):
        ms = [s.grid.moments(names=names) for s in self.slabs]
        return {k: np.concatenate([m[k] for m in ms], axis=1) for k in names}

    def residual(self):
        got = [s.grid.residual_parts() for s in self.slabs]
        parts = np.sum([p for p, _ in got], axis=0)
        parts[7] = max(p[7] for p, _ in got)
        return combine_parts(parts, got[0][1])

    def close(self):
        for s in self.slabs:
            s.close()
