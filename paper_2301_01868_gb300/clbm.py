"""Python binding of ``libclbm.so`` (the C ABI in include/clbm.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch supplies device memory (the grid workspace and device
outputs) and the CUDA stream.  If the library is missing the import fails;
there is no CPU fallback.
"""
import ctypes as C
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libclbm.so")

D2Q9, D2Q21 = 9, 21
FP64, FP32, FP32_F16STORE, FP32_BF16STORE = 0, 1, 2, 3
PLANAR, POLAR, GENERAL = 0, 1, 2
NOSLIP, MOVING = 0, 1
PRECISIONS = {"fp64": FP64, "fp32": FP32, "fp16": FP32_F16STORE, "bf16": FP32_BF16STORE}
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EUNSTABLE", 5: "ETIMEOUT", 6: "EBUSY"}


class ClbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class UnstableError(ClbmError):
    pass


class _Desc(C.Structure):
    _fields_ = [("lattice", C.c_int), ("precision", C.c_int), ("n1", C.c_int), ("n2", C.c_int),
                ("kind", C.c_int), ("edges1", C.POINTER(C.c_double)), ("step2", C.c_double),
                ("dx", C.c_double), ("bc_lo", C.c_int), ("bc_hi", C.c_int), ("device", C.c_int),
                ("stream", C.c_void_p), ("workspace", C.c_void_p), ("workspace_bytes", C.c_size_t),
                ("nodes", C.POINTER(C.c_double)), ("n2_period", C.c_int)]


class _Case(C.Structure):
    _fields_ = [("tau", C.c_double), ("rho0", C.c_double), ("u_wall_lo", C.c_double),
                ("u_wall_hi", C.c_double), ("g_ext", C.c_double * 2), ("force_iterations", C.c_int)]


_lib = None


class _Desc3(C.Structure):
    _fields_ = [("precision", C.c_int), ("n1", C.c_int), ("n2", C.c_int), ("n3", C.c_int),
                ("kind", C.c_int), ("edges", C.POINTER(C.c_double)), ("step2", C.c_double),
                ("step3", C.c_double), ("dx", C.c_double), ("bc_lo", C.c_int), ("bc_hi", C.c_int),
                ("device", C.c_int), ("stream", C.c_void_p)]


class _Case3(C.Structure):
    _fields_ = [("tau", C.c_double), ("rho0", C.c_double), ("u_wall_lo", C.c_double),
                ("u_wall_hi", C.c_double), ("g_ext", C.c_double * 3)]


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError("libclbm.so is not built; run __graft_entry__.build() "
                              "(paper_2301_01868_gb300/_build.py) on a machine with nvcc")
        L = C.CDLL(_LIB_PATH)
        dp, vp, ll = C.POINTER(C.c_double), C.c_void_p, C.c_longlong
        h = C.c_void_p
        sig = {
            "clbm_workspace_bytes": [C.POINTER(_Desc), C.POINTER(C.c_size_t)],
            "clbm_create_grid": [C.POINTER(_Desc), C.POINTER(C.c_void_p)],
            "clbm_set_case": [h, C.POINTER(_Case)],
            "clbm_set_state": [h, vp, vp, vp, C.c_int],
            "clbm_get_state": [h, vp, C.c_int],
            "clbm_set_equilibrium": [h, vp, vp, vp, C.c_int],
            "clbm_step": [h, ll],
            "clbm_moments": [h, vp, vp, vp, vp, vp, vp, vp, C.c_int],
            "clbm_residual": [h, dp, dp],
            "clbm_upload_state_async": [h, vp],
            "clbm_set_uploaded_state": [h],
            "clbm_download_moments_async": [h, vp, vp, vp],
            "clbm_wait_copies": [h],
            "clbm_residual_parts": [h, dp, C.POINTER(ll)],
            "clbm_fill_ghosts": [h],
            "clbm_halo_values": [h, C.POINTER(C.c_size_t)],
            "clbm_halo_pack": [h, C.c_int, vp],
            "clbm_halo_unpack": [h, C.c_int, vp],
            "clbm_no_flow_adjust": [h, ll, vp],
            "clbm_time": [h, C.POINTER(ll)],
            "clbm_set_stream": [h, vp],
            "clbm_set_profiling": [h, C.c_int],
            "clbm_kernel_time": [h, dp, C.POINTER(ll)],
            "clbm_launch_count": [h, C.POINTER(ll)],
            "clbm_set_kernel": [h, C.c_int],
            "clbm_checkpoint_bytes": [h, C.POINTER(C.c_size_t)],
            "clbm_checkpoint": [h, vp],
            "clbm_restore": [h, vp],
            "clbm_batch_create": [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_void_p)],
            "clbm_batch_step": [h, ll],
            "clbm_batch_residual": [h, vp, vp],
            "clbm_batch_set_variant": [h, C.c_int],
            "clbm_batch_tune": [h, C.c_int, C.POINTER(C.c_int), vp],
            "clbm_batch_get_variant": [h, C.POINTER(C.c_int), C.POINTER(C.c_int)],
            "clbm_batch_set_wave_bytes": [h, C.c_size_t],
            "clbm_batch_launch_count": [h, C.POINTER(ll)],
            "clbm_batch_destroy": [h],
            "clbm_destroy": [h],
            "clbm_selftest_bounded_wait": [C.c_int, C.c_int, dp],
            "clbm3_create_grid": [C.POINTER(_Desc3), C.POINTER(C.c_void_p)],
            "clbm3_set_case": [h, C.POINTER(_Case3)],
            "clbm3_set_state": [h, vp, vp, vp, vp, C.c_int],
            "clbm3_get_state": [h, vp, C.c_int],
            "clbm3_step": [h, ll],
            "clbm3_moments": [h, vp, vp, C.c_int],
            "clbm3_totals": [h, dp],
            "clbm3_time": [h, C.POINTER(ll)],
            "clbm3_set_kernel": [h, C.c_int],
            "clbm3_set_equilibrium": [h, vp, vp, C.c_int],
            "clbm3_checkpoint_bytes": [h, C.POINTER(C.c_size_t)],
            "clbm3_checkpoint": [h, vp],
            "clbm3_restore": [h, vp],
            "clbm3_destroy": [h],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.clbm_last_error.restype = C.c_char_p
        L.clbm_last_error.argtypes = []
        _lib = L
    return _lib


def _check(st):
    if st != 0:
        msg = lib().clbm_last_error().decode()
        if st == 4:
            raise UnstableError(st, msg)
        raise ClbmError(st, msg)


def _ptr(x):
    """Address of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _is_device(x):
    return x is not None and not isinstance(x, np.ndarray) and x.is_cuda


def _desc(lattice, precision, n1, n2, kind, edges, step2, dx, bc_lo, bc_hi, device, stream, nodes=None,
          n2_period=0):
    dp = C.POINTER(C.c_double)
    if kind == GENERAL:
        P = np.ascontiguousarray(nodes, dtype=np.float64)
        if P.shape != (n1 + 8, n2 + 8, 2):
            raise ValueError("nodes must be (n1+8, n2+8, 2)")
        d = _Desc(lattice, precision, n1, n2, kind, None, float(step2), float(dx), bc_lo, bc_hi,
                  device, stream, None, 0, P.ctypes.data_as(dp))
        return d, P
    e = np.ascontiguousarray(edges, dtype=np.float64)
    if e.shape != (n1 + 1,):
        raise ValueError("edges must have n1+1 entries")
    d = _Desc(lattice, precision, n1, n2, kind, e.ctypes.data_as(dp), float(step2), float(dx), bc_lo,
              bc_hi, device, stream, None, 0, None, int(n2_period))
    return d, e


def workspace_bytes(lattice, precision, n1, n2, kind=PLANAR):
    """Device bytes a grid of this size needs (general grids hold per-cell
    geometry and tables)."""
    e = np.arange(n1 + 1, dtype=np.float64) + 1.0
    nodes = np.zeros((n1 + 8, n2 + 8, 2)) if kind == GENERAL else None
    d, _ = _desc(lattice, precision, n1, n2, kind, e, 1.0, 1.0, 0, 0, 0, None, nodes)
    out = C.c_size_t()
    _check(lib().clbm_workspace_bytes(C.byref(d), C.byref(out)))
    return out.value


class Grid:
    """A lattice advanced on one GPU by the fused curvilinear LBM update.

    edges  : n1+1 wall-normal cell edges (radii for POLAR); None for GENERAL.
    step2  : q^2 step of PLANAR grids.
    nodes  : GENERAL grids: node positions (n1+8, n2+8, 2) of nodes i = -3..n1+4,
             j = -3..n2+4 at q = (i - 1/2, j - 1/2), ghosts and periodic images
             included (clbm_inputs.mapped_nodes builds them); dx > 0 required.
    precision : FP64, FP32, FP32_F16STORE or FP32_BF16STORE (or "fp64", ...).
    The device workspace is a torch uint8 tensor; work goes on torch's
    current stream of `device` unless `stream` (a torch.cuda.Stream) is given.
    """

    def __init__(self, lattice, n1, n2, edges, kind=PLANAR, step2=1.0, precision=FP64, dx=0.0,
                 bc_lo=NOSLIP, bc_hi=NOSLIP, device=0, stream=None, nodes=None, n2_period=0):
        import torch

        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        self.Q, self.n1, self.n2 = int(lattice), int(n1), int(n2)
        self.precision, self.kind = int(precision), int(kind)
        self.device = torch.device("cuda", device)
        self._torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        d, self._edges = _desc(self.Q, self.precision, self.n1, self.n2, self.kind, edges, step2, dx,
                               int(bc_lo), int(bc_hi), self.device.index, self.stream.cuda_stream,
                               nodes, n2_period)
        nb = C.c_size_t()
        _check(lib().clbm_workspace_bytes(C.byref(d), C.byref(nb)))
        self.workspace = torch.empty(nb.value, dtype=torch.uint8, device=self.device)
        d.workspace = self.workspace.data_ptr()
        d.workspace_bytes = nb.value
        h = C.c_void_p()
        _check(lib().clbm_create_grid(C.byref(d), C.byref(h)))
        self._h = h

    # lifetime ----------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().clbm_destroy(self._h)
            self._h = None
            self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # case and state ----------------------------------------------------------
    def set_case(self, tau, rho0=1.0, u_wall_lo=0.0, u_wall_hi=0.0, g_ext=(0.0, 0.0),
                 force_iterations=0):
        c = _Case(float(tau), float(rho0), float(u_wall_lo), float(u_wall_hi),
                  (C.c_double * 2)(float(g_ext[0]), float(g_ext[1])), int(force_iterations))
        _check(lib().clbm_set_case(self._h, C.byref(c)))

    def set_state(self, Np, rho_prev=None, ut2_prev=None):
        """N'(q, t-1) as (Q, n1, n2) float64, numpy (host) or torch (either)."""
        dev = _is_device(Np)
        arrs = []
        for x in (Np, rho_prev, ut2_prev):
            if x is None:
                arrs.append(None)
            elif dev:
                arrs.append(x.to(self._torch.float64).contiguous())
            else:
                x = x.cpu().numpy() if hasattr(x, "cpu") else x
                arrs.append(np.ascontiguousarray(x, dtype=np.float64))
        if arrs[0].shape != (self.Q, self.n1, self.n2):
            raise ValueError("state must be (Q, n1, n2)")
        _check(lib().clbm_set_state(self._h, _ptr(arrs[0]), _ptr(arrs[1]), _ptr(arrs[2]), int(dev)))

    def set_equilibrium(self, rho=None, U1=None, U2=None):
        """Start from J f^eq(rho, U, Ut = U) (Eq. 19) of the given fields:
        contravariant U^1, U^2 and rho, each (n1, n2) or broadcastable to it
        (e.g. an (n1, 1) wall-normal profile), numpy (host) or torch (either);
        None gives rho0 / 0.  t restarts at 0."""
        xs = [x for x in (rho, U1, U2) if x is not None]
        dev = bool(xs) and _is_device(xs[0])
        if any(_is_device(x) != dev for x in xs):
            raise ValueError("rho, U1, U2 must all be on the host or all on the device")
        arrs = []
        for x in (rho, U1, U2):
            if x is None:
                arrs.append(None)
            elif dev:
                arrs.append(x.to(self._torch.float64).expand(self.n1, self.n2).contiguous())
            else:
                x = x.cpu().numpy() if hasattr(x, "cpu") else x
                arrs.append(np.ascontiguousarray(np.broadcast_to(np.asarray(x, dtype=np.float64),
                                                                 (self.n1, self.n2))))
        _check(lib().clbm_set_equilibrium(self._h, _ptr(arrs[0]), _ptr(arrs[1]), _ptr(arrs[2]),
                                          int(dev)))

    def state(self, device=False):
        """N'(q, t-1) as float64 (Q, n1, n2): numpy, or a torch CUDA tensor."""
        if device:
            out = self._torch.empty((self.Q, self.n1, self.n2), dtype=self._torch.float64,
                                    device=self.device)
        else:
            out = np.empty((self.Q, self.n1, self.n2))
        _check(lib().clbm_get_state(self._h, _ptr(out), int(device)))
        return out

    def step(self, n=1):
        _check(lib().clbm_step(self._h, int(n)))

    def checkpoint(self):
        """The case and dynamic state (raw state buffer, wall moments, residual
        snapshot, geometry, time) as bytes; restore() continues from it bit
        for bit."""
        n = C.c_size_t()
        _check(lib().clbm_checkpoint_bytes(self._h, C.byref(n)))
        buf = np.empty(n.value, dtype=np.uint8)
        _check(lib().clbm_checkpoint(self._h, buf.ctypes.data))
        return buf.tobytes()

    def restore(self, blob):
        """Load a checkpoint() of a grid with the same description."""
        buf = np.frombuffer(blob, dtype=np.uint8)
        n = C.c_size_t()
        _check(lib().clbm_checkpoint_bytes(self._h, C.byref(n)))
        if buf.size != n.value:
            raise ClbmError(1, "checkpoint is %d bytes, this grid's are %d" % (buf.size, n.value))
        _check(lib().clbm_restore(self._h, buf.ctypes.data))

    @property
    def t(self):
        v = C.c_longlong()
        _check(lib().clbm_time(self._h, C.byref(v)))
        return v.value

    # diagnostics --------------------------------------------------------------
    def moments(self, device=False, names=("rho", "U1", "U2", "Ut1", "Ut2", "F1", "F2"), out=None):
        """Moments of the current state (what the next collision uses).  out:
        optional dict of preallocated (n1, n2) float64 arrays (host, e.g. views
        of pinned memory, or device tensors when device=True) to fill."""
        all_names = ("rho", "U1", "U2", "Ut1", "Ut2", "F1", "F2")
        out = dict(out) if out else {}
        for k in names:
            if k in out:
                continue
            if device:
                out[k] = self._torch.empty((self.n1, self.n2), dtype=self._torch.float64,
                                           device=self.device)
            else:
                out[k] = np.empty((self.n1, self.n2))
        ptrs = [_ptr(out.get(k)) for k in all_names]
        _check(lib().clbm_moments(self._h, *ptrs, int(device)))
        return out

    # asynchronous host copies -----------------------------------------------
    def upload_state_async(self, Np):
        """Start copying N'(q, t-1) (float64 (Q, n1, n2) in host memory, best
        page-locked) into one of the grid's two upload slots on its copy
        stream; returns at once.  The array must stay alive and unchanged
        until set_uploaded_state() has been called for it and the grid's
        stream has passed that point (e.g. wait_copies() or the next
        synchronising call)."""
        arr = Np.numpy() if hasattr(Np, "numpy") else Np
        if arr.shape != (self.Q, self.n1, self.n2) or arr.dtype != np.float64 or not arr.flags.c_contiguous:
            raise ValueError("state must be a contiguous float64 (Q, n1, n2) host array")
        _check(lib().clbm_upload_state_async(self._h, arr.ctypes.data))

    def set_uploaded_state(self):
        """Make the oldest upload the grid's state (on the grid's stream, after
        its copy; no host wait), as set_state would."""
        _check(lib().clbm_set_uploaded_state(self._h))

    def download_moments_async(self, out):
        """Compute rho, Ut1, Ut2 of the current state on the grid's stream and
        copy them on the copy stream into out's float64 (n1, n2) host arrays
        (keys rho, Ut1, Ut2, any may be missing; best page-locked); returns at
        once.  wait_copies() blocks until they have landed."""
        ptrs = []
        for k in ("rho", "Ut1", "Ut2"):
            a = out.get(k)
            if a is not None:
                a = a.numpy() if hasattr(a, "numpy") else a
                if a.shape != (self.n1, self.n2) or a.dtype != np.float64 or not a.flags.c_contiguous:
                    raise ValueError("%s must be a contiguous float64 (n1, n2) host array" % k)
                ptrs.append(a.ctypes.data)
            else:
                ptrs.append(None)
        _check(lib().clbm_download_moments_async(self._h, *ptrs))

    def wait_copies(self):
        """Block until every asynchronous copy issued so far has landed."""
        _check(lib().clbm_wait_copies(self._h))

    def residual(self):
        """(res, cons): cons = mass, P1, P2, kinetic energy, angular momentum, max|u|."""
        r = C.c_double()
        cons = (C.c_double * 6)()
        _check(lib().clbm_residual(self._h, C.byref(r), cons))
        return r.value, np.array(list(cons))

    def residual_parts(self):
        """(parts[9], dt): the sums behind residual() (clbm_residual_parts)."""
        parts = (C.c_double * 9)()
        dt = C.c_longlong()
        st = lib().clbm_residual_parts(self._h, parts, C.byref(dt))
        if st != 4:
            _check(st)
        return np.array(list(parts)), dt.value

    # slabs along q^2 (slab.py drives these) ----------------------------------
    def fill_ghosts(self):
        _check(lib().clbm_fill_ghosts(self._h))

    def halo_values(self):
        n = C.c_size_t()
        _check(lib().clbm_halo_values(self._h, C.byref(n)))
        return n.value

    def halo_pack(self, side, buf):
        """Pack side 0 (for the lower neighbour) or 1 into a device tensor of
        halo_values() storage-type values."""
        _check(lib().clbm_halo_pack(self._h, int(side), _ptr(buf)))

    def halo_unpack(self, side, buf):
        _check(lib().clbm_halo_unpack(self._h, int(side), _ptr(buf)))

    def no_flow_adjust(self, nsteps):
        rho_nf = np.empty((self.n1, self.n2))
        _check(lib().clbm_no_flow_adjust(self._h, int(nsteps), rho_nf.ctypes.data))
        return rho_nf

    def set_profiling(self, on=True, period=1):
        """Time every period-th update launch with CUDA events (on=False: stop)."""
        _check(lib().clbm_set_profiling(self._h, int(period) if on else 0))

    def kernel_time(self):
        """(ms, launches) of the fused update since profiling was switched on."""
        ms = C.c_double()
        n = C.c_longlong()
        _check(lib().clbm_kernel_time(self._h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def set_kernel(self, variant):
        """0 automatic, 1 one thread per cell, 2 TMA-staged tiles with a shared
        output tile, 3 TMA-staged warp-specialised pipeline, 4 the pipeline
        with two cells per thread, 5 / 6 kernels 3 / 4 with many time steps
        per launch (clbm.h)."""
        _check(lib().clbm_set_kernel(self._h, int(variant)))

    def launch_count(self):
        n = C.c_longlong()
        _check(lib().clbm_launch_count(self._h, C.byref(n)))
        return n.value


class Batch:
    """Several grids (same lattice, precision and device) advanced together by
    one persistent launch per phase, two steps per CUDA graph.  The grids stay
    owned by the caller and must outlive the batch."""

    VARIANTS = 5

    def __init__(self, grids):
        self.grids = list(grids)
        arr = (C.c_void_p * len(self.grids))(*[g._h.value for g in self.grids])
        h = C.c_void_p()
        _check(lib().clbm_batch_create(arr, len(self.grids), C.byref(h)))
        self._h = h

    def step(self, n=1):
        _check(lib().clbm_batch_step(self._h, int(n)))

    def residual(self):
        """(res[n], cons[n, 6]) for every grid, as clbm_residual gives them;
        res[k] is NaN for a grid that went unstable (the others stay valid)."""
        n = len(self.grids)
        res = np.empty(n)
        cons = np.empty((n, 6))
        st = lib().clbm_batch_residual(self._h, res.ctypes.data, cons.ctypes.data)
        if st != 4:
            _check(st)
        return res, cons

    def set_variant(self, v):
        """0-3: one thread per cell with tiles 128x1, 256x1 (2 per thread),
        32x4, 64x1; 4: the pipelined TMA update over 64x8 tiles."""
        _check(lib().clbm_batch_set_variant(self._h, int(v)))

    def tune(self, steps=5):
        """Time every tile variant on this batch; keeps and returns the fastest."""
        best = C.c_int()
        ms = np.empty(self.VARIANTS)
        _check(lib().clbm_batch_tune(self._h, int(steps), C.byref(best), ms.ctypes.data))
        return best.value, ms

    def set_wave_bytes(self, nbytes):
        """Run each time step as one launch per wave of consecutive lattices
        holding at most nbytes of workspace (4 GiB by default)."""
        _check(lib().clbm_batch_set_wave_bytes(self._h, int(nbytes)))

    def variant(self):
        """(variant, cached): the update variant and whether it came from the
        tuner's cache of this process when the batch was created."""
        v = C.c_int()
        cached = C.c_int()
        _check(lib().clbm_batch_get_variant(self._h, C.byref(v), C.byref(cached)))
        return v.value, bool(cached.value)

    def launch_count(self):
        n = C.c_longlong()
        _check(lib().clbm_batch_launch_count(self._h, C.byref(n)))
        return n.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().clbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wall_speed_planar(u_phys, step2, dx):
    """Contravariant U0^2 of a planar wall moving at physical speed u_phys
    (|g_2| = step2 / dx)."""
    return u_phys * dx / step2


def wall_speed_polar(u_phys, R_wall, n2, dx):
    """Contravariant U0^2 of a rigidly rotating circle of radius R_wall with
    surface speed u_phys (|g_2| = R sin(2 pi / n2) / dx, App. D)."""
    return u_phys * dx / (R_wall * math.sin(2.0 * math.pi / n2))


CHANNEL3, ANNULUS3 = 0, 1


class Grid3:
    """A three-dimensional lattice (D3Q39, clbm3.h) on one GPU: q^1 wall-normal
    between two walls, q^2 and q^3 periodic.  kind CHANNEL3 (edges along q^1,
    uniform q^2 / q^3 spacings) or ANNULUS3 (radial edges, n2 angular nodes,
    axial spacing step3).  precision FP64 or FP32.  Populations are float64
    (39, n1, n2, n3) arrays of N'(q, t-1)."""

    Q = 39

    def __init__(self, n1, n2, n3, edges, kind=CHANNEL3, step2=1.0, step3=1.0, precision=FP64, dx=0.0,
                 bc_lo=NOSLIP, bc_hi=NOSLIP, device=0, stream=None):
        import torch

        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        self.n1, self.n2, self.n3 = int(n1), int(n2), int(n3)
        self.device = torch.device("cuda", device)
        self._torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._edges = np.ascontiguousarray(edges, dtype=np.float64)
        if self._edges.shape != (self.n1 + 1,):
            raise ValueError("edges must have n1 + 1 entries")
        d = _Desc3(int(precision), self.n1, self.n2, self.n3, int(kind),
                   self._edges.ctypes.data_as(C.POINTER(C.c_double)), float(step2), float(step3),
                   float(dx), int(bc_lo), int(bc_hi), self.device.index, self.stream.cuda_stream)
        h = C.c_void_p()
        _check(lib().clbm3_create_grid(C.byref(d), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().clbm3_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (self.n1, self.n2, self.n3)

    def set_case(self, tau, rho0=1.0, u_wall_lo=0.0, u_wall_hi=0.0, g_ext=(0.0, 0.0, 0.0)):
        c = _Case3(float(tau), float(rho0), float(u_wall_lo), float(u_wall_hi),
                   (C.c_double * 3)(*[float(x) for x in g_ext]))
        _check(lib().clbm3_set_case(self._h, C.byref(c)))

    def set_state(self, Np, rho_prev=None, ut2_prev=None, ut3_prev=None):
        dev = _is_device(Np)
        arrs = []
        for x in (Np, rho_prev, ut2_prev, ut3_prev):
            if x is None:
                arrs.append(None)
            elif dev:
                arrs.append(x.to(self._torch.float64).contiguous())
            else:
                x = x.cpu().numpy() if hasattr(x, "cpu") else x
                arrs.append(np.ascontiguousarray(x, dtype=np.float64))
        if tuple(arrs[0].shape) != (self.Q,) + self.shape:
            raise ValueError("state must be (39, n1, n2, n3)")
        _check(lib().clbm3_set_state(self._h, *[_ptr(a) for a in arrs], int(dev)))

    def state(self, device=False):
        sh = (self.Q,) + self.shape
        out = (self._torch.empty(sh, dtype=self._torch.float64, device=self.device) if device
               else np.empty(sh))
        _check(lib().clbm3_get_state(self._h, _ptr(out), int(device)))
        return out

    def step(self, n=1):
        _check(lib().clbm3_step(self._h, int(n)))

    def set_equilibrium(self, rho=None, U=None):
        """Start from J f^eq(rho, U, Ut = U) (Eq. 19): rho (n1, n2, n3) and
        contravariant U (3, n1, n2, n3), float64 numpy (None: rho0 / 0)."""
        arrs = [None if x is None else np.ascontiguousarray(x, dtype=np.float64) for x in (rho, U)]
        if arrs[0] is not None and arrs[0].shape != self.shape:
            raise ValueError("rho must be (n1, n2, n3)")
        if arrs[1] is not None and arrs[1].shape != (3,) + self.shape:
            raise ValueError("U must be (3, n1, n2, n3)")
        _check(lib().clbm3_set_equilibrium(self._h, _ptr(arrs[0]), _ptr(arrs[1]), 0))

    def checkpoint(self):
        """Case, time, raw state and wall moments as bytes (restore() resumes bit for bit)."""
        n = C.c_size_t()
        _check(lib().clbm3_checkpoint_bytes(self._h, C.byref(n)))
        buf = np.empty(n.value, dtype=np.uint8)
        _check(lib().clbm3_checkpoint(self._h, buf.ctypes.data))
        return buf.tobytes()

    def restore(self, blob):
        buf = np.frombuffer(blob, dtype=np.uint8)
        n = C.c_size_t()
        _check(lib().clbm3_checkpoint_bytes(self._h, C.byref(n)))
        if buf.size != n.value:
            raise ClbmError(1, "checkpoint is %d bytes, this grid's are %d" % (buf.size, n.value))
        _check(lib().clbm3_restore(self._h, buf.ctypes.data))

    def moments(self):
        """dict: rho (n1, n2, n3) and Ut (3, n1, n2, n3), float64 numpy."""
        rho = np.empty(self.shape)
        ut = np.empty((3,) + self.shape)
        _check(lib().clbm3_moments(self._h, rho.ctypes.data, ut.ctypes.data, 0))
        return {"rho": rho, "Ut": ut}

    def totals(self):
        """(mass, momentum[3]) of the current state: sum N', sum c N'."""
        out = (C.c_double * 4)()
        _check(lib().clbm3_totals(self._h, out))
        return np.array(list(out))

    def set_kernel(self, kernel):
        """Update kernel: 0 automatic, 1 pulled populations in registers, 2 in
        shared memory (FP32 compute only; the automatic choice there)."""
        _check(lib().clbm3_set_kernel(self._h, int(kernel)))

    @property
    def t(self):
        v = C.c_longlong()
        _check(lib().clbm3_time(self._h, C.byref(v)))
        return v.value


def selftest_bounded_wait(polls=4096, device=0):
    """(status, ms) of the bounded-wait self-test: status must be ETIMEOUT (4)."""
    ms = C.c_double()
    st = lib().clbm_selftest_bounded_wait(int(device), int(polls), C.byref(ms))
    return st, ms.value
