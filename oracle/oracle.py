"""ctypes front end of the plain FP64 C oracle (``clbm_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
cpu_baseline / reference leg of ``bench.py`` may import this module.  It does
not import the CUDA library and the CUDA library does not import it.

Array conventions: populations are float64 numpy arrays of shape (Q, n1, n2)
holding N'(q, t-1); cell fields are (n1, n2).  Row i is wall-normal (q^1), the
column j periodic (q^2), as in App. B of the paper.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

PLANAR, POLAR, GENERAL = 0, 1, 2
NOSLIP, MOVING = 0, 1

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        L.orc_lattice.argtypes = [C.c_int, ip, dp, ip, ip, dp]
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, dp, C.c_double,
                                 dp, C.c_double, C.c_int, C.c_int]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_set_case.argtypes = [C.c_void_p] + [C.c_double] * 6
        L.orc_init_rest.argtypes = [C.c_void_p]
        L.orc_set_state.argtypes = [C.c_void_p, dp, dp, dp]
        L.orc_get_state.argtypes = [C.c_void_p, dp]
        L.orc_get_prev_moments.argtypes = [C.c_void_p, dp, dp]
        L.orc_step.argtypes = [C.c_void_p, C.c_longlong]
        L.orc_time.restype = C.c_longlong
        L.orc_time.argtypes = [C.c_void_p]
        L.orc_moments.argtypes = [C.c_void_p] + [dp] * 7
        L.orc_collide_one.argtypes = [C.c_void_p, C.c_int, C.c_int] + [dp] * 8
        L.orc_node_geometry.restype = C.c_int
        L.orc_node_geometry.argtypes = [C.c_void_p, C.c_int, C.c_int, dp]
        L.orc_theta.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, dp]
        L.orc_feq.restype = C.c_double
        L.orc_feq.argtypes = [C.c_void_p, C.c_int, C.c_double, dp, dp, dp]
        L.orc_totals.argtypes = [C.c_void_p, dp]
        L.orc_flow_diagnostics.argtypes = [C.c_void_p] + [dp] * 5 + [C.c_longlong, dp]
        L.orc_get_volume.argtypes = [C.c_void_p, dp]
        L.orc_set_volume.argtypes = [C.c_void_p, dp]
        L.orc_no_flow_adjust.argtypes = [C.c_void_p, C.c_longlong, dp]
        L.orc_set_force_iterations.argtypes = [C.c_void_p, C.c_int]
        L.orc_threads.restype = C.c_int
        _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def lattice(Q):
    """(c[Q,2] int, w[Q], star[Q], hat[Q], T0) exactly as the oracle holds them."""
    c = np.zeros((Q, 2), dtype=np.int32)
    w = np.zeros(Q)
    star = np.zeros(Q, dtype=np.int32)
    hat = np.zeros(Q, dtype=np.int32)
    T0 = C.c_double()
    rc = lib().orc_lattice(Q, c.ctypes.data_as(C.POINTER(C.c_int)), _p(w),
                           star.ctypes.data_as(C.POINTER(C.c_int)),
                           hat.ctypes.data_as(C.POINTER(C.c_int)), C.byref(T0))
    if rc != 0:
        raise ValueError("Q must be 9 or 21")
    return c.astype(np.int64), w, star.astype(np.int64), hat.astype(np.int64), T0.value


class Grid:
    """One lattice held by the oracle."""

    def __init__(self, Q, n1, n2, kind=PLANAR, edges=None, step2=1.0, nodes=None,
                 dx=0.0, bc_lo=NOSLIP, bc_hi=NOSLIP):
        self.Q, self.n1, self.n2 = int(Q), int(n1), int(n2)
        e = None if edges is None else np.ascontiguousarray(edges, dtype=np.float64)
        nd = None if nodes is None else np.ascontiguousarray(nodes, dtype=np.float64)
        if e is not None and e.shape != (n1 + 1,):
            raise ValueError("edges must have n1+1 entries")
        if nd is not None and nd.shape != (n1 + 8, n2 + 8, 2):
            raise ValueError("nodes must be (n1+8, n2+8, 2)")
        self._keep = (e, nd)
        h = lib().orc_create(self.Q, self.n1, self.n2, int(kind), _p(e), float(step2),
                             _p(nd), float(dx), int(bc_lo), int(bc_hi))
        if not h:
            raise ValueError("oracle rejected the grid description")
        self._h = C.c_void_p(h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.orc_destroy(h)
            self._h = None

    # case and state -------------------------------------------------------
    def set_case(self, tau, rho0=1.0, U0_lo=0.0, U0_hi=0.0, gext=(0.0, 0.0)):
        lib().orc_set_case(self._h, tau, rho0, U0_lo, U0_hi, gext[0], gext[1])

    def init_rest(self):
        lib().orc_init_rest(self._h)

    def set_state(self, Np, rho_prev=None, Ut2_prev=None):
        Np = np.ascontiguousarray(Np, dtype=np.float64)
        assert Np.shape == (self.Q, self.n1, self.n2)
        r = None if rho_prev is None else np.ascontiguousarray(rho_prev, dtype=np.float64)
        u = None if Ut2_prev is None else np.ascontiguousarray(Ut2_prev, dtype=np.float64)
        lib().orc_set_state(self._h, _p(Np), _p(r), _p(u))

    def state(self):
        out = np.empty((self.Q, self.n1, self.n2))
        lib().orc_get_state(self._h, _p(out))
        return out

    def prev_moments(self):
        r = np.empty((self.n1, self.n2))
        u = np.empty((self.n1, self.n2))
        lib().orc_get_prev_moments(self._h, _p(r), _p(u))
        return r, u

    def step(self, n=1):
        lib().orc_step(self._h, int(n))

    @property
    def t(self):
        return lib().orc_time(self._h)

    # diagnostics ----------------------------------------------------------
    def moments(self):
        """dict of rho, U1, U2, Ut1, Ut2, F1, F2 (each (n1, n2))."""
        names = ["rho", "U1", "U2", "Ut1", "Ut2", "F1", "F2"]
        arrs = {k: np.empty((self.n1, self.n2)) for k in names}
        lib().orc_moments(self._h, *[_p(arrs[k]) for k in names])
        return arrs

    def collide_one(self, i, j):
        """Internals of one cell's collision (1-based i, j) from the current state."""
        Q = self.Q
        o = {k: np.empty(Q) for k in ("Npost", "Nin", "feq", "dN")}
        F = np.empty(2)
        Ut = np.empty(2)
        dPi = np.empty(4)
        rho = C.c_double()
        lib().orc_collide_one(self._h, int(i), int(j), _p(o["Npost"]), _p(o["Nin"]),
                              _p(o["feq"]), _p(o["dN"]), _p(F), _p(Ut), _p(dPi),
                              C.byref(rho))
        o.update(F=F, Ut=Ut, dPi=dPi.reshape(2, 2), rho=rho.value)
        return o

    def node_geometry(self, i, j):
        out = np.empty(12)
        if lib().orc_node_geometry(self._h, int(i), int(j), _p(out)) != 0:
            raise IndexError((i, j))
        return dict(g1=out[0:2], g2=out[2:4], G1=out[4:6], G2=out[6:8], J=out[8],
                    ginv=np.array([[out[9], out[10]], [out[10], out[11]]]))

    def theta(self, i, j, alpha, s):
        out = np.empty(4)
        lib().orc_theta(self._h, int(i), int(j), int(alpha), int(s), _p(out))
        return out.reshape(2, 2)

    def feq(self, alpha, rho, U, Ut, ginv):
        U = np.ascontiguousarray(U, dtype=np.float64)
        Ut = np.ascontiguousarray(Ut, dtype=np.float64)
        gi = np.ascontiguousarray(ginv, dtype=np.float64).reshape(4)
        return lib().orc_feq(self._h, int(alpha), float(rho), _p(U), _p(Ut), _p(gi))

    def totals(self):
        out = np.empty(3)
        lib().orc_totals(self._h, _p(out))
        return out

    def flow_diagnostics(self, rho, Ut1, Ut2, prev=None, dt=0):
        """Sec. 3.1 diagnostics of given fields (each (n1, n2)); prev is the
        (Ut1, Ut2) pair dt steps earlier or None.  dict of res, ke, am (angular
        momentum about the origin; 0 on planar grids), umax, uu (sum J |u|^2)."""
        f = [np.ascontiguousarray(a, dtype=np.float64) for a in (rho, Ut1, Ut2)]
        for a in f:
            assert a.shape == (self.n1, self.n2)
        p = (None, None) if prev is None else tuple(
            np.ascontiguousarray(a, dtype=np.float64) for a in prev)
        out = np.empty(5)
        lib().orc_flow_diagnostics(self._h, _p(f[0]), _p(f[1]), _p(f[2]), _p(p[0]), _p(p[1]),
                                   int(dt), _p(out))
        return dict(res=out[0], ke=out[1], am=out[2], umax=out[3], uu=out[4])

    def diagnostics(self, prev=None, dt=0):
        """flow_diagnostics of the current state's moments (orc_moments),
        plus the moment fields themselves (rho, Ut1, Ut2) and the totals
        (mass, P1, P2 of the state N'(t-1))."""
        m = self.moments()
        d = self.flow_diagnostics(m["rho"], m["Ut1"], m["Ut2"], prev, dt)
        d.update(rho=m["rho"], Ut1=m["Ut1"], Ut2=m["Ut2"], totals=self.totals())
        return d

    def volume(self):
        out = np.empty((self.n1, self.n2))
        lib().orc_get_volume(self._h, _p(out))
        return out

    def set_volume(self, J):
        J = np.ascontiguousarray(J, dtype=np.float64)
        lib().orc_set_volume(self._h, _p(J))

    def set_force_iterations(self, n):
        lib().orc_set_force_iterations(self._h, int(n))

    def no_flow_adjust(self, nsteps):
        r = np.empty((self.n1, self.n2))
        lib().orc_no_flow_adjust(self._h, int(nsteps), _p(r))
        return r


def threads():
    return lib().orc_threads()
