"""ctypes front end of the plain FP64 3-D oracle (``clbm_oracle3d.c``, D3Q39).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
cpu_baseline leg of ``bench.py`` may import this module.  It does not import
the CUDA library and the CUDA library does not import it.

Populations are float64 arrays (39, n1, n2, n3) holding N'(q, t-1); cell
fields are (n1, n2, n3), vector fields (3, n1, n2, n3).  q^1 = i is
wall-normal, q^2 = j and q^3 = k periodic.
"""
import ctypes as C

import numpy as np

from . import oracle as _o

CHANNEL, ANNULUS = 0, 1
NOSLIP, MOVING = 0, 1
Q = 39

_done = False


def lib():
    global _done
    L = _o.lib()
    if not _done:
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        L.o3_lattice.argtypes = [ip, dp, ip, ip, dp]
        L.o3_create.restype = C.c_void_p
        L.o3_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, dp, C.c_double, C.c_double,
                                C.c_double, C.c_int, C.c_int]
        L.o3_destroy.argtypes = [C.c_void_p]
        L.o3_set_case.argtypes = [C.c_void_p] + [C.c_double] * 7
        L.o3_init_rest.argtypes = [C.c_void_p]
        L.o3_set_state.argtypes = [C.c_void_p, dp, dp, dp, dp]
        L.o3_get_state.argtypes = [C.c_void_p, dp]
        L.o3_step.argtypes = [C.c_void_p, C.c_longlong]
        L.o3_time.restype = C.c_longlong
        L.o3_time.argtypes = [C.c_void_p]
        L.o3_moments.argtypes = [C.c_void_p, dp, dp, dp, dp]
        L.o3_totals.argtypes = [C.c_void_p, dp]
        L.o3_row_geometry.restype = C.c_int
        L.o3_row_geometry.argtypes = [C.c_void_p, C.c_int, dp]
        L.o3_theta.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, dp]
        L.o3_feq.restype = C.c_double
        L.o3_feq.argtypes = [C.c_void_p, C.c_int, C.c_double, dp, dp, dp]
        L.o3_collide_one.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, dp, dp, dp, dp]
        _done = True
    return L


def _p(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def lattice():
    """(c [39, 3] int, w [39], star, hat, T0)."""
    c = (C.c_int * (3 * Q))()
    w = (C.c_double * Q)()
    st = (C.c_int * Q)()
    ht = (C.c_int * Q)()
    T0 = C.c_double()
    assert lib().o3_lattice(c, w, st, ht, C.byref(T0)) == 0
    return (np.array(list(c)).reshape(Q, 3), np.array(list(w)), np.array(list(st)),
            np.array(list(ht)), T0.value)


class Grid:
    def __init__(self, n1, n2, n3, kind=CHANNEL, edges=None, step2=1.0, step3=1.0, dx=0.0,
                 bc_lo=NOSLIP, bc_hi=NOSLIP):
        self.n1, self.n2, self.n3 = n1, n2, n3
        self.Q = Q
        e = np.ascontiguousarray(edges, dtype=np.float64)
        h = lib().o3_create(n1, n2, n3, kind, _p(e), float(step2), float(step3), float(dx),
                            int(bc_lo), int(bc_hi))
        if not h:
            raise ValueError("invalid 3-D oracle grid")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None:
            lib().o3_destroy(h)
            self._h = None

    def set_case(self, tau, rho0=1.0, U0_lo=0.0, U0_hi=0.0, gext=(0.0, 0.0, 0.0)):
        lib().o3_set_case(self._h, tau, rho0, U0_lo, U0_hi, gext[0], gext[1], gext[2])

    def init_rest(self):
        lib().o3_init_rest(self._h)

    def set_state(self, Np, rho_prev=None, ut2_prev=None, ut3_prev=None):
        Np = np.ascontiguousarray(Np, dtype=np.float64)
        assert Np.shape == (Q, self.n1, self.n2, self.n3)
        f = [None if x is None else np.ascontiguousarray(x, dtype=np.float64)
             for x in (rho_prev, ut2_prev, ut3_prev)]
        lib().o3_set_state(self._h, _p(Np), _p(f[0]), _p(f[1]), _p(f[2]))

    def state(self):
        out = np.empty((Q, self.n1, self.n2, self.n3))
        lib().o3_get_state(self._h, _p(out))
        return out

    def step(self, n=1):
        lib().o3_step(self._h, int(n))

    @property
    def t(self):
        return lib().o3_time(self._h)

    def moments(self):
        sh = (self.n1, self.n2, self.n3)
        rho = np.empty(sh)
        U, Ut, F = (np.empty((3,) + sh) for _ in range(3))
        lib().o3_moments(self._h, _p(rho), _p(U), _p(Ut), _p(F))
        return {"rho": rho, "U": U, "Ut": Ut, "F": F}

    def totals(self):
        out = np.empty(4)
        lib().o3_totals(self._h, _p(out))
        return out

    def row_geometry(self, i):
        out = np.empty(19)
        if lib().o3_row_geometry(self._h, int(i), _p(out)) != 0:
            raise IndexError(i)
        return {"J": out[0], "ginv": out[1:10].reshape(3, 3), "g": out[10:19].reshape(3, 3)}

    def theta(self, i, alpha, s):
        out = np.empty(9)
        lib().o3_theta(self._h, int(i), int(alpha), int(s), _p(out))
        return out.reshape(3, 3)

    def feq(self, alpha, rho, U, Ut, ginv):
        U = np.ascontiguousarray(U, dtype=np.float64)
        Ut = np.ascontiguousarray(Ut, dtype=np.float64)
        gi = np.ascontiguousarray(ginv, dtype=np.float64).reshape(9)
        return lib().o3_feq(self._h, int(alpha), float(rho), _p(U), _p(Ut), _p(gi))

    def collide_one(self, i, j, k):
        Npost, Nin, F = np.empty(Q), np.empty(Q), np.empty(3)
        rho = C.c_double()
        lib().o3_collide_one(self._h, int(i), int(j), int(k), _p(Npost), _p(Nin), _p(F), C.byref(rho))
        return {"Npost": Npost, "Nin": Nin, "F": F, "rho": rho.value}
