"""The paper's CPU production scheme (Section 6, Table 1's "CPU (interpolation)"
column) -- TEST INFRASTRUCTURE: a timed CPU comparison, not the parity oracle.

Temperatures come from a per-grain table of 2000 temperatures over 3-1500 K,
spaced uniformly in ln T and interpolated linearly in (P, T); the heating
power (Eq. 6) and the emission SED (Eqs. 8-10) are computed in full, in FP64
on OpenMP threads (``cpu_interp.c``).  Only the tests and the benchmark's CPU
leg use it.
"""
import ctypes

import numpy as np

from . import lib as _oracle_lib

#: The paper's table: 2000 temperatures between 3 K and 1500 K (Section 6).
NT = 2000
T_LO = 3.0
T_HI = 1500.0

_ready = False


def _lib():
    global _ready
    L = _oracle_lib()
    if not _ready:
        d, i, i64, p = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
        L.dust_interp_table.restype = i
        L.dust_interp_table.argtypes = [i, p, p, i, p, d, d, i, p, p]
        L.dust_interp_run.restype = i
        L.dust_interp_run.argtypes = [i64, i, i, p, p, p, p, p, i, p, p, p, p, p, i]
        _ready = True
    return L


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Table:
    """Per-grain emitted power at the table's temperatures (Eq. 7 at the nodes)."""

    def __init__(self, lam, w, C, T_lo=T_LO, T_hi=T_HI, nt=NT):
        self.lam, self.w, self.C = _f64(lam), _f64(w), _f64(C)
        G, K = self.C.shape
        assert self.lam.shape == (K,) and self.w.shape == (K,)
        self.T_nodes = np.empty(nt)
        self.P = np.empty((G, nt))
        rc = _lib().dust_interp_table(K, _ptr(self.lam), _ptr(self.w), G, _ptr(self.C), float(T_lo),
                                      float(T_hi), nt, _ptr(self.T_nodes), _ptr(self.P))
        if rc != 0:
            raise ValueError("dust_interp_table: bad sizes or bracket")

    def run(self, J, n, want_L=True, n_threads=0):
        """T, flags and (if asked) L for every row of J / n."""
        J, n = _f64(J), _f64(n)
        G, K = self.C.shape
        nc = J.shape[0]
        assert J.shape == (nc, K) and n.shape == (nc, G)
        T = np.empty((nc, G))
        fl = np.empty((nc, G), dtype=np.uint8)
        L = np.empty((nc, K)) if want_L else None
        rc = _lib().dust_interp_run(nc, K, G, _ptr(self.lam), _ptr(self.w), _ptr(self.C), _ptr(J), _ptr(n),
                                    len(self.T_nodes), _ptr(self.T_nodes), _ptr(self.P), _ptr(T),
                                    _ptr(L) if want_L else ctypes.c_void_p(0), _ptr(fl), int(n_threads))
        if rc != 0:
            raise MemoryError("dust_interp_run: scratch allocation failed")
        return dict(T=T, flags=fl, L=L)


def for_workload(wl, **kw):
    """The table of a synth.Workload's grains."""
    return Table(wl.lam, wl.w, wl.C_abs, **kw)
