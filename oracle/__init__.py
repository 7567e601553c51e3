"""FP64 CPU oracle of the dust temperature / emission path -- TEST INFRASTRUCTURE.

Plain, slow and obviously correct: direct quadrature of Eqs. 6-10 and a Brent
root solve of Eq. 7 to 1e-13 in ln T.  Only the tests, the smoke check and the
benchmark's CPU-baseline / reference leg may import this package; the CUDA
library never does, and the two share no code.
"""
import ctypes
import math
import os

import numpy as np

from .build import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build()
        L = ctypes.CDLL(path)
        d, i, i64, p = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
        L.dust_oracle_planck.restype = d
        L.dust_oracle_planck.argtypes = [d, d]
        L.dust_oracle_absorbed.restype = d
        L.dust_oracle_absorbed.argtypes = [i, p, p, p]
        L.dust_oracle_power.restype = d
        L.dust_oracle_power.argtypes = [i, p, p, p, d]
        L.dust_oracle_temperature.restype = i
        L.dust_oracle_temperature.argtypes = [i, p, p, p, d, d, d, d, p, p]
        L.dust_oracle_temperature_bisect.restype = d
        L.dust_oracle_temperature_bisect.argtypes = [i, p, p, p, d, d, d, i]
        L.dust_oracle_emission.restype = None
        L.dust_oracle_emission.argtypes = [i, i, p, p, p, p, p]
        L.dust_oracle_run.restype = i64
        L.dust_oracle_run.argtypes = [i64, i, i, p, p, p, p, p, d, d, d, p, p, p, p, p, i]
        L.dust_oracle_max_threads.restype = i
        L.dust_oracle_max_threads.argtypes = []
        _lib = L
    return _lib


TOL_U = 1e-13


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def planck(lam, T):
    """B(lambda, T) per unit wavelength [W m^-2 m^-1 sr^-1] (Eq. 1)."""
    f = lib().dust_oracle_planck
    lam = np.asarray(lam, dtype=np.float64)
    return np.vectorize(lambda x: f(float(x), float(T)))(lam) if lam.ndim else f(float(lam), float(T))


def power(lam, w, C_g, T):
    """P_g(T) = sum_k w_k C_k B(lambda_k, T) (Eq. 7)."""
    lam, w, C_g = _f64(lam), _f64(w), _f64(C_g)
    return lib().dust_oracle_power(len(lam), _ptr(lam), _ptr(w), _ptr(C_g), float(T))


def absorbed(w, C_g, J_c):
    """A = sum_k w_k C_k J_k (Eq. 6)."""
    w, C_g, J_c = _f64(w), _f64(C_g), _f64(J_c)
    return lib().dust_oracle_absorbed(len(w), _ptr(w), _ptr(C_g), _ptr(J_c))


def temperature(lam, w, C_g, A, T_min, T_max, tol_u=TOL_U):
    """(T, flag, quadratures) for one grain (root of Eq. 7 by Brent)."""
    lam, w, C_g = _f64(lam), _f64(w), _f64(C_g)
    T = ctypes.c_double()
    ev = ctypes.c_int()
    fl = lib().dust_oracle_temperature(len(lam), _ptr(lam), _ptr(w), _ptr(C_g), float(A),
                                       float(T_min), float(T_max), float(tol_u),
                                       ctypes.byref(T), ctypes.byref(ev))
    return T.value, fl, ev.value


def temperature_bisect(lam, w, C_g, A, T_min, T_max, steps=200):
    lam, w, C_g = _f64(lam), _f64(w), _f64(C_g)
    return lib().dust_oracle_temperature_bisect(len(lam), _ptr(lam), _ptr(w), _ptr(C_g), float(A),
                                                float(T_min), float(T_max), int(steps))


def emission(lam, C, n_c, T_c):
    """L_k = 4 pi sum_g n_g C[g,k] B(lambda_k, T_g) for one cell (Eqs. 8-10)."""
    lam, C, n_c, T_c = _f64(lam), _f64(C), _f64(n_c), _f64(T_c)
    G, K = C.shape
    out = np.empty(K)
    lib().dust_oracle_emission(K, G, _ptr(lam), _ptr(C), _ptr(n_c), _ptr(T_c), _ptr(out))
    return out


def run(lam, w, C, J, n, T_min, T_max, want_L=True, want_resid=True, n_threads=0, tol_u=TOL_U):
    """The whole path for every row of J / n.

    Returns a dict with A, T, flags, and (if asked) L and resid, all FP64
    (flags uint8), plus ``evals`` = quadratures spent in root solves.
    """
    lam, w, C = _f64(lam), _f64(w), _f64(C)
    J, n = _f64(J), _f64(n)
    G, K = C.shape
    nc = J.shape[0]
    assert J.shape == (nc, K) and n.shape == (nc, G)
    A = np.empty((nc, G))
    T = np.empty((nc, G))
    fl = np.empty((nc, G), dtype=np.uint8)
    L = np.empty((nc, K)) if want_L else None
    r = np.empty(nc) if want_resid else None
    nul = ctypes.c_void_p(0)
    ev = lib().dust_oracle_run(nc, K, G, _ptr(lam), _ptr(w), _ptr(C), _ptr(J), _ptr(n),
                               float(T_min), float(T_max), float(tol_u), _ptr(A), _ptr(T),
                               _ptr(L) if want_L else nul, _ptr(fl), _ptr(r) if want_resid else nul,
                               int(n_threads))
    return dict(A=A, T=T, flags=fl, L=L, resid=r, evals=int(ev))


def run_coupled(lam, w, C, J_ext, E, n, T_min, T_max, tol=1e-12, max_iters=500):
    """Self-absorption fixed point (Section 2: dust heated by its own emission
    needs an iteration of the radiation field and the temperatures), local
    form: J = J_ext + E * L with L the emission (Eqs. 8-10) at the temperatures
    solved from J.  Plain fixed-point iteration in FP64, stopped when the
    largest peak-normalised change of L falls to `tol`.  Returns (result of
    the last run, iterations, last change)."""
    J_ext, E = _f64(J_ext), _f64(E)
    J = J_ext
    prev, ch = None, math.inf
    for it in range(1, max_iters + 1):
        res = run(lam, w, C, J, n, T_min, T_max)
        L = res["L"]
        if prev is not None:
            ch = float((np.abs(L - prev).max(axis=1) / L.max(axis=1)).max())
            if ch <= tol:
                return res, it, ch
        prev = L
        J = J_ext + E * L
    return res, max_iters, ch


def max_threads():
    return lib().dust_oracle_max_threads()


def run_workload(wl, **kw):
    """Run the oracle on a synth.Workload (its FP32 J / n widened exactly)."""
    return run(wl.lam, wl.w, wl.C_abs, wl.J, wl.n, wl.T_min, wl.T_max, **kw)
