"""ctypes binding of libdust's C ABI (include/dust.h), function for function.

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  Loading fails loudly when libdust.so has not been built.
"""
import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdust.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "dust.h")

DUST_OK, DUST_EINVAL, DUST_ENOMEM, DUST_ECUDA, DUST_EBUSY, DUST_ETIMEOUT, DUST_ENOTFOUND = range(7)
STATUS_NAMES = {0: "DUST_OK", 1: "DUST_EINVAL", 2: "DUST_ENOMEM", 3: "DUST_ECUDA", 4: "DUST_EBUSY",
                5: "DUST_ETIMEOUT", 6: "DUST_ENOTFOUND"}
DUST_PREC_FP32, DUST_PREC_BF16X3, DUST_PREC_FP16X3 = 0, 1, 2
PRECISIONS = {"fp32": DUST_PREC_FP32, "bf16x3": DUST_PREC_BF16X3, "fp16x3": DUST_PREC_FP16X3}
DUST_FLAG_OK, DUST_FLAG_LOW, DUST_FLAG_HIGH, DUST_FLAG_INVALID, DUST_FLAG_NOCONV = 0, 1, 2, 4, 8


class DustError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None

_p, _i, _i64, _d, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
_SIGS = {
    "dust_ctx_create": (_i, [ctypes.POINTER(_p), _i, _p, _p, _i, _p, _d, _d, _i, _i, _i]),
    "dust_ctx_destroy": (None, [_p]),
    "dust_ctx_set_precision": (_i, [_p, _i]),
    "dust_ctx_set_fused": (_i, [_p, _i]),
    "dust_ctx_set_fused_emit": (_i, [_p, _i]),
    "dust_ctx_set_split_products": (_i, [_p, _i]),
    "dust_ctx_launch_count": (_i, [_p, ctypes.POINTER(ctypes.c_uint64)]),
    "dust_ctx_info": (_i, [_p, _p, _p, _p, _p, _p, _p]),
    "dust_solve": (_i, [_p, _i64, _p, _i64, _p, _p, _p, _p, _p, _p]),
    "dust_solve_prec": (_i, [_p, _i, _i64, _p, _i64, _p, _p, _p, _p, _p, _p]),
    "dust_solve_host": (_i, [_p, _i64, _p, _i64, _p, _p, _p, _p, _p]),
    "dust_ctx_check": (_i, [_p, _p]),
    "dust_ctx_profile": (_i, [_p, _i]),
    "dust_ctx_profile_read": (_i, [_p, _p, _p, _p, _p]),
    "dust_ctx_set_grain_sizes": (_i, [_p, _p]),
    "dust_ctx_set_fluctuating": (_i, [_p, _i, _p, _p, _p, _i]),
    "dust_solve_fluct": (_i, [_p, _i64, _p, _i64, _p, _p, _p, _p, _p]),
    "dust_solve_T_newton": (_i, [_p, _i64, _p, _i64, _p, _p, _p, _p]),
    "dust_solve_coupled": (_i, [_p, _i64, _p, _i64, _p, _p, _i, _d, _p, _p, _p, _p, _p, _p, _p]),
    "dust_ctx_set_grain_numbers": (_i, [_p, _p]),
    "dust_solve_mass": (_i, [_p, _i64, _p, _i64, _p, _p, _p, _p, _p, _p]),
    "dust_diag_wait_timeout": (_i, [_i, _d, _p, _p]),
    "dust_diag_throughput": (_i, [_i, _p, _p]),
    "dust_solve_noalloc": (_i, [_p, _i64, _p, _i64, _p, _p, _p, _p, _p, _p]),
    "dust_noalloc_max_cells": (_sz, [_p]),
    "dust_server_create": (_i, [ctypes.POINTER(_p), _sz, _i, _i]),
    "dust_serve_submit": (_i, [_p, _p, _i64, _p, _i64, _p, _p, _p, _p, _p, _p, ctypes.POINTER(ctypes.c_uint64)]),
    "dust_serve_poll": (_i, [_p, ctypes.c_uint64, _p, _p]),
    "dust_serve_wait": (_i, [_p, ctypes.c_uint64, _d, _p]),
    "dust_serve_cancel": (_i, [_p, ctypes.c_uint64]),
    "dust_server_stats": (_i, [_p, _p]),
    "dust_server_set_policy": (_i, [_p, _d, _d, _d, _d]),
    "dust_server_reset_stats": (_i, [_p]),
    "dust_server_destroy": (None, [_p]),
    "dust_last_error": (ctypes.c_char_p, []),
    "dust_version": (ctypes.c_char_p, []),
}


def header_functions(path=HEADER):
    """Names of every function declared in include/dust.h."""
    with open(path) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dust_[a-z0-9_]+)\s*\(", src)))


def lib():
    """The loaded libdust (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libdust is not built ({LIB_PATH} missing): run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def last_error():
    return lib().dust_last_error().decode()


def check(rc):
    if rc != DUST_OK:
        raise DustError(rc, last_error())
    return rc


# Thin wrappers with the C ABI's names (pointers as ints, NULL as 0 / None).
def dust_ctx_create(K, lambda_ptr, w_ptr, G, c_abs_ptr, T_min, T_max, n_table, precision, device):
    out = _p()
    check(lib().dust_ctx_create(ctypes.byref(out), K, lambda_ptr, w_ptr, G, c_abs_ptr, T_min, T_max,
                                n_table, precision, device))
    return out.value


def dust_ctx_destroy(ctx):
    lib().dust_ctx_destroy(ctx)


def dust_ctx_set_precision(ctx, precision):
    return check(lib().dust_ctx_set_precision(ctx, precision))


def dust_ctx_set_fused(ctx, fused):
    return check(lib().dust_ctx_set_fused(ctx, 1 if fused else 0))


def dust_ctx_set_fused_emit(ctx, fused):
    return check(lib().dust_ctx_set_fused_emit(ctx, 1 if fused else 0))


def dust_ctx_set_split_products(ctx, products):
    return check(lib().dust_ctx_set_split_products(ctx, int(products)))


def dust_ctx_launch_count(ctx):
    n = ctypes.c_uint64()
    check(lib().dust_ctx_launch_count(ctx, ctypes.byref(n)))
    return n.value


def dust_ctx_info(ctx):
    K, G, nt, prec, dev = (ctypes.c_int() for _ in range(5))
    nbytes = ctypes.c_size_t()
    check(lib().dust_ctx_info(ctx, ctypes.byref(K), ctypes.byref(G), ctypes.byref(nt),
                              ctypes.byref(prec), ctypes.byref(dev), ctypes.byref(nbytes)))
    return dict(K=K.value, G=G.value, n_table=nt.value, precision=prec.value, device=dev.value,
                device_bytes=nbytes.value)


def dust_solve(ctx, n_cells, J, ld, n, T, L, resid, flags, stream):
    return check(lib().dust_solve(ctx, n_cells, J, ld, n, T, L, resid, flags, stream))


def dust_solve_prec(ctx, precision, n_cells, J, ld, n, T, L, resid, flags, stream):
    return check(lib().dust_solve_prec(ctx, precision, n_cells, J, ld, n, T, L, resid, flags, stream))


def dust_solve_host(ctx, n_cells, J, ld, n, T, L, resid, flags):
    return check(lib().dust_solve_host(ctx, n_cells, J, ld, n, T, L, resid, flags))


def dust_ctx_check(ctx):
    st = ctypes.c_int()
    check(lib().dust_ctx_check(ctx, ctypes.byref(st)))
    return st.value


def dust_ctx_profile(ctx, enable):
    return check(lib().dust_ctx_profile(ctx, 1 if enable else 0))


def dust_ctx_profile_read(ctx):
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    cnt = ctypes.c_int64()
    check(lib().dust_ctx_profile_read(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(cnt)))
    return a.value, b.value, c.value, cnt.value


def dust_solve_noalloc(ctx, n_cells, J, ld, n, T, L, resid, flags, stream):
    return check(lib().dust_solve_noalloc(ctx, n_cells, J, ld, n, T, L, resid, flags, stream))


def dust_noalloc_max_cells(ctx):
    return lib().dust_noalloc_max_cells(ctx)


def dust_diag_throughput(device=0):
    a, b = ctypes.c_double(), ctypes.c_double()
    check(lib().dust_diag_throughput(device, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


class ServeStats(ctypes.Structure):
    """Mirror of dust_serve_stats."""
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "cancelled", "failed", "queued", "active",
                                              "cells_completed", "rounds", "launches")] + \
               [(n, ctypes.c_double) for n in ("p50_ms", "p99_ms", "max_ms", "mean_ms", "span_ms")] + \
               [("hbm_in_use", ctypes.c_size_t)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


SERVE_STATE = {0: "queued", 1: "active", 2: "done", 3: "cancelled"}


def dust_server_create(hbm_budget_bytes, max_inflight, device):
    out = _p()
    check(lib().dust_server_create(ctypes.byref(out), int(hbm_budget_bytes), int(max_inflight), int(device)))
    return out.value


def dust_serve_submit(srv, ctx, n_cells, J, ld, n, T, L, resid, flags, stream):
    t = ctypes.c_uint64()
    check(lib().dust_serve_submit(srv, ctx, n_cells, J, ld, n, T, L, resid, flags, stream, ctypes.byref(t)))
    return t.value


def dust_serve_poll(srv, ticket):
    st, lat = ctypes.c_int(), ctypes.c_double()
    check(lib().dust_serve_poll(srv, ticket, ctypes.byref(st), ctypes.byref(lat)))
    return st.value, lat.value


def dust_serve_wait(srv, ticket, timeout_ms):
    lat = ctypes.c_double()
    check(lib().dust_serve_wait(srv, ticket, float(timeout_ms), ctypes.byref(lat)))
    return lat.value


def dust_serve_cancel(srv, ticket):
    return check(lib().dust_serve_cancel(srv, ticket))


def dust_server_stats(srv):
    s = ServeStats()
    check(lib().dust_server_stats(srv, ctypes.byref(s)))
    return s.as_dict()


def dust_server_set_policy(srv, small_terms, batch_terms, chunk_terms, age_ms):
    return check(lib().dust_server_set_policy(srv, float(small_terms), float(batch_terms), float(chunk_terms),
                                              float(age_ms)))


def dust_server_reset_stats(srv):
    return check(lib().dust_server_reset_stats(srv))


def dust_server_destroy(srv):
    lib().dust_server_destroy(srv)


def dust_last_error():
    return last_error()


def dust_version():
    return lib().dust_version().decode()


def dust_diag_wait_timeout(device, limit_ms):
    """(device status word, elapsed ms) of the bounded-wait probe."""
    st, ms = ctypes.c_int(), ctypes.c_double()
    check(lib().dust_diag_wait_timeout(device, limit_ms, ctypes.byref(st), ctypes.byref(ms)))
    return st.value, ms.value


def dust_ctx_set_grain_sizes(ctx, a_m):
    return check(lib().dust_ctx_set_grain_sizes(ctx, a_m))


def dust_ctx_set_fluctuating(ctx, Gf, grains, n_atoms, theta, M):
    return check(lib().dust_ctx_set_fluctuating(ctx, Gf, grains, n_atoms, theta, M))


def dust_solve_fluct(ctx, n_cells, J, ld, n, L, P, dE, stream):
    return check(lib().dust_solve_fluct(ctx, n_cells, J, ld, n, L, P, dE, stream))


def dust_solve_T_newton(ctx, n_cells, J, ld, T, iters, flags, stream):
    return check(lib().dust_solve_T_newton(ctx, n_cells, J, ld, T, iters, flags, stream))


def dust_solve_coupled(ctx, n_cells, J_ext, ld, E, n, max_iters, tol, T, L, resid, flags, stream):
    """Returns (iterations run, last measured change of L)."""
    it, ch = ctypes.c_int(), ctypes.c_double()
    check(lib().dust_solve_coupled(ctx, n_cells, J_ext, ld, E, n, max_iters, tol, T, L, resid, flags,
                                   ctypes.byref(it), ctypes.byref(ch), stream))
    return it.value, ch.value


def dust_ctx_set_grain_numbers(ctx, n_g):
    return check(lib().dust_ctx_set_grain_numbers(ctx, n_g))


def dust_solve_mass(ctx, n_cells, J, ld, m, T, L, resid, flags, stream):
    return check(lib().dust_solve_mass(ctx, n_cells, J, ld, m, T, L, resid, flags, stream))
