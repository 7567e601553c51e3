"""Python front end of libdust: a context object over the C ABI.

PyTorch supplies device memory and streams; every number is computed by the
library's kernels.  There is no CPU fallback: without the built library or a
CUDA device the calls raise.
"""
import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import PRECISIONS


def _prec(p):
    if isinstance(p, str):
        return PRECISIONS[p.lower()]
    return int(p)


def _ptr(t):
    return 0 if t is None else t.data_ptr()


def padded_rows(J, multiple=4):
    """A [C, K] view of J whose row stride is a multiple of `multiple` elements
    (the tensor-core precisions read rows with 16-byte aligned TMA boxes)."""
    C, K = J.shape
    if J.stride(1) == 1 and J.stride(0) % multiple == 0 and J.data_ptr() % 16 == 0:
        return J
    ld = (K + multiple - 1) // multiple * multiple
    buf = torch.zeros((C, ld), dtype=torch.float32, device=J.device)
    buf[:, :K] = J
    return buf[:, :K]


class Context:
    """One wavelength grid + grain set, with its tables resident on `device`."""

    def __init__(self, lam, w, C_abs, T_min=2.0, T_max=3000.0, n_table=4096, precision="fp32", device=0):
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        w = np.ascontiguousarray(w, dtype=np.float64)
        C_abs = np.ascontiguousarray(C_abs, dtype=np.float64)
        G, K = C_abs.shape
        if lam.shape != (K,) or w.shape != (K,):
            raise ValueError("lambda / w must have C_abs.shape[1] entries")
        self.handle = None
        self.handle = _lib.dust_ctx_create(K, lam.ctypes.data, w.ctypes.data, G, C_abs.ctypes.data,
                                           float(T_min), float(T_max), int(n_table), _prec(precision),
                                           int(device))
        self.K, self.G, self.device = K, G, int(device)
        self.T_min, self.T_max = float(T_min), float(T_max)

    @classmethod
    def from_workload(cls, wl, precision="fp32", device=0):
        return cls(wl.lam, wl.w, wl.C_abs, wl.T_min, wl.T_max, wl.n_table, precision, device)

    def close(self):
        if self.handle:
            _lib.dust_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def info(self):
        return _lib.dust_ctx_info(self.handle)

    def set_precision(self, precision):
        _lib.dust_ctx_set_precision(self.handle, _prec(precision))

    def set_fused(self, fused=True):
        """Absorption and temperature solve as one kernel (tensor-core precisions)."""
        _lib.dust_ctx_set_fused(self.handle, fused)

    def set_fused_emit(self, fused=True):
        """Temperature solve and emission as one warp-specialized kernel, where it applies."""
        _lib.dust_ctx_set_fused_emit(self.handle, fused)

    def set_split_products(self, products=3):
        """Split products per K step of the tensor-core precisions: 3 (default) or 2
        (the J_hi W_lo product left out; an ablation, not held to the mixed tolerances)."""
        _lib.dust_ctx_set_split_products(self.handle, products)

    def check(self):
        """Device status word since the last check (0 = DUST_OK)."""
        return _lib.dust_ctx_check(self.handle)

    def _check_inputs(self, J, n):
        if not (J.is_cuda and n.is_cuda):
            raise ValueError("J and n must be CUDA tensors")
        if J.dtype != torch.float32 or n.dtype != torch.float32:
            raise ValueError("J and n must be float32")
        C = J.shape[0]
        if J.dim() != 2 or J.shape[1] != self.K or J.stride(1) != 1 or J.stride(0) < self.K:
            raise ValueError(f"J must be [C, {self.K}] with unit column stride")
        if n.shape != (C, self.G) or not n.is_contiguous():
            raise ValueError(f"n must be a contiguous [C, {self.G}] tensor")
        return C, J.stride(0)

    def alloc_outputs(self, C, ld, want_L=True, want_resid=True, want_flags=True):
        dev = torch.device("cuda", self.device)
        out = dict(T=torch.empty((C, self.G), dtype=torch.float32, device=dev))
        out["L_buf"] = torch.empty((C, ld), dtype=torch.float32, device=dev) if want_L else None
        out["L"] = out["L_buf"][:, :self.K] if want_L else None
        out["resid"] = torch.empty((C,), dtype=torch.float64, device=dev) if want_resid else None
        out["flags"] = torch.empty((C, self.G), dtype=torch.uint8, device=dev) if want_flags else None
        return out

    def solve(self, J, n, precision=None, want_L=True, want_resid=True, want_flags=True, out=None,
              stream=None):
        """Run the hot path on device tensors; returns a dict of output tensors
        (T [C,G], L [C,K] view, resid [C] float64, flags [C,G] uint8)."""
        C, ld = self._check_inputs(J, n)
        if out is None:
            out = self.alloc_outputs(C, ld, want_L, want_resid, want_flags)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        sptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        if precision is None:  # the context's own precision
            _lib.dust_solve(self.handle, C, J.data_ptr(), ld, n.data_ptr(), out["T"].data_ptr(),
                            _ptr(out["L_buf"]), _ptr(out["resid"]), _ptr(out["flags"]), sptr)
        else:
            _lib.dust_solve_prec(self.handle, _prec(precision), C, J.data_ptr(), ld, n.data_ptr(),
                                 out["T"].data_ptr(), _ptr(out["L_buf"]), _ptr(out["resid"]), _ptr(out["flags"]),
                                 sptr)
        return out

    def submit(self, server, J, n, out=None, want_L=True, want_resid=True, want_flags=True, stream=None):
        """Queue a solve on `server` (continuous batching); returns (ticket, out).
        J, n and out must stay alive until the request finishes.  `stream`
        (default: the current torch stream) is where J and n were produced;
        the server waits for it on the device, so no synchronisation is needed."""
        C, ld = self._check_inputs(J, n)
        if out is None:
            out = self.alloc_outputs(C, ld, want_L, want_resid, want_flags)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        sptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        t = _lib.dust_serve_submit(server.handle, self.handle, C, J.data_ptr(), ld, n.data_ptr(),
                                   out["T"].data_ptr(), _ptr(out["L_buf"]), _ptr(out["resid"]),
                                   _ptr(out["flags"]), sptr)
        return t, out

    def set_grain_numbers(self, n_g):
        """Grains of each kind per unit dust mass [G] (the paper's n_s), for solve_mass."""
        a = np.ascontiguousarray(n_g, dtype=np.float64)
        if a.shape != (self.G,):
            raise ValueError(f"n_g must have shape ({self.G},)")
        _lib.dust_ctx_set_grain_numbers(self.handle, a.ctypes.data)

    def solve_mass(self, J, m, out=None, want_L=True, want_resid=True, want_flags=True, stream=None):
        """The hot path with n[c,g] = n_g m_c (Eqs. 9-10): m [C] float32 CUDA
        tensor of the cells' dust masses; outputs as solve()."""
        C = J.shape[0]
        if m.shape != (C,) or m.dtype != torch.float32 or not m.is_cuda or not m.is_contiguous():
            raise ValueError("m must be a contiguous float32 CUDA tensor of shape [C]")
        if J.dim() != 2 or J.shape[1] != self.K or J.stride(1) != 1 or J.dtype != torch.float32 or not J.is_cuda:
            raise ValueError(f"J must be a [C, {self.K}] float32 CUDA tensor with unit column stride")
        ld = J.stride(0)
        if out is None:
            out = self.alloc_outputs(C, ld, want_L, want_resid, want_flags)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        sptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        _lib.dust_solve_mass(self.handle, C, J.data_ptr(), ld, m.data_ptr(), out["T"].data_ptr(),
                             _ptr(out["L_buf"]), _ptr(out["resid"]), _ptr(out["flags"]), sptr)
        return out

    def solve_coupled(self, J_ext, E, n, max_iters=50, tol=1e-6, stream=None):
        """Self-absorbing solve: J = J_ext + E L iterated with the solve until L
        changes by at most `tol` (peak-normalised).  J_ext and E are [C, K]
        views with the same row stride.  Returns (outputs, iterations, change)."""
        C, ld = self._check_inputs(J_ext, n)
        if E.shape != J_ext.shape or E.stride() != J_ext.stride() or E.dtype != torch.float32:
            raise ValueError("E must be a float32 tensor shaped and strided like J_ext")
        out = self.alloc_outputs(C, ld)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        sptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        it, ch = _lib.dust_solve_coupled(self.handle, C, J_ext.data_ptr(), ld, E.data_ptr(), n.data_ptr(),
                                         int(max_iters), float(tol), out["T"].data_ptr(),
                                         out["L_buf"].data_ptr(), out["resid"].data_ptr(),
                                         out["flags"].data_ptr(), sptr)
        return out, it, ch

    def set_grain_sizes(self, a_m):
        """Grain radii [G] in metres, for the paper's Newton kernel (Eqs. 11-12 guess)."""
        a = np.ascontiguousarray(a_m, dtype=np.float64)
        if a.shape != (self.G,):
            raise ValueError(f"a_m must have shape ({self.G},)")
        _lib.dust_ctx_set_grain_sizes(self.handle, a.ctypes.data)

    def solve_T_newton(self, J, stream=None):
        """Temperatures by the paper's own kernel-3 method (per-iterate quadrature
        Newton, 0.1 % stop); returns dict T [C,G], iters [C,G] uint8, flags."""
        C, K = J.shape
        if K != self.K or J.dtype != torch.float32 or J.stride(1) != 1 or not J.is_cuda:
            raise ValueError("J must be a [C, K] float32 CUDA tensor with unit-stride rows")
        dev = torch.device("cuda", self.device)
        out = dict(T=torch.empty((C, self.G), dtype=torch.float32, device=dev),
                   iters=torch.empty((C, self.G), dtype=torch.uint8, device=dev),
                   flags=torch.empty((C, self.G), dtype=torch.uint8, device=dev))
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        sptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        _lib.dust_solve_T_newton(self.handle, C, J.data_ptr(), J.stride(0), out["T"].data_ptr(),
                                 out["iters"].data_ptr(), out["flags"].data_ptr(), sptr)
        return out

    def set_fluctuating(self, grains, n_atoms, theta, M=128):
        """Treat grains `grains` as thermally fluctuating: Einstein-solid
        enthalpy with n_atoms atoms and characteristic temperature theta [K]
        each, distributions on M levels."""
        g = np.ascontiguousarray(grains, dtype=np.int32)
        na = np.ascontiguousarray(n_atoms, dtype=np.float64)
        th = np.ascontiguousarray(theta, dtype=np.float64)
        if g.ndim != 1 or na.shape != g.shape or th.shape != g.shape:
            raise ValueError("grains, n_atoms and theta must be 1-D of one length")
        _lib.dust_ctx_set_fluctuating(self.handle, len(g), g.ctypes.data, na.ctypes.data, th.ctypes.data, int(M))
        self.fluct_Gf, self.fluct_M = len(g), int(M)

    def solve_fluct(self, J, n_f, want_L=True, want_P=False, want_dE=True, out=None, stream=None):
        """Level distributions and emission of the fluctuating grains: J as in
        solve ([C, ld] rows), n_f [C, Gf] their numbers.  Returns dict L
        [C, ld] (columns >= K unwritten), P [C, Gf, M], dE [C, Gf] (J)."""
        C, ld = J.shape[0], J.stride(0)
        if J.dtype != torch.float32 or J.stride(1) != 1 or not J.is_cuda or J.shape[1] < self.K:
            raise ValueError("J must be a [C, >=K] float32 CUDA tensor with unit-stride rows")
        Gf, M = self.fluct_Gf, self.fluct_M
        if n_f.shape != (C, Gf) or n_f.dtype != torch.float32 or not n_f.is_contiguous() or not n_f.is_cuda:
            raise ValueError(f"n_f must be a contiguous [C, {Gf}] float32 CUDA tensor")
        dev = torch.device("cuda", self.device)
        if out is None:
            out = {}
            if want_L:
                out["L"] = torch.empty((C, ld), dtype=torch.float32, device=dev)
            if want_P:
                out["P"] = torch.empty((C, Gf, M), dtype=torch.float32, device=dev)
            if want_dE:
                out["dE"] = torch.empty((C, Gf), dtype=torch.float32, device=dev)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        sptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        ptr = lambda k: out[k].data_ptr() if out.get(k) is not None else None
        _lib.dust_solve_fluct(self.handle, C, J.data_ptr(), ld, n_f.data_ptr(), ptr("L"), ptr("P"), ptr("dE"), sptr)
        return out

    def solve_host(self, J, n, T=None, L=None, resid=None, flags=None):
        """The hot path on host arrays (numpy or CPU tensors, ideally pinned);
        outputs are written into / returned as host arrays."""
        Jn = J.numpy() if isinstance(J, torch.Tensor) else J
        nn = n.numpy() if isinstance(n, torch.Tensor) else n
        C, K = Jn.shape
        if K != self.K or Jn.dtype != np.float32 or nn.dtype != np.float32 or nn.shape != (C, self.G):
            raise ValueError("J [C,K] and n [C,G] must be float32 host arrays")
        if Jn.strides[1] != 4 or not nn.flags.c_contiguous:
            raise ValueError("J rows must be unit stride and n contiguous")
        ld = Jn.strides[0] // 4
        T = np.empty((C, self.G), np.float32) if T is None else T
        if L is None:
            Lb = np.empty((C, ld), np.float32)
            L = Lb[:, :K]
        else:
            Lb = L
        resid = np.empty(C, np.float64) if resid is None else resid
        flags = np.empty((C, self.G), np.uint8) if flags is None else flags
        _lib.dust_solve_host(self.handle, C, Jn.ctypes.data, ld, nn.ctypes.data, T.ctypes.data,
                             Lb.ctypes.data, resid.ctypes.data, flags.ctypes.data)
        return dict(T=T, L=L, resid=resid, flags=flags)


class Server:
    """Continuous-batching request server on one GPU (see include/dust.h)."""

    def __init__(self, hbm_budget_bytes, max_inflight=32, device=0):
        self.handle = None
        self.handle = _lib.dust_server_create(int(hbm_budget_bytes), int(max_inflight), int(device))

    def poll(self, ticket):
        """(state name, latency ms); a finished ticket is released by the poll."""
        st, lat = _lib.dust_serve_poll(self.handle, ticket)
        return _lib.SERVE_STATE.get(st, st), lat

    def wait(self, ticket, timeout_ms=60000.0):
        return _lib.dust_serve_wait(self.handle, ticket, timeout_ms)

    def cancel(self, ticket):
        _lib.dust_serve_cancel(self.handle, ticket)

    def stats(self):
        return _lib.dust_server_stats(self.handle)

    def set_policy(self, small_terms=1e9, batch_terms=5e9, chunk_terms=1e10, age_ms=20.0):
        """Round sizes and the aging of the shortest-work-first ranking (see include/dust.h)."""
        _lib.dust_server_set_policy(self.handle, small_terms, batch_terms, chunk_terms, age_ms)

    def reset_stats(self):
        _lib.dust_server_reset_stats(self.handle)

    def close(self):
        if self.handle:
            _lib.dust_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
