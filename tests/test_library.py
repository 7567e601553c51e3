"""CPU-side checks of the C ABI: the library builds, loads, exports every
function include/dust.h declares, and rejects bad arguments on the host
before touching a device."""
import ctypes

import numpy as np
import pytest

import __graft_entry__
import paper_0907_3768_gb300 as pkg
from paper_0907_3768_gb300 import _lib


@pytest.fixture(scope="module")
def L():
    __graft_entry__.build()
    return pkg.lib()


def test_exports_every_declared_function(L):
    names = pkg.header_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(L, name), f"{name} declared in include/dust.h but not exported"


def test_version(L):
    assert "sm_103a" in _lib.dust_version()


def _grid(K=16, G=3):
    lam = np.geomspace(1e-7, 1e-3, K)
    w = np.gradient(lam)
    C = np.ones((G, K)) * 1e-14
    return lam, w, C


@pytest.mark.parametrize("case,frag", [
    (dict(K=1), "K=1"),
    (dict(G=0), "G=0"),
    (dict(Tmin=5.0, Tmax=5.0), "T_min < T_max"),
    (dict(n_table=10), "n_table"),
    (dict(precision=7), "precision"),
    (dict(bad_lambda=True), "lambda"),
    (dict(neg_w=True), "w["),
    (dict(zero_grain=True), "absorbs nothing"),
    (dict(tiny_x=True), "emission kernel"),
])
def test_ctx_create_rejects(L, case, frag):
    K, G = case.get("K", 16), case.get("G", 3)
    lam, w, C = _grid(max(K, 2), max(G, 1))
    lam, w, C = lam[:K].copy(), w[:K].copy(), C[:max(G, 1), :K].copy()
    if case.get("bad_lambda"):
        lam[3] = lam[2]
    if case.get("neg_w"):
        w[2] = -1.0
    if case.get("zero_grain"):
        C[1] = 0.0
    Tmin, Tmax = case.get("Tmin", 2.0), case.get("Tmax", 3000.0)
    if case.get("tiny_x"):
        lam = np.geomspace(1e-7, 1.0, K)  # 1 m at 3000 K: x = 4.8e-6
    out = ctypes.c_void_p()
    rc = L.dust_ctx_create(ctypes.byref(out), K, lam.ctypes.data, w.ctypes.data, G, C.ctypes.data, Tmin,
                           Tmax, case.get("n_table", 0), case.get("precision", 0), 0)
    assert rc == _lib.DUST_EINVAL
    assert out.value is None
    assert frag in _lib.last_error()


def test_null_arguments(L):
    assert L.dust_ctx_create(None, 4, None, None, 1, None, 2.0, 3.0, 0, 0, 0) == _lib.DUST_EINVAL
    assert L.dust_solve(None, 10, None, 4, None, None, None, None, None, None) == _lib.DUST_EINVAL
    assert L.dust_solve_host(None, 10, None, 4, None, None, None, None, None) == _lib.DUST_EINVAL
    assert L.dust_ctx_set_precision(None, 0) == _lib.DUST_EINVAL
    assert L.dust_ctx_check(None, None) == _lib.DUST_EINVAL
    assert L.dust_ctx_set_fluctuating(None, 1, None, None, None, 128) == _lib.DUST_EINVAL
    assert L.dust_solve_fluct(None, 10, None, 4, None, None, None, None, None) == _lib.DUST_EINVAL
    L.dust_ctx_destroy(None)


def test_server_null_arguments(L):
    assert L.dust_server_create(None, 1 << 30, 4, 0) == _lib.DUST_EINVAL
    out = ctypes.c_void_p()
    assert L.dust_server_create(ctypes.byref(out), 1000, 4, 0) == _lib.DUST_EINVAL  # budget < 1 MiB
    assert L.dust_server_create(ctypes.byref(out), 1 << 30, 0, 0) == _lib.DUST_EINVAL
    t = ctypes.c_uint64()
    assert L.dust_serve_submit(None, None, 1, None, 4, None, None, None, None, None, None, ctypes.byref(t)) == \
        _lib.DUST_EINVAL
    assert L.dust_serve_poll(None, 1, None, None) == _lib.DUST_EINVAL
    assert L.dust_serve_wait(None, 1, 1.0, None) == _lib.DUST_EINVAL
    assert L.dust_serve_cancel(None, 1) == _lib.DUST_EINVAL
    assert L.dust_server_stats(None, None) == _lib.DUST_EINVAL
    L.dust_server_destroy(None)


def test_python_wrapper_raises(L):
    with pytest.raises(_lib.DustError) as e:
        _lib.dust_ctx_create(1, 0, 0, 1, 0, 2.0, 3000.0, 0, 0, 0)
    assert e.value.code == _lib.DUST_EINVAL


def test_wait_probe_rejects_bad_limits(L):
    # argument checks come before any CUDA call, so this needs no GPU
    for bad in (0.0, -1.0, 2000.5, float("nan")):
        assert L.dust_diag_wait_timeout(0, bad, None, None) == _lib.DUST_EINVAL
