"""GPU parity: the CUDA path against the FP64 oracle on identical seeded inputs.

Tolerances (relative): FP32 path T <= 1e-5, L <= 1e-4; tensor-core mixed
paths T <= 1e-3, L <= 5e-3, with L measured peak-floored (tests/metrics.py).
Full-size configurations run on the GPU in the launch configuration the
benchmark times, and are checked on sampled cells the oracle computes one by
one.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from metrics import assert_flags_match, l_err, t_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": (1e-5, 1e-4), "bf16x3": (1e-3, 5e-3), "fp16x3": (1e-3, 5e-3)}
RESID_TOL = {"fp32": 2e-5, "bf16x3": 2e-4, "fp16x3": 2e-4}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()


def _ctx(wl, prec):
    from paper_0907_3768_gb300 import Context

    return Context.from_workload(wl, precision=prec)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run(ctx, J, n, **kw):
    from paper_0907_3768_gb300 import padded_rows

    Jd = J if isinstance(J, torch.Tensor) else _dev(J)
    if kw.get("precision", None) not in (None, "fp32"):
        Jd = padded_rows(Jd)
    out = ctx.solve(Jd, n if isinstance(n, torch.Tensor) else _dev(n), **kw)
    torch.cuda.synchronize()
    assert ctx.check() == 0
    return {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in out.items()}


def _compare(out, ref, prec, wl, rows=None):
    tT, tL = TOL[prec]
    T = out["T"] if rows is None else out["T"][rows]
    L = out["L"] if rows is None else out["L"][rows]
    fl = out["flags"] if rows is None else out["flags"][rows]
    r = out["resid"] if rows is None else out["resid"][rows]
    assert_flags_match(fl, ref, wl)
    eT = t_err(T, ref["T"], ref["flags"])
    eL = l_err(L, ref["L"])
    assert eT.max(initial=0.0) <= tT, f"T err {eT.max():.3g}"
    assert eL.max() <= tL, f"L err {eL.max():.3g}"
    assert np.abs(r).max() <= RESID_TOL[prec], f"resid {np.abs(r).max():.3g}"
    return eT.max(initial=0.0), eL.max()


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "fp16x3"])
def test_tiny_config_full(prec):
    wl = synth.make_workload(0)
    ref = oracle.run_workload(wl)
    with _ctx(wl, prec) as ctx:
        out = _run(ctx, wl.J, wl.n, precision=prec)
    _compare(out, ref, prec, wl)


@pytest.mark.parametrize("cfg,prec", [(1, "fp32"), (2, "bf16x3"), (2, "fp16x3"), (3, "bf16x3"), (3, "fp32")])
def test_full_size_sampled(cfg, prec):
    """Whole configuration on the GPU; oracle on every (C/384)-th cell."""
    wl = synth.make_workload(cfg)
    C = wl.n_cells_total
    rows = np.arange(0, C, C // 384)
    if cfg == 3:  # add opaque cells explicitly
        _, _, opaque, _ = synth.workloads._cell_draws(synth.CONFIGS[3], C, wl.seed)
        rows = np.union1d(rows, np.nonzero(opaque)[0][:: max(1, opaque.sum() // 128)])
    sub = synth.make_workload(cfg, cells=rows)
    np.testing.assert_array_equal(sub.J, wl.J[rows])
    ref = oracle.run_workload(sub)
    with _ctx(wl, prec) as ctx:
        out = _run(ctx, wl.J, wl.n, precision=prec)
    del wl
    assert np.isfinite(out["T"]).all() and np.isfinite(out["L"]).all()
    _compare(out, ref, prec, sub, rows)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_blackbody_field_gives_its_temperature(prec):
    """Closed form independent of the oracle: J = B(T0) returns T = T0."""
    wl = synth.make_workload(0, cells=np.arange(64))
    T0 = np.exp(np.linspace(math.log(5.0), math.log(2000.0), 64))
    sig = synth.workloads._SIGMA_SB
    J = np.stack([synth.blackbody_shape(wl.lam, t) * sig * t ** 4 / math.pi for t in T0]).astype(np.float32)
    with _ctx(wl, prec) as ctx:
        out = _run(ctx, J, wl.n, precision=prec)
    assert (out["flags"] == 0).all()
    err = np.abs(out["T"] / T0[:, None] - 1.0).max()
    assert err <= (2e-6 if prec == "fp32" else 1e-4), err


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
@pytest.mark.parametrize("C", [1, 2, 127, 129, 1000, 2049, 5000])
def test_ragged_cell_counts(prec, C):
    wl = synth.make_workload(0 if C <= 1024 else 1, cells=np.arange(C))
    ref = oracle.run_workload(wl)
    with _ctx(wl, prec) as ctx:
        out = _run(ctx, wl.J, wl.n, precision=prec)
    _compare(out, ref, prec, wl)


@pytest.mark.parametrize("n_table,tol_L", [(64, 1e-3), (256, 1e-4)])
def test_coarse_tables(n_table, tol_L):
    """Small tables.  At n_table = 64 the inverse-table intervals of the tiny
    configuration span up to 0.18 in log2 T (more than 1/8), so 2^(tau du)
    takes ex2 instead of its five-term series; in FP64 the cubic there is
    good to 3e-6 in T (1e-8 at 256), so the FP32 T tolerance holds and L,
    whose Wien terms scale T's error by up to ~90, gets 1e-3."""
    from paper_0907_3768_gb300 import Context

    wl = synth.make_workload(0)
    ref = oracle.run_workload(wl)
    with Context(wl.lam, wl.w, wl.C_abs, wl.T_min, wl.T_max, n_table, "fp32") as ctx:
        assert ctx.info()["n_table"] == n_table
        out = _run(ctx, wl.J, wl.n, precision="fp32")
    assert_flags_match(out["flags"], ref, wl)
    eT = t_err(out["T"], ref["T"], ref["flags"])
    assert eT.max(initial=0.0) <= 1e-5, f"T err {eT.max():.3g}"
    assert l_err(out["L"], ref["L"]).max() <= tol_L


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3"])
def test_two_split_products(prec):
    """The ablation of the split's third product (J_hi W_lo): with it left out,
    W is rounded to 16 bits once (relative error up to 2^-9 in BF16), so the
    absorbed power moves by up to ~2e-3 and T by that over d ln P / d ln T
    (>= 1, about 5 on these grains): T is held to 1e-3 and L, whose Wien
    terms scale T's error further, to 2e-2.  Switching back gives the
    three-product bits again."""
    from paper_0907_3768_gb300 import _lib

    wl = synth.make_workload(0)
    ref = oracle.run_workload(wl)
    with _ctx(wl, prec) as ctx:
        a = _run(ctx, wl.J, wl.n, precision=prec)
        ctx.set_split_products(2)
        b = _run(ctx, wl.J, wl.n, precision=prec)
        ctx.set_split_products(3)
        c = _run(ctx, wl.J, wl.n, precision=prec)
        with pytest.raises(_lib.DustError) as e:
            ctx.set_split_products(4)
        assert e.value.code == _lib.DUST_EINVAL
    for k in ("T", "L", "flags", "resid"):
        np.testing.assert_array_equal(a[k], c[k])
    assert not np.array_equal(a["T"], b["T"])
    assert t_err(b["T"], ref["T"], ref["flags"]).max(initial=0.0) <= 1e-3
    assert l_err(b["L"], ref["L"]).max() <= 2e-2


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_odd_shapes(prec):
    """G not a multiple of 16, K not a multiple of 8 or of the 32-wavelength chunk."""
    cfg = dict(synth.CONFIGS[0])
    cfg.update(K=37, n_sizes=5, species=("silicate",), n_cells=300, seed=77)
    wl = synth.make_workload(cfg)
    ref = oracle.run_workload(wl)
    with _ctx(wl, prec) as ctx:
        out = _run(ctx, wl.J, wl.n, precision=prec)
    _compare(out, ref, prec, wl)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
@pytest.mark.parametrize("K,sizes,species,lam_um", [(2048, 256, ("silicate", "graphite"), (0.09, 1000.0)),
                                                     (2, 1, ("graphite",), (5.0, 200.0))])
def test_size_limits(prec, K, sizes, species, lam_um):
    """The documented limits.  K = 2048, G = 512: a second tensor-core MMA for
    grain columns past 256, four solve passes per cell, the emission's
    cross-section chunks at one cell pair per tile, 256 residual partials.
    K = 2, G = 1 (two mid-infrared wavelengths, so that the grains solve inside
    the bracket): one padded wavelength chunk and one padded grain group."""
    cfg = dict(synth.CONFIGS[0])
    cfg.update(K=K, n_sizes=sizes, species=species, n_cells=49, seed=91, lam_um=lam_um)
    wl = synth.make_workload(cfg)
    assert (wl.K, wl.G) == (K, sizes * len(species))
    ref = oracle.run_workload(wl)
    with _ctx(wl, prec) as ctx:
        out = _run(ctx, wl.J, wl.n, precision=prec)
    _compare(out, ref, prec, wl)


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3"])
@pytest.mark.parametrize("sizes,C", [(64, 255), (64, 513), (65, 257)])
def test_gemm_orientation_boundary(prec, sizes, C):
    """Two species x 64 sizes = 128 grains: the grain-major GEMM with every one of
    its 128 MMA rows a real grain; x 65 = 130 grains: the cell-major GEMM.  Cell
    counts just off the 256-cell tile of the former."""
    cfg = dict(synth.CONFIGS[0])
    cfg.update(K=100, n_sizes=sizes, species=("silicate", "graphite"), n_cells=C, seed=123)
    wl = synth.make_workload(cfg)
    assert wl.G == 2 * sizes
    ref = oracle.run_workload(wl)
    with _ctx(wl, prec) as ctx:
        out = _run(ctx, wl.J, wl.n, precision=prec)
    _compare(out, ref, prec, wl)


def test_edge_inputs_flags():
    wl = synth.make_workload(0, cells=np.arange(8))
    J = wl.J.copy()
    J[0] = 0.0
    J[1] *= np.float32(1e25)
    J[2, 7] = np.nan
    J[3] *= np.float32(1e-30)
    ref = oracle.run(wl.lam, wl.w, wl.C_abs, J, wl.n, wl.T_min, wl.T_max)
    with _ctx(wl, "fp32") as ctx:
        out = _run(ctx, J, wl.n)
    np.testing.assert_array_equal(out["flags"], ref["flags"])
    assert (out["flags"][0] == 1).all() and (out["T"][0] == np.float32(wl.T_min)).all()
    assert (out["flags"][1] == 2).all() and (out["T"][1] == np.float32(wl.T_max)).all()
    assert (out["flags"][2] == 4).all() and np.isnan(out["T"][2]).all()
    ok = [0, 1, 3, 4, 5, 6, 7]
    assert l_err(out["L"][ok], ref["L"][ok]).max() <= 1e-4
    assert np.abs(out["resid"][ok]).max() <= 2e-5


def test_modes_agree_bitwise():
    """T-only, residual-only and full calls give identical T; ld > K padding works."""
    wl = synth.make_workload(0, cells=np.arange(500))
    with _ctx(wl, "fp32") as ctx:
        full = _run(ctx, wl.J, wl.n)
        tonly = _run(ctx, wl.J, wl.n, want_L=False, want_resid=False)
        ronly = _run(ctx, wl.J, wl.n, want_L=False)
        buf = torch.full((500, wl.K + 11), 7.0, device="cuda")
        buf[:, :wl.K] = _dev(wl.J)
        pad = _run(ctx, buf[:, :wl.K], _dev(wl.n))
    np.testing.assert_array_equal(tonly["T"], full["T"])
    np.testing.assert_array_equal(ronly["T"], full["T"])
    np.testing.assert_array_equal(ronly["resid"], full["resid"])
    np.testing.assert_array_equal(pad["T"], full["T"])
    np.testing.assert_array_equal(pad["L"], full["L"])


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_cell_results_independent_of_batch(prec):
    """A cell's outputs are bitwise the same whatever batch it is solved in."""
    wl = synth.make_workload(1, cells=np.arange(3000))
    with _ctx(wl, prec) as ctx:
        a = _run(ctx, wl.J, wl.n, precision=prec)
        b = _run(ctx, wl.J[1234:2345], wl.n[1234:2345], precision=prec)
    for k in ("T", "L", "resid", "flags"):
        np.testing.assert_array_equal(a[k][1234:2345], b[k])


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_host_entry_point_matches_device(prec):
    """Host buffers through the copy-in / compute / copy-out pipeline: six
    chunks of growing size over 3 buffer sets (a ragged last one), called
    twice in a row."""
    from paper_0907_3768_gb300 import Context

    wl = synth.make_workload(1, cells=np.arange(40001))  # K = 200: rows already 16-byte multiples
    with Context.from_workload(wl, precision=prec) as ctx:
        dev = _run(ctx, wl.J, wl.n, precision=prec)
        for _ in range(2):
            host = ctx.solve_host(wl.J, wl.n)
            for k in ("T", "L", "resid", "flags"):
                np.testing.assert_array_equal(host[k], dev[k])


def test_invalid_device_arguments():
    from paper_0907_3768_gb300 import DustError
    from paper_0907_3768_gb300 import _lib

    wl = synth.make_workload(0, cells=np.arange(4))
    with _ctx(wl, "fp32") as ctx:
        J = _dev(wl.J)
        n = _dev(wl.n)
        T = torch.empty((4, wl.G), device="cuda")
        with pytest.raises(DustError):  # host pointer where device memory is required
            _lib.dust_solve(ctx.handle, 4, wl.J.ctypes.data, wl.K, n.data_ptr(), T.data_ptr(), 0, 0, 0, 0)
        with pytest.raises(DustError):  # ld < K
            _lib.dust_solve(ctx.handle, 4, J.data_ptr(), wl.K - 1, n.data_ptr(), T.data_ptr(), 0, 0, 0, 0)
        # zero cells is a no-op
        _lib.dust_solve(ctx.handle, 0, 0, wl.K, 0, 0, 0, 0, 0, 0)
        assert ctx.check() == 0
