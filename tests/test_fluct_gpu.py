"""Thermally fluctuating grains on the GPU (dust_solve_fluct) against the FP64
oracle of the same method (oracle/fluct.py): level spacing, level
probabilities and emission, element by element, over several level counts,
ragged cell and grain counts, and the degenerate fields.

Tolerances.  The kernel runs in FP32 and takes T_eq from the context's table
solve (relative error ~1e-7 in T); the level spacing depends on T_eq through
E_g(T_eq), whose logarithmic derivative theta/T reaches ~50 for cold grains,
so dE agrees to ~5e-6 and is held to 1e-4.  The distribution is a product of
M ratios of FP32 rates (~M 1e-7) on that slightly moved grid: level
probabilities are held to 2e-4 of the largest plus 2e-3 of their own value,
and the emission to 2e-3 in the peak-floored relative metric."""
import numpy as np
import pytest

import synth
from metrics import l_err
from oracle import fluct as ofl
from synth.workloads import heat_capacity_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_DE, TOL_P_ABS, TOL_P_REL, TOL_L = 1e-4, 2e-4, 2e-3, 2e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()


def _workload(cells, K=64, n_sizes=6, a_um=(0.0006, 0.02), log10U=(-3.0, 5.0), seed=21,
              species=("silicate", "graphite")):
    cfg = dict(synth.CONFIGS[0])
    cfg.update(K=K, n_sizes=n_sizes, species=species, a_um=a_um, n_cells=cells, log10U=log10U, seed=seed)
    wl = synth.make_workload(cfg)
    N, th = heat_capacity_params(species, wl.sp_of_g, wl.a_of_g)
    return wl, N, th


def _gpu(wl, grains, N, th, M, J=None, precision="fp32"):
    from paper_0907_3768_gb300 import Context, padded_rows

    J = wl.J if J is None else J
    with Context.from_workload(wl, precision=precision) as ctx:
        ctx.set_fluctuating(grains, N[grains], th[grains], M)
        Jd = padded_rows(torch.from_numpy(np.ascontiguousarray(J)).cuda())
        n_f = torch.from_numpy(np.ascontiguousarray(wl.n[:, grains])).cuda()
        o = ctx.solve_fluct(Jd, n_f, want_P=True)
        torch.cuda.synchronize()
        assert ctx.check() == 0
        return {k: v.cpu().numpy() for k, v in o.items()}


def _compare(g, ref, K):
    np.testing.assert_allclose(g["dE"], ref["dE"], rtol=TOL_DE)
    P, Pr = g["P"], ref["P"]
    bound = TOL_P_ABS * Pr.max(axis=2, keepdims=True) + TOL_P_REL * Pr
    assert (np.abs(P - Pr) <= bound).all(), float((np.abs(P - Pr) / np.maximum(bound, 1e-300)).max())
    assert l_err(g["L"][:, :K], ref["L"]).max() <= TOL_L


@pytest.mark.parametrize("M", [32, 64, 128])
def test_fluct_matches_oracle(M):
    wl, N, th = _workload(40)
    grains = np.arange(wl.G)
    g = _gpu(wl, grains, N, th, M)
    ref = ofl.run(wl.lam, wl.w, wl.C_abs, wl.J, wl.n[:, grains], grains, N[grains], th[grains], M,
                  wl.T_min, wl.T_max)
    _compare(g, ref, wl.K)


@pytest.mark.parametrize("K,M", [(300, 64), (48, 32), (130, 256)])
def test_fluct_wavelength_passes(K, M):
    """Whole 256-wavelength passes, 1-3 pairs per lane, and the last < 64
    wavelengths with the levels split between 1 to 8 lanes."""
    wl, N, th = _workload(8, K=K, n_sizes=3)
    grains = np.arange(wl.G)
    g = _gpu(wl, grains, N, th, M)
    ref = ofl.run(wl.lam, wl.w, wl.C_abs, wl.J, wl.n[:, grains], grains, N[grains], th[grains], M,
                  wl.T_min, wl.T_max)
    _compare(g, ref, wl.K)


def test_fluct_many_levels_and_ragged_grain_count():
    """M = 512 (16 levels per lane), 13 grains over 7 warps, odd K."""
    wl, N, th = _workload(6, K=37, n_sizes=7, species=("silicate", "graphite"))
    grains = np.array([0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 13])
    g = _gpu(wl, grains, N, th, 512)
    ref = ofl.run(wl.lam, wl.w, wl.C_abs, wl.J, wl.n[:, grains], grains, N[grains], th[grains], 512,
                  wl.T_min, wl.T_max)
    _compare(g, ref, wl.K)


@pytest.mark.parametrize("C,M,off,species,n_sizes", [
    (1, 64, 50, ("silicate", "graphite"), 6), (7, 64, 50, ("silicate", "graphite"), 6),
    (333, 64, 50, ("silicate", "graphite"), 6), (333, 64, 51, ("silicate", "graphite"), 6),
    (1, 128, 51, ("silicate", "graphite"), 6), (6, 128, 51, ("silicate", "graphite"), 6),
    (5, 128, 51, ("silicate", "graphite", "pah"), 12), (8, 128, 50, ("silicate", "graphite", "pah"), 12)])
def test_fluct_cell_results_independent_of_batch(C, M, off, species, n_sizes):
    """A cell's results do not depend on the batch around it: cells at odd
    and even offsets, at 64 and 128 levels, with 12 and 36 grains, equal the
    same cells inside a larger batch, bit for bit."""
    from paper_0907_3768_gb300 import Context, padded_rows

    wl, N, th = _workload(400, species=species, n_sizes=n_sizes)
    grains = np.arange(wl.G)
    with Context.from_workload(wl) as ctx:
        ctx.set_fluctuating(grains, N, th, M)
        J = padded_rows(torch.from_numpy(wl.J).cuda())
        n_f = torch.from_numpy(np.ascontiguousarray(wl.n)).cuda()
        a = {k: v.cpu().numpy() for k, v in ctx.solve_fluct(J, n_f, want_P=True).items()}
        b = {k: v.cpu().numpy() for k, v in ctx.solve_fluct(J[off:off + C], n_f[off:off + C], want_P=True).items()}
    for k in ("L", "P", "dE"):
        np.testing.assert_array_equal(a[k][off:off + C], b[k])


def test_fluct_benchmark_grain_count_against_oracle():
    """36 grains at 128 levels (the benchmark's shape: 8 problem slots, so
    the fifth pass over the grains is half full) on an odd cell count,
    element by element against the oracle."""
    wl, N, th = _workload(9, species=("silicate", "graphite", "pah"), n_sizes=12)
    grains = np.arange(wl.G)
    assert len(grains) == 36
    g = _gpu(wl, grains, N, th, 128)
    ref = ofl.run(wl.lam, wl.w, wl.C_abs, wl.J, wl.n[:, grains], grains, N[grains], th[grains], 128,
                  wl.T_min, wl.T_max)
    _compare(g, ref, wl.K)


def test_fluct_energy_balance():
    """sum_k w_k L_k = sum_g n 4 pi A (1 - clipped): the emitted power of the
    distributions is the absorbed power less what the top level loses."""
    wl, N, th = _workload(60, K=120)
    grains = np.arange(wl.G)
    g = _gpu(wl, grains, N, th, 128)
    ref = ofl.run(wl.lam, wl.w, wl.C_abs, wl.J, wl.n[:, grains], grains, N, th, 128, wl.T_min, wl.T_max,
                  want_P=False)
    emitted = g["L"][:, :wl.K].astype(np.float64) @ wl.w
    absorbed = (wl.n * ref["heat"] * (1.0 - ref["clipped"])).sum(axis=1)
    np.testing.assert_allclose(emitted, absorbed, rtol=1e-3)


def test_fluct_degenerate_fields():
    """No field: the grain sits in level 0 and emits nothing.  NaN field:
    NaN outputs for that cell only.  A huge field: finite, normalised."""
    wl, N, th = _workload(4, K=48)
    grains = np.arange(wl.G)
    J = wl.J.copy()
    J[0] = 0.0
    J[1, 5] = np.nan
    J[2] *= np.float32(1e12)
    g = _gpu(wl, grains, N, th, 64, J=J)
    assert (g["P"][0][:, 0] == 1.0).all() and (g["P"][0][:, 1:] == 0.0).all()
    assert (g["L"][0, :wl.K] == 0.0).all()
    assert np.isnan(g["P"][1]).all() and np.isnan(g["dE"][1]).all() and np.isnan(g["L"][1, :wl.K]).all()
    for c in (2, 3):
        assert np.isfinite(g["P"][c]).all() and np.isfinite(g["L"][c, :wl.K]).all()
        np.testing.assert_allclose(g["P"][c].sum(axis=1), 1.0, rtol=1e-5)
    ref = ofl.run(wl.lam, wl.w, wl.C_abs, J[[2, 3]], wl.n[[2, 3]], grains, N, th, 64, wl.T_min, wl.T_max)
    _compare({k: v[[2, 3]] for k, v in g.items()}, ref, wl.K)


def test_fluct_any_context_precision():
    """The method runs in FP32 whatever the context's GEMM precision."""
    wl, N, th = _workload(30)
    grains = np.arange(wl.G)
    a = _gpu(wl, grains, N, th, 64, precision="fp32")
    b = _gpu(wl, grains, N, th, 64, precision="bf16x3")
    for k in ("L", "P", "dE"):
        np.testing.assert_array_equal(a[k], b[k])


def test_fluct_full_size_sampled():
    """The benchmark's launch: 2^18 cells of the 200-wavelength, 96-grain
    workload with its 36 grains of 0.5-10 nm on 128 levels; sampled cells
    against the oracle, every cell normalised and finite."""
    from paper_0907_3768_gb300 import Context, padded_rows

    wl = synth.make_workload(1)
    grains = synth.fluctuating_selection(wl.a_of_g)
    N, th = heat_capacity_params(synth.CONFIGS[1]["species"], wl.sp_of_g, wl.a_of_g)
    with Context.from_workload(wl) as ctx:
        ctx.set_fluctuating(grains, N[grains], th[grains], 128)
        J = padded_rows(torch.from_numpy(wl.J).cuda())
        n_f = torch.from_numpy(np.ascontiguousarray(wl.n[:, grains])).cuda()
        o = ctx.solve_fluct(J, n_f, want_P=True)
        torch.cuda.synchronize()
        assert ctx.check() == 0
        assert bool(torch.isfinite(o["P"]).all()) and bool(torch.isfinite(o["L"][:, :wl.K]).all())
        z = o["P"].sum(dim=2)
        assert float((z - 1).abs().max()) < 1e-5
        rng = np.random.default_rng(5)
        cells = np.sort(rng.choice(wl.J.shape[0], 4, replace=False))
        g = {k: o[k][torch.from_numpy(cells).cuda()].cpu().numpy() for k in ("L", "P", "dE")}
    ref = ofl.run(wl.lam, wl.w, wl.C_abs, wl.J[cells], wl.n[cells][:, grains], grains, N[grains], th[grains], 128,
                  wl.T_min, wl.T_max)
    _compare(g, ref, wl.K)


def test_fluct_rejects_bad_arguments():
    """Argument errors come back as DUST_EINVAL before any launch."""
    from paper_0907_3768_gb300 import Context, _lib

    wl, N, th = _workload(4)
    with Context.from_workload(wl) as ctx:
        J = torch.from_numpy(wl.J).cuda()
        with pytest.raises(_lib.DustError):  # before dust_ctx_set_fluctuating
            _lib.dust_solve_fluct(ctx.handle, 4, J.data_ptr(), wl.K, J.data_ptr(), None, None, None, None)
        for grains, na, t, M in (([0], [50.0], [500.0], 100),      # M not a power of two in range
                                 ([0], [50.0], [500.0], 1024),
                                 ([wl.G], [50.0], [500.0], 64),    # grain index out of range
                                 ([0], [0.0], [500.0], 64),        # no atoms
                                 ([0], [50.0], [-1.0], 64)):       # negative theta
            with pytest.raises(_lib.DustError) as e:
                ctx.set_fluctuating(grains, na, t, M)
            assert e.value.code == _lib.DUST_EINVAL
        ctx.set_fluctuating([0, 1], N[:2], th[:2], 64)
        with pytest.raises(ValueError):  # n_f of the wrong width
            ctx.solve_fluct(J, torch.zeros((4, 3), dtype=torch.float32, device="cuda"))
        with pytest.raises(_lib.DustError):  # ld < K
            _lib.dust_solve_fluct(ctx.handle, 4, J.data_ptr(), wl.K - 1, J.data_ptr(), None, None, None, None)
