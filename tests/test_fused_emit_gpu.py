"""Temperature solve and emission in one warp-specialized kernel (solver warps
solve the next tile of cells into shared memory while emission warps emit the
current one, Eqs. 7-10) against the two-kernel path and the FP64 oracle.

The solver warps run the stand-alone solve's per-cell code and the emission
warps the emission kernel's arithmetic in its order, so T, the flags, L and
the residual must be bitwise equal."""
import numpy as np
import pytest

import oracle
import synth
from metrics import assert_flags_match, l_err, t_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": (1e-5, 1e-4), "bf16x3": (1e-3, 5e-3), "fp16x3": (1e-3, 5e-3)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()


def _both(wl, prec, J=None, **kw):
    from paper_0907_3768_gb300 import Context, padded_rows

    J = wl.J if J is None else J
    out = {}
    with Context.from_workload(wl, precision=prec) as ctx:
        Jd = padded_rows(torch.from_numpy(np.ascontiguousarray(J)).cuda())
        n = torch.from_numpy(wl.n).cuda()
        for fused in (False, True):
            ctx.set_fused_emit(fused)
            o = ctx.solve(Jd, n, precision=prec, **kw)
            torch.cuda.synchronize()
            assert ctx.check() == 0
            out[fused] = {k: v.cpu().numpy() for k, v in o.items() if v is not None}
    return out[False], out[True]


def _same(two, one):
    """Every output the call asked for (L without its unwritten padding columns)."""
    assert two.keys() == one.keys()
    for k in ("T", "flags", "L", "resid"):
        if k in two:
            np.testing.assert_array_equal(one[k], two[k], err_msg=k)


def _shape(K, sizes, species, lam_um, C, seed):
    cfg = dict(synth.CONFIGS[0])
    cfg.update(K=K, n_sizes=sizes, species=species, n_cells=C, seed=seed, lam_um=lam_um)
    return synth.make_workload(cfg)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "fp16x3"])
@pytest.mark.parametrize("case", ["tiny", "bench-G96", "odd-K37-G5", "K2-G1", "G128", "K2048-G512"])
def test_fused_emit_equals_two_kernel_path_and_oracle(prec, case):
    """Tiles of 64, 20 and 39 cells; one to four grain passes per lane; the
    last case does not fit shared memory and must fall back to two kernels."""
    wl = {
        "tiny": lambda: synth.make_workload(0, cells=np.arange(1000)),
        "bench-G96": lambda: synth.make_workload(1, cells=np.arange(3001)),
        "odd-K37-G5": lambda: _shape(37, 5, ("silicate",), (0.09, 1000.0), 300, 77),
        "K2-G1": lambda: _shape(2, 1, ("graphite",), (5.0, 200.0), 49, 91),
        "G128": lambda: _shape(100, 64, ("silicate", "graphite"), (0.09, 1000.0), 513, 123),
        "K2048-G512": lambda: _shape(2048, 256, ("silicate", "graphite"), (0.09, 1000.0), 49, 91),
    }[case]()
    two, one = _both(wl, prec)
    _same(two, one)
    ref = oracle.run_workload(wl)
    tT, tL = TOL[prec]
    assert_flags_match(one["flags"], ref, wl)
    assert t_err(one["T"], ref["T"], ref["flags"]).max(initial=0.0) <= tT
    assert l_err(one["L"], ref["L"]).max() <= tL


@pytest.mark.parametrize("C", [1, 19, 20, 21, 152 * 20 + 7, 40000])
def test_fused_emit_ragged_cell_counts(C):
    """Partial last tiles, fewer tiles than SMs, and many tiles per CTA."""
    wl = synth.make_workload(1, cells=np.arange(C))
    two, one = _both(wl, "bf16x3")
    _same(two, one)


@pytest.mark.parametrize("want_L,want_resid", [(False, True), (True, False), (False, False)])
def test_fused_emit_output_modes(want_L, want_resid):
    """Residual only, L only, and T only (no emission: the kernel does not apply)."""
    wl = synth.make_workload(1, cells=np.arange(2000))
    two, one = _both(wl, "bf16x3", want_L=want_L, want_resid=want_resid)
    _same(two, one)


def test_fused_emit_edge_inputs():
    wl = synth.make_workload(0, cells=np.arange(8))
    J = wl.J.copy()
    J[0] = 0.0
    J[1] *= np.float32(1e25)
    J[2, 7] = np.nan
    J[3] *= np.float32(1e-30)
    two, one = _both(wl, "fp32", J=J)
    _same(two, one)
    assert (one["flags"][2] == 4).all()


def test_fused_emit_cell_results_independent_of_batch():
    from paper_0907_3768_gb300 import Context, padded_rows

    wl = synth.make_workload(1, cells=np.arange(3000))
    with Context.from_workload(wl, precision="bf16x3") as ctx:
        ctx.set_fused_emit(True)
        J = padded_rows(torch.from_numpy(wl.J).cuda())
        n = torch.from_numpy(wl.n).cuda()
        a = {k: v.cpu().numpy() for k, v in ctx.solve(J, n).items()}
        b = {k: v.cpu().numpy() for k, v in ctx.solve(J[1234:2345], n[1234:2345]).items()}
    for k in ("T", "L", "resid", "flags"):
        np.testing.assert_array_equal(a[k][1234:2345], b[k])


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_fused_emit_mass_form(prec):
    """The dust-mass form n[c,g] = n_g m_c (Eqs. 9-10): 1/T-only pairs, the
    weights carrying n_g, L scaled by the cell's mass; dust-free cells too."""
    from paper_0907_3768_gb300 import Context, padded_rows

    wl = synth.make_workload(1, cells=np.arange(2500))
    rng = np.random.default_rng(3)
    n_g = wl.n[0].astype(np.float64) * np.exp(rng.normal(0.0, 1.0, wl.G))
    m = np.exp(rng.normal(0.0, 2.0, 2500)).astype(np.float32)
    m[::41] = 0.0
    out = {}
    with Context.from_workload(wl, precision=prec) as ctx:
        ctx.set_grain_numbers(n_g)
        J = padded_rows(torch.from_numpy(wl.J).cuda())
        for fused in (False, True):
            ctx.set_fused_emit(fused)
            o = ctx.solve_mass(J, torch.from_numpy(m).cuda())
            torch.cuda.synchronize()
            assert ctx.check() == 0
            out[fused] = {k: v.cpu().numpy() for k, v in o.items() if v is not None}
    _same(out[False], out[True])
    n_full = m.astype(np.float64)[:, None] * n_g[None, :]
    ref = oracle.run(wl.lam, wl.w, wl.C_abs, wl.J, n_full, wl.T_min, wl.T_max)
    dusty = m > 0
    assert l_err(out[True]["L"][dusty], ref["L"][dusty]).max() <= TOL[prec][1]

