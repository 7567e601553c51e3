"""Absorption contraction and temperature solve fused into one kernel (the
accumulator of Eq. 6 is solved for T straight from tensor memory, Eq. 7)
against the two-kernel path and the FP64 oracle.

Both paths run every grain through the same solve arithmetic, so T, the
flags and L must be bitwise equal; the residual sums the cell's absorbed
power in another order and agrees to rounding."""
import numpy as np
import pytest

import oracle
import synth
from metrics import assert_flags_match, l_err, t_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"bf16x3": (1e-3, 5e-3), "fp16x3": (1e-3, 5e-3)}


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
            ctx.set_fused(fused)
            o = ctx.solve(Jd, n, **kw)
            torch.cuda.synchronize()
            assert ctx.check() == 0
            out[fused] = {k: v.cpu().numpy() for k, v in o.items() if v is not None}
    return out[False], out[True]


def _same(two, one):
    for k in ("T", "flags", "L"):
        if k in two:
            np.testing.assert_array_equal(one[k], two[k], err_msg=k)
    if "resid" in two:
        assert np.abs(one["resid"] - two["resid"]).max() <= 1e-6


def _shape(K, sizes, species, lam_um, C, seed):
    cfg = dict(synth.CONFIGS[0])
    cfg.update(K=K, n_sizes=sizes, species=species, n_cells=C, seed=seed, lam_um=lam_um)
    return synth.make_workload(cfg)


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3"])
@pytest.mark.parametrize("case", ["tiny", "bench-G96", "large-G240", "odd-K37-G5", "K2048-G512", "K2-G1"])
def test_fused_equals_two_kernel_path_and_oracle(prec, case):
    """One accumulator per group of solver warps: four at G <= 128, two at
    G = 240, one at G = 512; ragged last tiles; G not a multiple of 4."""
    wl = {
        "tiny": lambda: synth.make_workload(0, cells=np.arange(1000)),
        "bench-G96": lambda: synth.make_workload(1, cells=np.arange(3001)),
        "large-G240": lambda: synth.make_workload(3, cells=np.arange(700)),
        "odd-K37-G5": lambda: _shape(37, 5, ("silicate",), (0.09, 1000.0), 300, 77),
        "K2048-G512": lambda: _shape(2048, 256, ("silicate", "graphite"), (0.09, 1000.0), 49, 91),
        "K2-G1": lambda: _shape(2, 1, ("graphite",), (5.0, 200.0), 49, 91),
    }[case]()
    two, one = _both(wl, prec)
    _same(two, one)
    ref = oracle.run_workload(wl)
    tT, tL = TOL[prec]
    assert_flags_match(one["flags"], ref, wl)
    assert t_err(one["T"], ref["T"], ref["flags"]).max(initial=0.0) <= tT
    assert l_err(one["L"], ref["L"]).max() <= tL
    assert np.abs(one["resid"]).max() <= 2e-4


@pytest.mark.parametrize("C", [1, 127, 128, 129, 5000])
def test_fused_ragged_cell_counts(C):
    wl = synth.make_workload(1, cells=np.arange(C))
    two, one = _both(wl, "bf16x3")
    _same(two, one)


@pytest.mark.parametrize("want_L,want_resid", [(False, False), (False, True), (True, False)])
def test_fused_output_modes(want_L, want_resid):
    """T only (no pairs, no n), residual only, L only."""
    wl = synth.make_workload(1, cells=np.arange(2000))
    two, one = _both(wl, "bf16x3", want_L=want_L, want_resid=want_resid)
    _same(two, one)


def test_fused_edge_inputs():
    """Zero, huge, NaN and tiny fields: clamp and invalid flags as in the two-kernel path."""
    wl = synth.make_workload(0, cells=np.arange(8))
    J = wl.J.copy()
    J[0] = 0.0
    J[1] *= np.float32(1e25)
    J[2, 7] = np.nan
    J[3] *= np.float32(1e-30)
    two, one = _both(wl, "bf16x3", J=J)
    np.testing.assert_array_equal(one["flags"], two["flags"])
    np.testing.assert_array_equal(one["T"], two["T"])
    assert (one["flags"][2] == 4).all()
    ok = [0, 1, 3, 4, 5, 6, 7]
    np.testing.assert_array_equal(one["L"][ok], two["L"][ok])


def test_fused_mass_form():
    """The dust-mass form (Eqs. 9-10) through the fused kernel."""
    from paper_0907_3768_gb300 import Context, padded_rows

    wl = synth.make_workload(1, cells=np.arange(2500))
    rng = np.random.default_rng(3)
    n_g = wl.n[0].astype(np.float64) * np.exp(rng.normal(0.0, 1.0, wl.G))
    m = np.exp(rng.normal(0.0, 2.0, 2500)).astype(np.float32)
    m[::41] = 0.0
    out = {}
    with Context.from_workload(wl, precision="bf16x3") as ctx:
        ctx.set_grain_numbers(n_g)
        J = padded_rows(torch.from_numpy(wl.J).cuda())
        for fused in (False, True):
            ctx.set_fused(fused)
            o = ctx.solve_mass(J, torch.from_numpy(m).cuda())
            torch.cuda.synchronize()
            assert ctx.check() == 0
            out[fused] = {k: v.cpu().numpy() for k, v in o.items() if v is not None}
    _same(out[False], out[True])


def test_fused_cell_results_independent_of_batch():
    from paper_0907_3768_gb300 import Context, padded_rows

    wl = synth.make_workload(1, cells=np.arange(3000))
    with Context.from_workload(wl, precision="bf16x3") as ctx:
        ctx.set_fused(True)
        J = padded_rows(torch.from_numpy(wl.J).cuda())
        n = torch.from_numpy(wl.n).cuda()
        a = {k: v.cpu().numpy() for k, v in ctx.solve(J, n).items()}
        b = {k: v.cpu().numpy() for k, v in ctx.solve(J[1234:2345], n[1234:2345]).items()}
    for k in ("T", "L", "resid", "flags"):
        np.testing.assert_array_equal(a[k][1234:2345], b[k])
