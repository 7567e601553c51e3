"""The paper's own temperature kernel (per-iterate quadrature Newton, Eqs. 11-12
guess, 0.1 % stop; Section 4.3), kept as an ablation of the table solve.

Its result is an approximation with a stated error bound, so it is pinned to
that bound: for every solved grain the FP64 oracle's P_g(T) at the kernel's T
must match the oracle's absorbed power A to the paper's 0.1 %, flags must be
the oracle's, and T must lie within what that criterion allows of the
oracle's exact root (d ln P / d ln T >= 4 here, so |dT/T| <= 2.5e-4)."""
import numpy as np
import pytest

import oracle
import synth
from metrics import assert_flags_match

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()


def _solve(wl, prec):
    from paper_0907_3768_gb300 import Context, padded_rows

    with Context.from_workload(wl, precision=prec) as ctx:
        ctx.set_grain_sizes(wl.a_of_g)
        J = padded_rows(torch.from_numpy(wl.J).cuda())
        out = ctx.solve_T_newton(J)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("cfg,cells,prec", [(0, 1024, "fp32"), (0, 1024, "bf16x3"), (1, 250, "bf16x3"),
                                            (3, 60, "bf16x3")])
def test_energy_criterion_holds_for_every_solved_grain(cfg, cells, prec):
    wl = synth.make_workload(cfg, cells=np.arange(cells))
    got = _solve(wl, prec)
    ref = oracle.run_workload(wl, want_L=False, want_resid=False)
    assert_flags_match(got["flags"], ref, wl)
    ok = ref["flags"] == 0
    assert ok.sum() > 0.9 * ok.size or cfg == 3
    worst = 0.0
    for c, g in zip(*np.nonzero(ok)):
        A = oracle.absorbed(wl.w, wl.C_abs[g], wl.J[c].astype(np.float64))
        P = oracle.power(wl.lam, wl.w, wl.C_abs[g], float(got["T"][c, g]))
        worst = max(worst, abs(P / A - 1.0))
    assert worst <= 1.02e-3, worst  # the paper's 0.1 %, plus FP32 evaluation and the GEMM's rounding
    rel = np.abs(got["T"][ok] / ref["T"][ok] - 1.0)
    assert rel.max() <= 2.6e-4
    assert got["iters"].max() <= 64


def test_needs_grain_sizes_and_rejects_bad_ones():
    from paper_0907_3768_gb300 import Context, DustError, _lib

    wl = synth.make_workload(0, cells=np.arange(8))
    with Context.from_workload(wl) as ctx:
        J = torch.from_numpy(wl.J).cuda()
        with pytest.raises(DustError) as e:
            ctx.solve_T_newton(J)
        assert e.value.code == _lib.DUST_EINVAL
        bad = wl.a_of_g.copy()
        bad[3] = -1.0
        with pytest.raises(DustError):
            ctx.set_grain_sizes(bad)
