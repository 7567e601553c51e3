"""Self-absorbing solve (dust_solve_coupled) against the oracle's FP64 fixed
point of J = J_ext + E L.

The coupling is E[c,k] = f_c / (4 pi sum_g n[c,g] C[g,k]) with f_c < 1: a
fraction f_c of a cell's absorbed power is its own re-absorbed emission, so
the iteration contracts at about f_c per pass."""
import math

import numpy as np
import pytest

import oracle
import synth
from metrics import assert_flags_match, l_err, t_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": (1e-5, 1e-4), "bf16x3": (1e-3, 5e-3)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()


def _coupling(wl, fmax, seed):
    f = np.random.default_rng(seed).uniform(0.0, fmax, len(wl.cells))
    kappa = wl.n.astype(np.float64) @ wl.C_abs  # [C, K]
    return (f[:, None] / (4.0 * math.pi * kappa)).astype(np.float32)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_coupled_matches_oracle_fixed_point(prec):
    from paper_0907_3768_gb300 import Context

    wl = synth.make_workload(0, cells=np.arange(300))
    E = _coupling(wl, 0.6, 5)
    ref, it_ref, _ = oracle.run_coupled(wl.lam, wl.w, wl.C_abs, wl.J, E, wl.n, wl.T_min, wl.T_max)
    with Context.from_workload(wl, precision=prec) as ctx:
        out, it, ch = ctx.solve_coupled(torch.from_numpy(wl.J).cuda(), torch.from_numpy(E).cuda(),
                                        torch.from_numpy(wl.n).cuda(), max_iters=200, tol=1e-6)
        torch.cuda.synchronize()
        assert ctx.check() == 0
    assert ch <= 1e-6 and it <= 200
    T, L = out["T"].cpu().numpy(), out["L"].cpu().numpy()
    assert_flags_match(out["flags"].cpu().numpy(), ref, wl)
    tT, tL = TOL[prec]
    assert t_err(T, ref["T"], ref["flags"]).max() <= tT
    assert l_err(L, ref["L"]).max() <= tL
    assert np.abs(out["resid"].cpu().numpy()).max() <= 2e-4
    # the coupling heated the dust: some cells are warmer than without it
    plain = oracle.run_workload(wl, want_L=False, want_resid=False)
    assert (ref["T"] > plain["T"] * 1.01).any()


def test_zero_coupling_is_the_plain_solve():
    from paper_0907_3768_gb300 import Context

    wl = synth.make_workload(0, cells=np.arange(200))
    J, n = torch.from_numpy(wl.J).cuda(), torch.from_numpy(wl.n).cuda()
    with Context.from_workload(wl, precision="fp32") as ctx:
        plain = ctx.solve(J, n)
        out, it, ch = ctx.solve_coupled(J, torch.zeros_like(J), n)
        torch.cuda.synchronize()
    assert it == 2 and ch == 0.0
    for k in ("T", "L", "resid", "flags"):
        assert torch.equal(out[k], plain[k]), k


def test_coupled_rejects_bad_arguments():
    from paper_0907_3768_gb300 import Context, DustError

    wl = synth.make_workload(0, cells=np.arange(8))
    J, n = torch.from_numpy(wl.J).cuda(), torch.from_numpy(wl.n).cuda()
    with Context.from_workload(wl) as ctx:
        with pytest.raises(DustError):
            ctx.solve_coupled(J, torch.zeros_like(J), n, max_iters=0)
        with pytest.raises(ValueError):
            ctx.solve_coupled(J, torch.zeros((8, wl.K + 1), device="cuda")[:, :wl.K], n)
