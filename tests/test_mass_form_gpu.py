"""The dust-mass form n[c,g] = n_g m_c (the paper's n_s m_d;c, Eqs. 9-10)
against the oracle and against the general path on the same grain numbers."""
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


def _rank1(wl, seed):
    rng = np.random.default_rng(seed)
    n_g = wl.n[0].astype(np.float64) * np.exp(rng.normal(0.0, 1.0, wl.G))  # some spread across grains
    m = np.exp(rng.normal(0.0, 2.0, len(wl.cells))).astype(np.float32)
    m[::37] = 0.0  # dust-free cells
    return n_g, m


@pytest.mark.parametrize("cfg,cells,prec", [(0, 1024, "fp32"), (1, 3000, "bf16x3"), (3, 400, "bf16x3")])
def test_mass_form_matches_oracle_and_general_path(cfg, cells, prec):
    from paper_0907_3768_gb300 import Context, padded_rows

    wl = synth.make_workload(cfg, cells=np.arange(cells))
    n_g, m = _rank1(wl, cfg)
    n_full = (m.astype(np.float64)[:, None] * n_g[None, :])
    ref = oracle.run(wl.lam, wl.w, wl.C_abs, wl.J, n_full, wl.T_min, wl.T_max)
    with Context.from_workload(wl, precision=prec) as ctx:
        ctx.set_grain_numbers(n_g)
        J = padded_rows(torch.from_numpy(wl.J).cuda())
        got = ctx.solve_mass(J, torch.from_numpy(m).cuda())
        gen = ctx.solve(J, torch.from_numpy(n_full.astype(np.float32)).cuda())
        torch.cuda.synchronize()
        assert ctx.check() == 0
    got = {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in got.items()}
    gen = {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in gen.items()}
    np.testing.assert_array_equal(got["T"], gen["T"])  # the same solve
    assert_flags_match(got["flags"], ref, wl)
    tT, tL = TOL[prec]
    assert t_err(got["T"], ref["T"], ref["flags"]).max() <= tT
    dusty = m > 0
    assert l_err(got["L"][dusty], ref["L"][dusty]).max() <= tL
    assert (got["L"][~dusty] == 0).all()
    assert np.abs(got["resid"]).max() <= 2e-4  # per unit mass: defined for dust-free cells too
    assert np.abs(got["resid"][dusty] - ref["resid"][dusty]).max() <= 2e-4


def test_mass_form_needs_grain_numbers():
    from paper_0907_3768_gb300 import Context, DustError, _lib

    wl = synth.make_workload(0, cells=np.arange(8))
    with Context.from_workload(wl) as ctx:
        J = torch.from_numpy(wl.J).cuda()
        m = torch.ones(8, device="cuda")
        with pytest.raises(DustError) as e:
            ctx.solve_mass(J, m)
        assert e.value.code == _lib.DUST_EINVAL
        with pytest.raises(DustError):
            ctx.set_grain_numbers(np.zeros(wl.G))
