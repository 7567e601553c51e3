"""Seeded random shapes through every kernel layout, against the FP64 oracle.

Each case draws a wavelength count, a grain set, a cell count and a precision,
so that tile sizes, grain passes, GEMM orientations and padding land on values
the fixed-shape tests do not: K from 2 to 700, 1 to 60 sizes of 1 to 3
species, 1 to 2500 cells.  The default path is checked against the oracle
within the stated tolerances; the two-kernel solve + emission and the fused
absorption + solve (tensor-core precisions) must reproduce it bit for bit."""
import numpy as np
import pytest

import oracle
import synth
from metrics import assert_flags_match, l_err, t_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": (1e-5, 1e-4), "bf16x3": (1e-3, 5e-3), "fp16x3": (1e-3, 5e-3)}
SPECIES = ("silicate", "graphite", "pah")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()


def _draw(seed):
    rng = np.random.default_rng(7000 + seed)
    K = int(rng.integers(2, 701)) if seed % 3 else int(rng.integers(2, 40))
    n_species = int(rng.integers(1, 4))
    species = tuple(rng.choice(SPECIES, n_species, replace=False))
    sizes = int(rng.integers(1, 61))
    C = int(np.exp(rng.uniform(0.0, np.log(2500.0))))
    prec = ("fp32", "bf16x3", "fp16x3")[seed % 3]
    lam = (0.09, 1000.0) if K > 8 else (5.0, 200.0)  # a short grid sits in the mid-infrared
    cfg = dict(synth.CONFIGS[0])
    cfg.update(K=K, n_sizes=sizes, species=species, n_cells=C, seed=8000 + seed, lam_um=lam)
    return synth.make_workload(cfg), prec


@pytest.mark.parametrize("seed", range(12))
def test_random_shape(seed):
    from paper_0907_3768_gb300 import Context, padded_rows

    wl, prec = _draw(seed)
    ref = oracle.run_workload(wl)
    outs = {}
    with Context.from_workload(wl, precision=prec) as ctx:
        J = padded_rows(torch.from_numpy(wl.J).cuda())
        n = torch.from_numpy(wl.n).cuda()
        layouts = [("default", {}), ("two_kernel", {"fused_emit": False})]
        if prec != "fp32":
            layouts.append(("absorb_solve", {"fused": True, "fused_emit": False}))
        for name, opts in layouts:
            ctx.set_fused(opts.get("fused", False))
            ctx.set_fused_emit(opts.get("fused_emit", True))
            o = ctx.solve(J, n, precision=prec)
            torch.cuda.synchronize()
            assert ctx.check() == 0, name
            outs[name] = {k: o[k].cpu().numpy() for k in ("T", "flags", "L", "resid")}
    base = outs["default"]
    for name, o in outs.items():
        for k in ("T", "flags", "L"):
            np.testing.assert_array_equal(o[k], base[k], err_msg=f"{name} {k}")
        if name == "absorb_solve":  # sums the absorbed power in another order
            assert np.abs(o["resid"] - base["resid"]).max() <= 1e-6
        else:
            np.testing.assert_array_equal(o["resid"], base["resid"], err_msg=name)
    tT, tL = TOL[prec]
    assert_flags_match(base["flags"], ref, wl)
    assert t_err(base["T"], ref["T"], ref["flags"]).max(initial=0.0) <= tT
    assert l_err(base["L"], ref["L"]).max() <= tL
