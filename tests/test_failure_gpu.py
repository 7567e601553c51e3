"""Failure detection on the GPU without a GPU fault: the bounded mbarrier wait
that guards every pipeline hand-off of the tensor-core absorption kernel must
give up on a phase that never completes, report DUST_ETIMEOUT through the
status word, and leave the device usable."""
import numpy as np
import pytest

import oracle
import synth
from metrics import t_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()


def test_bounded_wait_gives_up_and_reports_timeout():
    from paper_0907_3768_gb300 import _lib

    st, ms = _lib.dust_diag_wait_timeout(0, 20.0)
    assert st == _lib.DUST_ETIMEOUT
    assert 19.0 <= ms <= 500.0  # the limit, plus the check interval and scheduling slack


def test_device_usable_after_a_timed_out_wait():
    from paper_0907_3768_gb300 import Context, _lib

    st, _ = _lib.dust_diag_wait_timeout(0, 5.0)
    assert st == _lib.DUST_ETIMEOUT
    wl = synth.make_workload(0, cells=np.arange(300))
    ref = oracle.run_workload(wl)
    with Context.from_workload(wl, precision="bf16x3") as ctx:
        out = ctx.solve(torch.from_numpy(wl.J).cuda().contiguous(), torch.from_numpy(wl.n).cuda())
        torch.cuda.synchronize()
        assert ctx.check() == 0  # the context's own status word is untouched
        assert t_err(out["T"].cpu().numpy(), ref["T"], ref["flags"]).max() <= 1e-3
