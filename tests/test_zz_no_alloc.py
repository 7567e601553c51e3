"""The allocation-free entry point (dust_solve_noalloc) against dust_solve.

Some callers cannot allocate device memory (their device memory belongs to a
host framework's pool, or a real-time loop cannot take cudaMalloc's implicit
synchronisation); dust_solve_noalloc serves them with a fixed scratch array
in the library's device data.  Here it must reproduce dust_solve on two calls
in a row with different batches (the second call reuses the array the first
one left behind), and refuse a batch larger than its array.  This file is
named so that pytest collects it last.
"""
import numpy as np
import pytest

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


def _noalloc(ctx, J, n):
    from paper_0907_3768_gb300 import _lib

    C, ld = J.shape[0], J.stride(0)
    out = ctx.alloc_outputs(C, ld)
    _lib.dust_solve_noalloc(ctx.handle, C, J.data_ptr(), ld, n.data_ptr(), out["T"].data_ptr(),
                            out["L_buf"].data_ptr(), out["resid"].data_ptr(), out["flags"].data_ptr(),
                            torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_noalloc_matches_dust_solve_on_two_calls(prec):
    from paper_0907_3768_gb300 import Context, _lib

    wl = synth.make_workload(1, cells=np.arange(60000))
    J = torch.from_numpy(wl.J).cuda()
    n = torch.from_numpy(wl.n).cuda()
    with Context.from_workload(wl, precision=prec) as ctx:
        big = min(50000, _lib.dust_noalloc_max_cells(ctx.handle))  # as large as the array allows
        batches = [(J[:big], n[:big]), (J[13:21013], n[13:21013])]  # second call: other cells, fewer of them
        for Jb, nb in batches:
            ref = ctx.solve(Jb, nb)
            torch.cuda.synchronize()
            got = _noalloc(ctx, Jb, nb)
            # the same kernels' arithmetic on the same inputs: bitwise equal
            # (a scratch-layout mistake would show here, where a tolerance could hide it)
            for k in ("T", "L", "resid", "flags"):
                np.testing.assert_array_equal(got[k].cpu().numpy(), ref[k].cpu().numpy())
            assert t_err(got["T"].cpu().numpy(), ref["T"].cpu().numpy().astype(np.float64)).max() == 0.0
        assert ctx.check() == 0


def _al16(b):
    return (b + 15) // 16 * 16


def _scratch_bytes(C, G, K):
    """Scratch of C cells: absorbed powers [C][Gs], (1/T, n) pairs [C][G8], 16-byte cell records,
    residual partials [C][NKG] float2, the emission order [C] int32, the cells' classes [C] uint16
    and 2 x 1024 class counts, each array rounded up to 16 bytes."""
    Gs, G8, NKG = -(-G // 16) * 16, -(-G // 8) * 8, -(-K // 8)
    return (_al16(4 * C * Gs) + _al16(8 * C * G8) + 16 * C + _al16(8 * C * NKG) + _al16(4 * C) + _al16(2 * C)
            + 2 * 1024 * 4)


def test_noalloc_rejects_batches_beyond_its_array():
    from paper_0907_3768_gb300 import Context, DustError, _lib

    wl = synth.make_workload(0, cells=np.arange(4))
    with Context.from_workload(wl) as ctx:
        cap = _lib.dust_noalloc_max_cells(ctx.handle)
        # G = 16 grains, K = 64: 278 B per cell, plus the class counts
        assert _scratch_bytes(cap, wl.G, wl.K) <= (64 << 20) < _scratch_bytes(cap + 1, wl.G, wl.K)
        assert cap == 241369
        # buffers sized for cap + 1 cells, so that the call would stay in bounds
        # even if the check let it through; refused with and without outputs
        out = ctx.alloc_outputs(cap + 1, wl.K)
        J = torch.zeros((cap + 1, wl.K), device="cuda")
        n = torch.zeros((cap + 1, wl.G), device="cuda")
        for L, resid in ((out["L_buf"].data_ptr(), out["resid"].data_ptr()), (0, 0)):
            with pytest.raises(DustError) as e:
                _lib.dust_solve_noalloc(ctx.handle, cap + 1, J.data_ptr(), wl.K, n.data_ptr(), out["T"].data_ptr(),
                                        L, resid, 0, 0)
            assert e.value.code == _lib.DUST_EINVAL and "split the batch" in str(e.value)
        torch.cuda.synchronize()
