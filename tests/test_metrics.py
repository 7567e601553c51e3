"""The parity tests' own helpers, on the CPU."""
import numpy as np
import pytest

import oracle
import synth
from metrics import assert_flags_match, l_err, t_err


def test_flag_mismatch_tolerated_only_at_the_bracket_ends():
    wl = synth.make_workload(0, cells=np.arange(2))
    G = wl.G
    P0 = np.array([oracle.power(wl.lam, wl.w, wl.C_abs[g], wl.T_min) for g in range(G)])
    A = np.vstack([P0 * (1 + 2e-6), P0 * 1.5])  # row 0 at the lower end, row 1 well inside
    ref = {"A": A, "flags": np.zeros((2, G), np.uint8)}
    fl = ref["flags"].copy()
    fl[0, 3] = 1  # FP32 put a grain at the lower end just outside: tolerated
    assert assert_flags_match(fl, ref, wl) == 1
    fl[1, 5] = 1  # a grain well inside the bracket flagged: not tolerated
    with pytest.raises(AssertionError):
        assert_flags_match(fl, ref, wl)


def test_error_metrics():
    T_ref = np.array([[10.0, 20.0], [30.0, 40.0]])
    flags = np.array([[0, 1], [0, 0]], np.uint8)
    e = t_err(T_ref * (1 + 1e-6), T_ref, flags)
    assert e.shape == (3,) and np.allclose(e, 1e-6)
    L_ref = np.array([[1.0, 1e-9, 0.5]])
    L = L_ref * np.array([[1.0, 2.0, 1.0]])  # a 100 % error far below the 1e-6 peak floor
    assert l_err(L, L_ref).max() == pytest.approx(1e-9 / 1e-6)
