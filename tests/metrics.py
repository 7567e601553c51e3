"""Error metrics of the parity tests (shared by the test modules)."""
import numpy as np


def t_err(T, T_ref, flags_ref=None):
    """|T - T*| / T* over grains the oracle solved inside the bracket."""
    T = np.asarray(T, np.float64)
    m = np.ones(T_ref.shape, bool) if flags_ref is None else flags_ref == 0
    if not m.any():
        return np.zeros(0)
    return np.abs(T[m] / T_ref[m] - 1.0)


def l_err(L, L_ref):
    """Peak-floored relative error |L - L*| / max(L*[c,k], 1e-6 max_k L*[c,k]).

    The floor keeps the FP32 underflow of the Wien tail, which the paper shows
    is of no consequence (Section 5.1), from dominating the statistic."""
    L = np.asarray(L, np.float64)
    floor = np.maximum(L_ref, 1e-6 * L_ref.max(axis=1, keepdims=True))
    return np.abs(L - L_ref) / floor


def sed_weighted_ratio(L, L_ref):
    """The paper's accuracy statistic (Section 5.1): per wavelength, the mean over
    cells of L/L* weighted by L*, and its weighted standard deviation."""
    L = np.asarray(L, np.float64)
    w = L_ref
    ws = w.sum(axis=0)
    ok = ws > 0
    ratio = np.where(L_ref > 0, L / np.where(L_ref > 0, L_ref, 1.0), 1.0)
    mean = np.where(ok, (w * ratio).sum(axis=0) / np.where(ok, ws, 1.0), 1.0)
    var = np.where(ok, (w * (ratio - mean) ** 2).sum(axis=0) / np.where(ok, ws, 1.0), 0.0)
    return mean, np.sqrt(var)


def assert_flags_match(flags, ref, wl, band=1e-5):
    """Clamp flags equal to the oracle's, except for grains whose oracle A lies
    within `band` (relative) of P_g(T_min) or P_g(T_max).  There the GPU
    decides in FP32 and the oracle in FP64, and both are right to their
    precision.  Returns the number of such tolerated differences."""
    import oracle

    fl = np.asarray(flags)
    rf = ref["flags"]
    diff = fl != rf
    if not diff.any():
        return 0
    G = wl.C_abs.shape[0]
    P0 = np.array([oracle.power(wl.lam, wl.w, wl.C_abs[g], wl.T_min) for g in range(G)])
    P1 = np.array([oracle.power(wl.lam, wl.w, wl.C_abs[g], wl.T_max) for g in range(G)])
    A = ref["A"]
    with np.errstate(invalid="ignore", divide="ignore"):
        near = (np.abs(A / P0[None, :] - 1.0) < band) | (np.abs(A / P1[None, :] - 1.0) < band)
    bad = diff & ~near
    assert not bad.any(), f"{int(bad.sum())} flags differ away from the bracket ends"
    return int(diff.sum())
