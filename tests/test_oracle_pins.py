"""Pins of the FP64 oracle against what the physics and the mathematics fix.

Each test checks the oracle against something other than itself: exact SI
constants and their CODATA consequences (Stefan-Boltzmann, Wien displacement),
the analytic limits of Planck's law, closed-form temperatures (blackbody
fields, gray grains), the energy-balance identity that follows from Eqs. 6-10,
scaling invariances, an independent root finder, and 50-digit brute force on
tiny inputs.  A dropped term, a wrong power, sign or index in the oracle fails
at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
import synth

UM = 1e-6


def ext_grid(K=2000, lo=0.01, hi=1.0e6):
    """Extended grid on which the trapezoid rule is exact to ~1e-11 for 20-3000 K."""
    return synth.wavelength_grid(K, lo * UM, hi * UM)


def sigma_closed_form(si):
    h, c, k = si["h"], si["c"], si["k_B"]
    return 2.0 * math.pi ** 5 * k ** 4 / (15.0 * h ** 3 * c ** 2)


def test_sigma_closed_form_matches_codata(si):
    assert sigma_closed_form(si) == pytest.approx(si["sigma_SB"], rel=2e-10)


@pytest.mark.parametrize("T", [20.0, 55.0, 300.0, 1000.0, 3000.0])
def test_stefan_boltzmann_quadrature(si, T):
    """Gray grain with C = 1: P(T) = sum_k w_k B_k(T) must equal sigma T^4 / pi."""
    lam, w = ext_grid()
    P = oracle.power(lam, w, np.ones_like(lam), T)
    assert P == pytest.approx(sigma_closed_form(si) * T ** 4 / math.pi, rel=1e-10)


@pytest.mark.parametrize("T", [3.0, 40.0, 800.0, 3000.0])
def test_wien_displacement(si, T):
    """The maximum of B(lambda, T) over lambda sits at b / T."""
    from scipy.optimize import minimize_scalar

    b = si["b_wien"]
    f = lambda s: -oracle.planck(b / T * math.exp(s), T)  # noqa: E731
    res = minimize_scalar(f, bracket=(-0.2, 0.0, 0.2), tol=1e-12)
    assert abs(res.x) < 3e-8


def test_planck_limits(si):
    h, c, k = si["h"], si["c"], si["k_B"]
    T = 100.0
    # Rayleigh-Jeans: B -> 2 c k T / lambda^4 (1 - x/2 + x^2/12) for x -> 0
    for x in (1e-3, 1e-6):
        lam = h * c / (k * T * x)
        rj = 2.0 * c * k * T / lam ** 4
        assert oracle.planck(lam, T) / rj == pytest.approx(1.0 - x / 2.0 + x * x / 12.0, rel=1e-12)
    # Wien: B -> 2 h c^2 lambda^-5 e^-x for x >> 1
    for x in (40.0, 300.0):
        lam = h * c / (k * T * x)
        wien = 2.0 * h * c * c / lam ** 5 * math.exp(-x)
        assert oracle.planck(lam, T) / wien == pytest.approx(1.0, rel=1e-13)
    # far Wien side underflows to zero, never to NaN / inf
    assert oracle.planck(1e-9, 2.0) == 0.0


def _bb_field(lam, T0, si):
    """B(lambda, T0) built from the input generator's own blackbody (independent code)."""
    return synth.blackbody_shape(lam, T0) * si["sigma_SB"] * T0 ** 4 / math.pi


@pytest.mark.parametrize("cfg", [0, 3])
def test_blackbody_field_returns_its_temperature(si, cfg):
    """J = B(T0) gives A = P_g(T0) for every grain, so T = T0 (any C, any grid)."""
    wl = synth.make_workload(cfg, cells=np.arange(4))
    rng = np.random.default_rng(7)
    T0 = np.exp(rng.uniform(math.log(3.0), math.log(2500.0), 12))
    J = np.stack([_bb_field(wl.lam, t, si) for t in T0])
    n = np.ones((len(T0), wl.G))
    r = oracle.run(wl.lam, wl.w, wl.C_abs, J, n, wl.T_min, wl.T_max)
    assert (r["flags"] == 0).all()
    np.testing.assert_allclose(r["T"], np.repeat(T0[:, None], wl.G, 1), rtol=1e-11)


def test_gray_grain_in_dilute_blackbody(si):
    """Gray C: T = W^(1/4) T* in the field W B(T*), whatever the gray constant."""
    lam, w = ext_grid()
    C = np.array([1e-20, 3.3e-14, 7.0e-9])[:, None] * np.ones((1, len(lam)))
    cases = [(0.3, 120.0), (1e-3, 2000.0), (1e-9, 5000.0), (2.5e-14, 20000.0)]
    J = np.stack([W * _bb_field(lam, Ts, si) for W, Ts in cases])
    r = oracle.run(lam, w, C, J, np.ones((len(cases), 3)), 2.0, 3000.0, want_L=False, want_resid=False)
    expect = np.array([W ** 0.25 * Ts for W, Ts in cases])
    np.testing.assert_allclose(r["T"], np.repeat(expect[:, None], 3, 1), rtol=1e-10)


def test_gray_grain_in_stellar_field(si):
    """Gray C in U J_ISRF x (unit-integral spectrum): T = (pi U J_ISRF / sigma)^(1/4)."""
    lam, w = ext_grid()
    U = np.array([1e2, 1e4, 1e6])  # T = 10-103 K: grid truncation < 1e-10
    J = U[:, None] * synth.workloads.J_ISRF * synth.workloads.stellar_shape(lam)[None, :]
    C = np.full((1, len(lam)), 2e-15)
    r = oracle.run(lam, w, C, J, np.ones((3, 1)), 2.0, 3000.0, want_L=False, want_resid=False)
    expect = (math.pi * U * synth.workloads.J_ISRF / si["sigma_SB"]) ** 0.25
    np.testing.assert_allclose(r["T"][:, 0], expect, rtol=1e-9)


@pytest.mark.parametrize("cfg", [0, 3])
def test_energy_balance(cfg):
    """sum_k w_k L[c,k] = 4 pi sum_g n A for every cell (Eqs. 6, 7, 10)."""
    cells = np.arange(1024) if cfg == 0 else np.arange(0, 1 << 20, 1 << 13)
    wl = synth.make_workload(cfg, cells=cells)
    r = oracle.run_workload(wl)
    assert np.abs(r["resid"]).max() < 1e-12


def test_energy_balance_catches_a_wrong_emission():
    """The residual is a real check: L of the wrong grains breaks it."""
    wl = synth.make_workload(0, cells=np.arange(8))
    r = oracle.run_workload(wl)
    L_bad = np.stack([oracle.emission(wl.lam, wl.C_abs[::-1], wl.n[c], r["T"][c]) for c in range(8)])
    em = L_bad @ wl.w
    ab = 4.0 * math.pi * np.sum(wl.n.astype(np.float64) * r["A"], axis=1)
    assert np.abs(em / ab - 1.0).max() > 1e-3


def test_homogeneity_and_monotonicity():
    wl = synth.make_workload(0, cells=np.arange(16))
    base = oracle.run_workload(wl)
    # n -> s n: L -> s L, T unchanged
    r = oracle.run(wl.lam, wl.w, wl.C_abs, wl.J, 3.0 * wl.n.astype(np.float64), wl.T_min, wl.T_max)
    np.testing.assert_array_equal(r["T"], base["T"])
    np.testing.assert_allclose(r["L"], 3.0 * base["L"], rtol=1e-14)
    # C -> s C: T unchanged (to root tolerance)
    r = oracle.run(wl.lam, wl.w, 7.0 * wl.C_abs, wl.J, wl.n, wl.T_min, wl.T_max)
    np.testing.assert_allclose(r["T"], base["T"], rtol=1e-12)
    # J -> s J, s > 1: T strictly increases for every grain
    r = oracle.run(wl.lam, wl.w, wl.C_abs, 1.5 * wl.J.astype(np.float64), wl.n, wl.T_min, wl.T_max)
    assert (r["T"] > base["T"]).all()


def test_rayleigh_sizes_share_a_temperature():
    """Grains with 2 pi a <= lambda_min have C proportional to a^3, so one T per species."""
    wl = synth.make_workload(1, cells=np.arange(0, 1 << 18, 1 << 12))
    r = oracle.run_workload(wl, want_L=False, want_resid=False)
    small = 2.0 * math.pi * wl.a_of_g <= wl.lam[0]
    for s in np.unique(wl.sp_of_g):
        idx = np.nonzero(small & (wl.sp_of_g == s))[0]
        assert len(idx) >= 4
        T = r["T"][:, idx]
        np.testing.assert_allclose(T, np.repeat(T[:, :1], len(idx), 1), rtol=1e-12)
    # and larger grains differ from them
    big = np.nonzero(~small & (wl.sp_of_g == 0))[0]
    assert np.abs(r["T"][:, big[-1]] / r["T"][:, 0] - 1.0).min() > 1e-3


@pytest.mark.parametrize("cfg", [1, 3])
def test_brent_agrees_with_bisection(cfg):
    wl = synth.make_workload(cfg, cells=np.arange(0, synth.CONFIGS[cfg]["n_cells"], 1 << 14))
    r = oracle.run_workload(wl, want_L=False, want_resid=False)
    rng = np.random.default_rng(3)
    for _ in range(40):
        c = rng.integers(0, len(wl.cells))
        g = rng.integers(0, wl.G)
        if r["flags"][c, g]:
            continue
        Tb = oracle.temperature_bisect(wl.lam, wl.w, wl.C_abs[g], r["A"][c, g], wl.T_min, wl.T_max)
        assert r["T"][c, g] == pytest.approx(Tb, rel=1e-12)


def test_clamps_and_invalid_input():
    wl = synth.make_workload(0, cells=np.arange(3))
    J = wl.J.astype(np.float64)
    J[0] = 0.0                 # nothing absorbed -> T_min, flag 1
    J[1] *= 1e30               # far too hot      -> T_max, flag 2
    J[2, 5] = np.nan           # invalid          -> flag 4, T NaN
    r = oracle.run(wl.lam, wl.w, wl.C_abs, J, wl.n, wl.T_min, wl.T_max)
    assert (r["flags"][0] == 1).all() and (r["T"][0] == wl.T_min).all()
    assert (r["flags"][1] == 2).all() and (r["T"][1] == wl.T_max).all()
    assert (r["flags"][2] == 4).all() and np.isnan(r["T"][2]).all()
    # clamped grains emit at their clamp temperature: energy still balances
    assert abs(r["resid"][0]) < 1e-12 and abs(r["resid"][1]) < 1e-12


def test_mpmath_brute_force_tiny():
    """50-digit evaluation of the definitions on a tiny case (C=3, G=2, K=8)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    lam, w = synth.wavelength_grid(8, 0.1 * UM, 300.0 * UM)
    sp, a = synth.grain_table(("silicate",), 2, 0.01 * UM, 0.3 * UM)
    C = synth.cross_sections(lam, ("silicate",), sp, a)
    J = np.stack([_bb_field(lam, T0, {"sigma_SB": synth.workloads._SIGMA_SB}) * s
                  for T0, s in ((5000.0, 1e-14), (20000.0, 1e-12), (3000.0, 1e-6))])
    n = np.array([[1e20, 1e15], [3e19, 2e14], [1.0, 1.0]])
    h, c, k = mp.mpf("6.62607015e-34"), mp.mpf(299792458), mp.mpf("1.380649e-23")

    def B(l, T):
        return 2 * h * c ** 2 / l ** 5 / (mp.exp(h * c / (k * l * T)) - 1)

    r = oracle.run(lam, w, C, J, n, 2.0, 3000.0)
    for ci in range(3):
        Lref = [mp.mpf(0)] * 8
        for g in range(2):
            A = mp.fsum(mp.mpf(w[i]) * mp.mpf(C[g, i]) * mp.mpf(J[ci, i]) for i in range(8))
            P = lambda T: mp.fsum(mp.mpf(w[i]) * mp.mpf(C[g, i]) * B(mp.mpf(lam[i]), T) for i in range(8))  # noqa: E731
            u = mp.findroot(lambda u: mp.log(P(mp.exp(u))) - mp.log(A), (mp.log(2), mp.log(3000)),
                            solver="anderson")
            T = mp.exp(u)
            assert float(A) == pytest.approx(r["A"][ci, g], rel=1e-14)
            assert float(T) == pytest.approx(r["T"][ci, g], rel=1e-12)
            for i in range(8):
                Lref[i] += mp.mpf(n[ci, g]) * mp.mpf(C[g, i]) * B(mp.mpf(lam[i]), T)
        for i in range(8):
            assert float(4 * mp.pi * Lref[i]) == pytest.approx(r["L"][ci, i], rel=1e-11)


def test_coupled_without_coupling_is_the_plain_solve():
    """E = 0: the self-absorption iteration stops at its second pass with the
    plain result."""
    wl = synth.make_workload(0, cells=np.arange(40))
    plain = oracle.run_workload(wl)
    res, it, ch = oracle.run_coupled(wl.lam, wl.w, wl.C_abs, wl.J, np.zeros_like(wl.J, dtype=np.float64), wl.n,
                                     wl.T_min, wl.T_max)
    assert it == 2 and ch == 0.0
    for k in ("T", "L", "resid"):
        np.testing.assert_array_equal(res[k], plain[k])


def test_coupled_gray_grain_closed_form(si):
    """One gray grain (cross section c, number n) in W B(T*) with a constant
    coupling e: absorbed c (J_bol + e sum w L) with sum w L = 4 pi n c sigma T^4 / pi
    equals emitted c sigma T^4 / pi, so T = T* (W / (1 - 4 pi e n c))^(1/4)."""
    lam, w = ext_grid()
    c = 3.0e-14
    Ts, W = 300.0, 1e-3
    J = (W * _bb_field(lam, Ts, si))[None, :]
    for frac in (0.0, 0.3, 0.7):          # 4 pi e n c
        n = np.array([[2.0]])
        e = frac / (4.0 * math.pi * n[0, 0] * c)
        res, it, ch = oracle.run_coupled(lam, w, np.full((1, len(lam)), c), J, np.full_like(J, e), n, 2.0, 3000.0)
        expect = Ts * (W / (1.0 - frac)) ** 0.25
        assert res["T"][0, 0] == pytest.approx(expect, rel=1e-10), (frac, it)
        assert abs(res["resid"][0]) < 1e-10
