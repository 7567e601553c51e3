"""Pins of the fluctuating-grain oracle (oracle/fluct.py) against what the
mathematics fixes, independent of the oracle's own construction:

* the Einstein enthalpy is the integral of the Einstein heat capacity;
* the cut-flux recursion gives the null vector of the full master equation
  (a dense linear solve), for random and for physical rate matrices;
* each photon's two-level split conserves its energy;
* the steady state balances energy: emitted power = absorbed - clipped;
* large grains converge to the equilibrium temperature at first order in 1/M.
The paper prints no fluctuating-grain values, so nothing is pinned to it."""
import math

import numpy as np
import pytest

import synth
from oracle import fluct
from synth.workloads import heat_capacity_params

K_B = 1.380649e-23


def _wl(K=80, n_sizes=4, a_um=(0.0006, 0.01), cells=6, log10U=(-1.0, 4.0), seed=11):
    cfg = dict(synth.CONFIGS[0])
    cfg.update(K=K, n_sizes=n_sizes, species=("silicate", "graphite"), a_um=a_um, n_cells=cells,
               log10U=log10U, seed=seed)
    wl = synth.make_workload(cfg)
    N, th = heat_capacity_params(cfg["species"], wl.sp_of_g, wl.a_of_g)
    return wl, N, th


def _null_vector(A):
    """Stationary distribution of the master equation dP/dt = Q P with
    Q[f,i] = A[f,i] (f != i), Q[i,i] = -sum_f A[f,i]: one balance row
    replaced by the normalisation sum P = 1, dense LU solve."""
    M = A.shape[0]
    Q = A - np.diag(np.diag(A))
    Q -= np.diag(Q.sum(axis=0))
    Q[-1, :] = 1.0
    rhs = np.zeros(M)
    rhs[-1] = 1.0
    return np.linalg.solve(Q, rhs)


@pytest.mark.parametrize("theta,N", [(500.0, 70.0), (900.0, 3.0e4)])
def test_einstein_enthalpy_is_integral_of_heat_capacity(theta, N):
    from scipy.integrate import quad

    def cap(T):  # Einstein heat capacity, 3 N k_B (theta/T)^2 e^(theta/T) / (e^(theta/T) - 1)^2
        x = theta / T
        return 3.0 * N * K_B * x * x * math.exp(-x) / (-math.expm1(-x)) ** 2

    for T in (5.0, 40.0, 300.0, 2500.0):
        ref = quad(cap, 1e-3, T, limit=200, epsabs=0.0, epsrel=1e-12)[0]
        assert abs(float(fluct.enthalpy(T, N, theta)) / ref - 1.0) < 1e-9
        assert abs(float(fluct.temperature_of(fluct.enthalpy(T, N, theta), N, theta)) / T - 1.0) < 1e-12
    # classical limit: E -> 3 N k_B (T - theta / 2 + theta^2 / (12 T))
    T = 1e5
    ref = 3 * N * K_B * (T - theta / 2 + theta * theta / (12 * T))
    assert abs(float(fluct.enthalpy(T, N, theta)) / ref - 1.0) < 1e-10
    assert fluct.enthalpy(0.0, N, theta) == 0.0 and fluct.temperature_of(0.0, N, theta) == 0.0


@pytest.mark.parametrize("M", [2, 3, 7, 17, 40])
def test_recursion_equals_null_space_random_rates(M):
    rng = np.random.default_rng(M)
    A = np.zeros((M, M))
    for i in range(M):
        for f in range(i + 1, M):
            if rng.random() < 0.6:
                A[f, i] = np.exp(rng.normal(0.0, 2.0))
    for j in range(1, M):
        A[j - 1, j] = np.exp(rng.normal(1.0, 1.0))
    A[1, 0] += 1.0  # level 0 must be able to leave
    P = fluct.steady_state(A)
    ref = _null_vector(A)
    assert abs(P.sum() - 1.0) < 1e-14
    np.testing.assert_allclose(P, ref, rtol=1e-9, atol=1e-13 * ref.max())


@pytest.mark.parametrize("cell,grain", [(0, 0), (3, 1), (5, 4), (2, 6)])
def test_recursion_equals_null_space_physical_rates(cell, grain):
    wl, N, th = _wl(log10U=(0.0, 2.0))
    lam, w, C, J = wl.lam, wl.w, wl.C_abs[grain], wl.J[cell].astype(np.float64)
    M = 24
    dE = fluct.H_PL * fluct.C_LI / lam[0] / 5.0
    T_lev = fluct.temperature_of(np.arange(M) * dE, N[grain], th[grain])
    cool = 4 * math.pi * (fluct.planck(lam, np.maximum(T_lev, wl.T_min)) @ (w * C)) / dE
    eps = fluct.H_PL * fluct.C_LI / lam
    A, _ = fluct.rate_matrix(eps, 4 * math.pi * w * C * J / eps, dE, cool)
    P = fluct.steady_state(A)
    ref = _null_vector(A)
    np.testing.assert_allclose(P, ref, rtol=1e-7, atol=1e-12 * ref.max())


def test_photon_split_conserves_energy():
    wl, N, th = _wl()
    lam, w, C, J = wl.lam, wl.w, wl.C_abs[1], wl.J[2].astype(np.float64)
    eps = fluct.H_PL * fluct.C_LI / lam
    R = 4 * math.pi * w * C * J / eps
    M = 30
    dE = eps[0] / 7.3
    A, lost = fluct.rate_matrix(eps, R, dE, np.ones(M))
    heat = float(np.dot(R, eps))
    for i in range(M):
        gain = sum(A[f, i] * (f - i) * dE for f in range(i + 1, M))
        assert abs(gain + lost[i] - heat) <= 1e-12 * heat
        if i + eps[0] / dE < M - 1:
            assert lost[i] == 0.0
    # photons below one level move up with probability eps / dE
    low = eps < dE
    up = A[1, 0] + A[2:, 0].sum()
    assert abs(up - (R[~low].sum() + (R[low] * eps[low] / dE).sum())) <= 1e-12 * R.sum()


@pytest.mark.parametrize("M", [32, 64])
def test_emitted_power_balances_absorbed_minus_clipped(M):
    wl, N, th = _wl(cells=5)
    grains = np.arange(wl.G)
    r = fluct.run(wl.lam, wl.w, wl.C_abs, wl.J, wl.n, grains, N, th, M, wl.T_min, wl.T_max)
    T1 = fluct.temperature_of(r["dE"], N[None, :], th[None, :])
    assert (T1 >= wl.T_min).all()  # no level cools at a floored temperature
    emitted = r["L"] @ wl.w
    absorbed = (wl.n * r["heat"] * (1.0 - r["clipped"])).sum(axis=1)
    np.testing.assert_allclose(emitted, absorbed, rtol=1e-10)
    assert r["clipped"].max() < 1e-2
    np.testing.assert_allclose(r["P"].sum(axis=2), 1.0, rtol=1e-13)


def test_large_grains_converge_to_equilibrium_at_first_order():
    wl, N, th = _wl(n_sizes=3, a_um=(0.03, 0.3), cells=3, log10U=(2.0, 4.0))
    g = 2  # 0.3 um silicate: thousands of photons per cooling time
    errs = []
    for M in (64, 128, 256):
        r = fluct.run(wl.lam, wl.w, wl.C_abs, wl.J, wl.n[:, [g]], [g], N[[g]], th[[g]], M, wl.T_min, wl.T_max)
        E_mean = (r["P"][:, 0] * np.arange(M)[None, :]).sum(axis=1) * r["dE"][:, 0]
        E_eq = fluct.enthalpy(r["T_eq"][:, 0], N[g], th[g])
        e = np.abs(E_mean / E_eq - 1.0)
        assert (e < 1.0 / M).all()
        errs.append(e)
    for a, b in zip(errs, errs[1:]):
        assert ((a / b > 1.8) & (a / b < 2.2)).all()


def test_grid_rule_and_field_monotonicity():
    wl, N, th = _wl(n_sizes=2, a_um=(0.001, 0.005), cells=1)
    g = 0
    means = []
    for s in (1.0, 10.0, 100.0, 1000.0):
        r = fluct.run(wl.lam, wl.w, wl.C_abs, wl.J * s, wl.n[:, [g]] * 3.0, [g], N[[g]], th[[g]], 48,
                      wl.T_min, wl.T_max)
        eps_max = fluct.H_PL * fluct.C_LI / wl.lam[0]
        top = min(2 * (fluct.enthalpy(r["T_eq"][0, 0], N[g], th[g]) + eps_max), fluct.enthalpy(wl.T_max, N[g], th[g]))
        assert abs(r["dE"][0, 0] * 47 / top - 1.0) < 1e-14
        means.append(float((r["P"][0, 0] * np.arange(48)).sum() * r["dE"][0, 0]))
        r1 = fluct.run(wl.lam, wl.w, wl.C_abs, wl.J * s, wl.n[:, [g]], [g], N[[g]], th[[g]], 48,
                       wl.T_min, wl.T_max)
        np.testing.assert_allclose(r["L"], 3.0 * r1["L"], rtol=1e-13)
        np.testing.assert_array_equal(r["P"], r1["P"])
    assert all(a < b for a, b in zip(means, means[1:]))


def test_zero_field_sits_in_the_ground_level():
    """No photons: nothing leaves level 0, so P = (1, 0, ...) and L = 0."""
    wl, N, th = _wl(cells=2)
    grains = np.arange(wl.G)
    J = np.zeros_like(wl.J)
    r = fluct.run(wl.lam, wl.w, wl.C_abs, J, wl.n, grains, N, th, 32, wl.T_min, wl.T_max)
    assert (r["P"][:, :, 0] == 1.0).all() and (r["P"][:, :, 1:] == 0.0).all()
    assert (r["L"] == 0.0).all() and (r["heat"] == 0.0).all()


@pytest.mark.parametrize("cell,grain,M", [(0, 0, 24), (3, 5, 40), (5, 2, 64)])
def test_cumulative_rates_are_two_prefix_sums(cell, grain, M):
    """On a uniform level grid the rate of jumps of at least m levels, from
    any level i below the top, is one function Phi(m) = sum_k R_k
    clamp(x_k - m + 1, 0, 1) of m = f - i (x_k = eps_k / dE), which the CUDA
    kernel reads off two exclusive prefix sums over the wavelengths (x_k
    falls as k rises):  Phi(m) = Sh[kb(m)] + Sf[kb(m-1)] - Sf[kb(m)] with
    kb(m) = #{k : x_k >= m}.  Checked against the full transition matrix the
    oracle builds one photon landing at a time."""
    wl, N, th = _wl(log10U=(0.0, 3.0))
    lam, w, C, J = wl.lam, wl.w, wl.C_abs[grain], wl.J[cell].astype(np.float64)
    eps = fluct.H_PL * fluct.C_LI / lam
    R = 4 * math.pi * w * C * J / eps
    dE = eps[0] / 9.37
    A, _ = fluct.rate_matrix(eps, R, dE, np.ones(M))
    x = eps / dE
    assert (np.diff(x) < 0).all()
    Sh = np.concatenate([[0.0], np.cumsum(R)])
    Sf = np.concatenate([[0.0], np.cumsum(R * (x - np.floor(x)))])
    kb = np.array([np.count_nonzero(x >= m) for m in range(M)])
    phi = np.zeros(M)
    for m in range(1, M):
        phi[m] = Sh[kb[m]] + Sf[kb[m - 1]] - Sf[kb[m]]
    up = np.tril(A, -1)
    for i in range(M - 1):
        for f in range(i + 1, M):
            np.testing.assert_allclose(up[f:, i].sum(), phi[f - i], rtol=1e-12, atol=1e-300)
