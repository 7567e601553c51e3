"""Thermally fluctuating grains, FP64 CPU oracle -- TEST INFRASTRUCTURE.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this module; the CUDA library never does, and the two share no code.

The paper stops at equilibrium temperatures and names the calculation of
grains whose temperature fluctuates as the next step (Sections 1 and 6): the
temperature probability distribution of a small grain, which needs one
transition-matrix solve per grain species and cell, after Guhathakurta &
Draine (1989).  This module computes that distribution, from its definition,
as follows.

* Enthalpy: an Einstein solid, E_g(T) = c_g / (exp(theta_g / T) - 1) with
  c_g = 3 N_g k_B theta_g; its inverse T_g(E) = theta_g / ln(1 + c_g / E).
* Level grid per (cell, grain): M levels E_j = j dE, j = 0..M-1, with
  E_top = (M-1) dE = min(2 (E_g(T_eq) + eps_max), E_g(T_max)), where T_eq
  is the cell's equilibrium temperature of the grain (the root of Eq. 7) and
  eps_max = h c / lambda_0 the most energetic photon of the grid.
* Heating (Eq. 6 per photon): photons of wavelength lambda_k are absorbed at
  R_k = 4 pi w_k C[g,k] J[c,k] / eps_k per second, eps_k = h c / lambda_k.  From
  level i such a photon lands at y = i + eps_k / dE (in level units); the
  transition goes to floor(y) with probability 1 - frac(y) and to
  floor(y) + 1 with probability frac(y), which conserves the energy on
  average.  A landing at or beyond the top level goes to the top level; the
  energy above E_top is lost ("clipped").
* Cooling (thermal-continuous approximation): only j -> j-1, at the rate
  4 pi P_g(T_j') / dE with T_j' = max(T_j, T_min) and P_g of Eq. 7, so that
  the mean cooling power of a level is its emitted power.
* Steady state: the flux of probability upward across the cut between
  levels j-1 and j equals the flux downward,
  sum_{i<j} P_i sum_{f>=j} A[f,i] = P_j A[j-1,j],  j = 1..M-1,
  solved in order of j from P_0 = 1 and normalised to sum 1.
* Emission (Eqs. 8-10 over the distribution):
  L[c,k] = 4 pi sum_g n[c,g] sum_j P_j C[g,k] B_k(T_j)  (T_0 = 0 emits nothing).
"""
import math

import numpy as np

from . import run as _equilibrium

H_PL = 6.62607015e-34
C_LI = 299792458.0
K_BO = 1.380649e-23


def planck(lam, T):
    """B_k(T) per unit wavelength [W m^-2 m^-1 sr^-1] for arrays lam [K] and
    T [M] -> [M, K]; exactly 0 where T <= 0 or h c / (lam k_B T) > 709."""
    lam = np.asarray(lam, dtype=np.float64)
    T = np.atleast_1d(np.asarray(T, dtype=np.float64))
    out = np.zeros((len(T), len(lam)))
    pos = T > 0
    if pos.any():
        x = H_PL * C_LI / (K_BO * lam[None, :] * T[pos, None])
        pref = 2.0 * H_PL * C_LI * C_LI / lam ** 5
        with np.errstate(over="ignore", divide="ignore"):
            b = np.where(x <= 709.0, pref[None, :] / np.expm1(np.minimum(x, 709.0)), 0.0)
        out[pos] = b
    return out


def enthalpy(T, n_atoms, theta):
    """E(T) = 3 N k_B theta / (exp(theta / T) - 1) [J]; 0 at T = 0."""
    T = np.asarray(T, dtype=np.float64)
    c = 3.0 * n_atoms * K_BO * theta
    with np.errstate(over="ignore", divide="ignore"):
        return np.where(T > 0, c / np.expm1(theta / np.where(T > 0, T, 1.0)), 0.0)


def temperature_of(E, n_atoms, theta):
    """T(E) = theta / ln(1 + 3 N k_B theta / E) [K]; 0 at E = 0."""
    E = np.asarray(E, dtype=np.float64)
    c = 3.0 * n_atoms * K_BO * theta
    with np.errstate(divide="ignore"):
        return np.where(E > 0, theta / np.log1p(c / np.where(E > 0, E, 1.0)), 0.0)


def level_spacing(T_eq, n_atoms, theta, M, lam0, T_max):
    """dE of the level grid (see the module docstring)."""
    eps_max = H_PL * C_LI / lam0
    top = min(2.0 * (float(enthalpy(T_eq, n_atoms, theta)) + eps_max),
              float(enthalpy(T_max, n_atoms, theta)))
    return top / (M - 1)


def rate_matrix(eps, R, dE, cool):
    """Transition rates A[f, i] (i -> f, per second) of one (cell, grain):
    upward by photon absorption with the energy-conserving split, downward
    j -> j-1 at cool[j].  Also returns the power each level i loses to the
    top clip, lost[i] (W).  Built one transition at a time."""
    M = len(cool)
    A = np.zeros((M, M))
    lost = np.zeros(M)
    lost[M - 1] = float(np.dot(R, eps))  # the top level keeps none of what it absorbs
    for i in range(M - 1):
        for e, r in zip(eps, R):
            y = i + e / dE
            if y >= M - 1:
                A[M - 1, i] += r
                lost[i] += r * (y - (M - 1)) * dE
                continue
            f = math.floor(y)
            a = y - f
            if f > i:
                A[f, i] += r * (1.0 - a)
            A[f + 1, i] += r * a
    for j in range(1, M):
        A[j - 1, j] += cool[j]
    return A, lost


def steady_state(A):
    """Guhathakurta-Draine recursion on the cut fluxes: P_0 = 1,
    P_j = sum_{i<j} P_i B[j,i] / A[j-1,j] with B[j,i] = sum_{f>=j} A[f,i];
    rescaled whenever the values grow large, normalised to sum 1."""
    M = A.shape[0]
    up = np.tril(A, -1)                           # f > i: upward rates
    B = np.cumsum(up[::-1], axis=0)[::-1]         # B[j, i] = sum_{f >= j} up[f, i]
    P = np.zeros(M)
    P[0] = 1.0
    for j in range(1, M):
        P[j] = np.dot(B[j, :j], P[:j]) / A[j - 1, j]
        if P[j] > 1e200:
            P[: j + 1] *= 1e-200
    return P / P.sum()


def solve_one(lam, w, C_g, J_c, T_eq, n_atoms, theta, M, T_min, T_max):
    """Distribution of one (cell, grain): (dE, T_levels, P, lost power,
    absorbed power 4 pi A)."""
    lam, w, C_g, J_c = (np.asarray(v, dtype=np.float64) for v in (lam, w, C_g, J_c))
    dE = level_spacing(T_eq, n_atoms, theta, M, lam[0], T_max)
    T_lev = temperature_of(np.arange(M) * dE, n_atoms, theta)
    T_cool = np.maximum(T_lev, T_min)
    P_em = planck(lam, T_cool) @ (w * C_g)                 # P_g(T'_j), Eq. 7
    cool = 4.0 * math.pi * P_em / dE
    eps = H_PL * C_LI / lam
    R = 4.0 * math.pi * w * C_g * J_c / eps
    A, lost = rate_matrix(eps, R, dE, cool)
    P = steady_state(A)
    return dE, T_lev, P, float(P @ lost), 4.0 * math.pi * float(np.dot(w * C_g, J_c))


def run(lam, w, C, J, n_f, grains, n_atoms, theta, M, T_min, T_max, want_P=True):
    """Fluctuating grains `grains` (indices into C's rows) in every cell.

    n_f [cells, Gf]: grain numbers of those grains.  Returns a dict with
    T_eq, flags (equilibrium solve of the same grains), dE [cells, Gf] (J),
    P [cells, Gf, M], L [cells, K] (their emission), clipped [cells, Gf] (lost
    fraction of the absorbed power) and heat [cells, Gf] (4 pi A, W).
    """
    lam, w, C = (np.asarray(v, dtype=np.float64) for v in (lam, w, C))
    J = np.asarray(J, dtype=np.float64)
    n_f = np.asarray(n_f, dtype=np.float64)
    grains = np.asarray(grains)
    nc, K = J.shape
    Gf = len(grains)
    Cf = C[grains]
    eq = _equilibrium(lam, w, Cf, J, np.ones((nc, Gf)), T_min, T_max, want_L=False, want_resid=False)
    dE = np.empty((nc, Gf))
    P = np.empty((nc, Gf, M)) if want_P else None
    L = np.zeros((nc, K))
    clipped = np.zeros((nc, Gf))
    heat = np.zeros((nc, Gf))
    for c in range(nc):
        for q in range(Gf):
            d, T_lev, p, lost, h = solve_one(lam, w, Cf[q], J[c], eq["T"][c, q], n_atoms[q], theta[q],
                                             M, T_min, T_max)
            dE[c, q] = d
            if want_P:
                P[c, q] = p
            L[c] += 4.0 * math.pi * n_f[c, q] * (p @ planck(lam, T_lev)) * Cf[q]
            clipped[c, q] = lost / h if h > 0 else 0.0
            heat[c, q] = h
    return dict(T_eq=eq["T"], flags=eq["flags"], dE=dE, P=P, L=L, clipped=clipped, heat=heat)
