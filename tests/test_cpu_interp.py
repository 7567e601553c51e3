"""The paper's CPU interpolation scheme (Section 6, Table 1's "CPU
(interpolation)" column), checked against the FP64 oracle and against what
linear interpolation of a concave function fixes.

P_g(T) is a sum of Planck functions with non-negative weights, each convex in
T, so T(P) is concave and a chord between two nodes lies below it: the
interpolated temperature never exceeds the root, and falls short of it by at
most about (s - 1) d^2 / 8 of T, with d the node spacing in ln T and
s = d ln P / d ln T.  A node's own power must give back the node's
temperature.  A wrong bracket, a reversed interpolation weight or a table
built at the wrong temperatures fails one of these.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from metrics import l_err
from oracle import cpu_interp as ci


@pytest.fixture(scope="module")
def wl0():
    return synth.make_workload(0)


@pytest.fixture(scope="module")
def tab0(wl0):
    return ci.for_workload(wl0)


def _field_rows(wl, A_rows):
    """J rows that make grain 0's absorbed power A: a gray field scaled per row."""
    J1 = np.ones(wl.K)
    a1 = oracle.absorbed(wl.w, wl.C_abs[0], J1)
    return np.outer(np.asarray(A_rows) / a1, J1)


def test_nodes_log_uniform(tab0):
    d = np.diff(np.log(tab0.T_nodes))
    assert tab0.T_nodes[0] == ci.T_LO and tab0.T_nodes[-1] == ci.T_HI
    assert len(tab0.T_nodes) == ci.NT
    assert np.allclose(d, math.log(ci.T_HI / ci.T_LO) / (ci.NT - 1), rtol=1e-9, atol=0)


def test_node_power_gives_node_temperature(wl0, tab0):
    """A = P_g(T_j) from the oracle's own quadrature returns T_j."""
    rng = np.random.default_rng(7)
    js = rng.integers(1, ci.NT - 1, size=24)
    A = np.array([oracle.power(wl0.lam, wl0.w, wl0.C_abs[0], tab0.T_nodes[j]) for j in js])
    r = tab0.run(_field_rows(wl0, A), np.ones((len(js), wl0.G)), want_L=False)
    assert (r["flags"][:, 0] == 0).all()
    np.testing.assert_allclose(r["T"][:, 0], tab0.T_nodes[js], rtol=1e-10, atol=0)


@pytest.mark.parametrize("g", [0, 7, 15])
def test_blackbody_field_below_root_within_chord_bound(wl0, tab0, g):
    """J = B(T0) gives A = P_g(T0) (Eq. 7's identity), so the root is T0: the
    chord stays below it, by at most (s - 1) d^2 / 8 of T0 (10 % margin for
    the change of s across one interval)."""
    T0s = np.exp(np.random.default_rng(g).uniform(math.log(4.0), math.log(1400.0), size=40))
    J = np.stack([[oracle.planck(l, T0) for l in wl0.lam] for T0 in T0s])
    r = tab0.run(J, np.ones((len(T0s), wl0.G)), want_L=False)
    T = r["T"][:, g]
    assert (r["flags"][:, g] == 0).all()
    d = math.log(ci.T_HI / ci.T_LO) / (ci.NT - 1)
    for T0, Ti in zip(T0s, T):
        eps = 1e-4
        s = (math.log(oracle.power(wl0.lam, wl0.w, wl0.C_abs[g], T0 * (1 + eps)))
             - math.log(oracle.power(wl0.lam, wl0.w, wl0.C_abs[g], T0 * (1 - eps)))) / (2 * eps)
        assert Ti <= T0 * (1 + 1e-12)
        assert T0 - Ti <= 1.1 * (s - 1) * d * d / 8 * T0 + 1e-12 * T0


def test_against_oracle_tiny_workload(wl0, tab0):
    """The 1024-cell, 64-wavelength, 16-grain workload: T within the chord
    bound (s < 12 there gives 1.3e-5), never above the root, flags equal, and
    L within the T error times d ln B / d ln T (peak-floored)."""
    r = tab0.run(wl0.J, wl0.n)
    ref = oracle.run_workload(wl0)
    assert (r["flags"] == ref["flags"]).all()
    ok = ref["flags"] == 0
    rel = (r["T"][ok] - ref["T"][ok]) / ref["T"][ok]
    assert rel.max() <= 1e-12
    assert -rel.min() <= 1.5e-5
    assert l_err(r["L"], ref["L"]).max() <= 1e-3


def test_clamps_and_invalid(wl0, tab0):
    P0, P1 = tab0.P[0, 0], tab0.P[0, -1]
    A = np.array([0.0, 0.5 * P0, 2.0 * P1, P0 * (1 + 1e-9), P1 * (1 - 1e-9)])
    J = _field_rows(wl0, A)
    J = np.vstack([J, np.full(wl0.K, np.nan), -np.ones(wl0.K)])
    r = tab0.run(J, np.ones((len(J), wl0.G)), want_L=False)
    fl, T = r["flags"][:, 0], r["T"][:, 0]
    assert list(fl[:3]) == [1, 1, 2]
    assert T[0] == ci.T_LO and T[1] == ci.T_LO and T[2] == ci.T_HI
    assert fl[3] == 0 and T[3] == pytest.approx(ci.T_LO, rel=1e-9)
    assert fl[4] == 0 and T[4] == pytest.approx(ci.T_HI, rel=1e-9)
    assert list(fl[5:]) == [4, 4] and np.isnan(T[5:]).all()


def test_thread_count_does_not_change_results(wl0, tab0):
    a = tab0.run(wl0.J[:200], wl0.n[:200], n_threads=1)
    b = tab0.run(wl0.J[:200], wl0.n[:200], n_threads=0)
    for k in ("T", "flags", "L"):
        assert np.array_equal(a[k], b[k])
