"""Pins of variable coefficients c_k(x, t) = b_k gamma(x, t) (Sec. 1, Eq. nonlinear_new; Example 5).

The coefficient acts where and when a particle splits: at the split position
and at the PDE time left to the children (Sec. 2.1, Eq. probexp1).  Pinned by
  * a time-only profile with constant u0, where the PDE is the ODE
    u' = eps b(t) u^2 with b(t) = b2 / (t + t0): 1/u = 1/c0 - eps b2 ln((t+t0)/t0),
    so a_n = c0^{n+1} (b2 ln((t + t0)/t0))^n exactly.  The PDE time matters from
    order 2 on (order 1 is the same integral either way round);
  * a mask selecting one of two terms, against RK4 on the eps-hierarchy of
    u' = eps (b2 gamma(t) u^2 + b3 u^3);
  * the order-1 coefficient of a space-time profile against quadrature: with
    constant u0 the single split happens at elapsed time s, position
    x + sqrt(2 D s) Z, PDE time t - s, so
    a_1 = b2 c0^2 int_0^t prod_i (1 + 4 w_i D s)^{-1/2} exp(-w_i (x_i - m_i)^2 / (1 + 4 w_i D s)) / (t - s + t0) ds;
  * gamma == 1 leaving every tree bit-identical to the constant-coefficient walk.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from checkers import eps_hierarchy_rk4_t


def _pooled(oracle_mod, pb, x, t, n_total, K, copies=8, seed=21):
    d = pb["dim"]
    xs = np.tile(np.asarray(x, float).reshape(1, d), (copies, 1))
    r = oracle_mod.solve(pb, xs, np.full(copies, t), np.full(copies, n_total // copies, np.uint64), K,
                         K // 2, K // 2, seed)
    N = float(n_total // copies * copies)
    a = r["s1"].sum(axis=0) / N
    se = np.sqrt(np.maximum(r["s2"].sum(axis=0) / N - a * a, 0.0) / (N - 1))
    return a, se


def _check(a, se, expect, nsig=4.5):
    for n in range(len(expect)):
        assert abs(a[n] - expect[n]) <= nsig * se[n] + 1e-13 * abs(expect[n]), (n, a[n], expect[n], se[n])


def _problem(strategy, f_coef, coef, c0=0.6, dim=1, D=0.5, q=2.0 / 3.0):
    return dict(dim=dim, D=D, f_coef=list(f_coef), u0=("const", (c0,)), strategy=strategy, lam=1.0, c_pot=0.0,
                q=q, arity_law="uniform", coef=coef)


@pytest.mark.parametrize("strategy", ["A", "B"])
def test_time_profile_closed_form(oracle_mod, strategy):
    c0, b2, t0, t, K = 0.6, -1.0, 0.1, 0.5, 8
    pb = _problem(strategy, [0.0, 0.0, b2], ("gauss_over_t", (0, 0, 0, 0, 0, 0, t0), [2]), c0=c0)
    a, se = _pooled(oracle_mod, pb, [0.3], t, 400_000, K)
    C = b2 * math.log((t + t0) / t0)
    _check(a, se, [c0 ** (n + 1) * C ** n for n in range(K + 1)])


def test_mask_selects_the_term(oracle_mod):
    c0, b2, b3, t0, t, K = 0.7, 1.0, -0.8, 0.25, 0.6, 8
    pb = _problem("B", [0.0, 0.0, b2, b3], ("gauss_over_t", (0, 0, 0, 0, 0, 0, t0), [2]), c0=c0)
    a, se = _pooled(oracle_mod, pb, [0.0], t, 400_000, K)
    # the split at elapsed s acts at PDE time t - s: in ODE time that is the coefficient at time t - s
    expect = eps_hierarchy_rk4_t(lambda s: [0.0, 0.0, b2 / (s + t0), b3], 0.0, c0, t, K)
    _check(a, se, expect)


@pytest.mark.parametrize("strategy", ["A", "B"])
def test_first_order_space_time_profile_quadrature(oracle_mod, strategy):
    c0, b2, D, t, K = 0.8, 1.5, 0.5, 0.7, 6
    w, m, t0 = (0.7, 0.3), (0.2, -0.1), 0.3
    x = (0.5, 0.4)
    pb = _problem(strategy, [0.0, 0.0, b2], ("gauss_over_t", (w[0], w[1], 0.0, m[0], m[1], 0.0, t0), [2]), c0=c0,
                  dim=2, D=D)
    a, se = _pooled(oracle_mod, pb, x, t, 400_000, K)

    def integrand(s):
        v = 1.0 / (t - s + t0)
        for i in range(2):
            g = 1.0 + 4.0 * w[i] * D * s
            v *= math.exp(-w[i] * (x[i] - m[i]) ** 2 / g) / math.sqrt(g)
        return v

    a1 = b2 * c0 * c0 * integrate.quad(integrand, 0.0, t, epsabs=1e-13, epsrel=1e-12)[0]
    assert abs(a[1] - a1) <= 4.5 * se[1], (a[1], a1, se[1])
    # the wrong time argument (elapsed instead of left) would give a clearly different a_1
    wrong = b2 * c0 * c0 * integrate.quad(lambda s: integrand(s) * (t - s + t0) / (s + t0), 0.0, t)[0]
    assert abs(wrong - a1) > 12 * se[1]


@pytest.mark.parametrize("strategy", ["A", "B"])
def test_unit_profile_leaves_trees_unchanged(oracle_mod, strategy):
    base = dict(dim=2, D=0.5, f_coef=[0.2, -0.5, 1.0, 0.3], u0=("gauss", (0.1, 1.0, 0.8, 0.2, -0.3)),
                strategy=strategy, lam=1.3, c_pot=0.0, q=0.55, arity_law="abs")
    unit = dict(base, coef=("gauss", (0, 0, 0, 0.4, 0.5, 0), [0, 1, 2, 3]))
    r0 = oracle_mod.trees(base, [0.3, -0.2], 0.8, 3, 0, 3000, 10, 5)
    r1 = oracle_mod.trees(unit, [0.3, -0.2], 0.8, 3, 0, 3000, 10, 5)
    assert np.array_equal(r0["hash"], r1["hash"]) and np.array_equal(r0["order"], r1["order"])
    assert np.array_equal(r0["w"], r1["w"])
    assert (r0["order"] > 0).sum() > 1000


def test_invalid_profiles_rejected(oracle_mod):
    pb = _problem("B", [0.0, 0.0, 1.0], ("gauss_over_t", (0, 0, 0, 0, 0, 0, 0.0), [2]))
    with pytest.raises(ValueError):
        oracle_mod.trees(pb, [0.0], 0.5, 0, 0, 4, 4, 0)
    pa = dict(_problem("A", [0.0, 0.5, 1.0], ("gauss", (1, 0, 0, 0, 0, 0), [1, 2])), c_pot=1.0)
    with pytest.raises(ValueError):
        oracle_mod.trees(pa, [0.0], 0.5, 0, 0, 4, 4, 0)
