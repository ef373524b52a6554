"""Pin: the spatial part of the walk against heat-semigroup closed forms.

* a_0 is the contribution of single-leaf trees: under Strategy B it equals
  E[g(x + sqrt(2 D t) n)] = (P_t g)(x), the Gaussian convolution of the initial
  data (Eqs. integraleq, green, SDE with sigma^2 = 2D); under Strategy A it is
  e^{-c t} (P_t g)(x).
* a_1 is the contribution of trees with one split; for f = b u^2 and Gaussian
  g it equals b int_0^t P_s[(P_{t-s} g)^2] ds (times e^{-c s - 2c(t-s)} under
  Strategy A), which fixes the split-time law, the split position and the
  children's start.
The oracle's estimates must lie within 4.5 standard errors.
"""
import math

import numpy as np
import pytest

import workloads
from checkers import first_order_gauss_1d, heat_cos_prod, heat_gauss, heat_quadrature_1d


def _solve(oracle_mod, pb, x, t, N, K, seed=3):
    x = np.asarray(x, float).reshape(-1, pb["dim"])
    r = oracle_mod.solve(pb, x, np.full(len(x), t), np.full(len(x), N, np.uint64), K, 1, 1, seed)
    return r["coef"], r["se"]


def test_a0_gauss_2d_strategy_b(oracle_mod):
    pb = workloads.problem_sin_2d()
    x = np.array([[0.0, 0.0], [1.0, -0.5], [2.5, 2.5], [-3.0, 1.0]])
    for t in (0.25, 1.0):
        a, se = _solve(oracle_mod, pb, x, t, 200_000, 10)
        expect = heat_gauss(x, t, pb["D"], 0.0, 1.2, 1.0, (0.0, 0.0))
        assert np.all(np.abs(a[:, 0] - expect) <= 4.5 * se[:, 0] + 1e-15), (a[:, 0], expect, se[:, 0])


def test_a0_gauss_1d_strategy_a_mckean(oracle_mod):
    pb = workloads.problem_kpp_1d()
    x = np.array([[-2.0], [-0.5], [0.0], [1.3]])
    t = 0.5
    a, se = _solve(oracle_mod, pb, x, t, 200_000, 8)
    expect = math.exp(-pb["c_pot"] * t) * heat_gauss(x, t, pb["D"], 0.5, 0.3, 1 / math.sqrt(2), (0.0,))
    assert np.all(np.abs(a[:, 0] - expect) <= 4.5 * se[:, 0]), (a[:, 0], expect, se[:, 0])


def test_a0_cos_product_2d(oracle_mod):
    pb = workloads.problem_uneven_2d()
    x = np.array([[0.3, 0.7], [2.0, 5.5], [7.5, 1.0]])
    t = 0.8
    a, se = _solve(oracle_mod, pb, x, t, 200_000, 6)
    expect = heat_cos_prod(x, t, pb["D"], 1.5, 0.5, (1.0, 1.0))
    assert np.all(np.abs(a[:, 0] - expect) <= 4.5 * se[:, 0]), (a[:, 0], expect, se[:, 0])


def test_a0_tanh_product_3d(oracle_mod):
    pb = workloads.problem_pdd_3d()
    x = np.array([[2.0, 1.5, 2.5], [1.0, 3.2, 0.4], [2.7, 2.1, 1.9]])
    t = 1.0
    a, se = _solve(oracle_mod, pb, x, t, 200_000, 6)
    expect = []
    for p in x:
        pr = 1.0
        for i in range(3):
            pr *= heat_quadrature_1d(lambda z: np.tanh(z - 2.0), p[i], t, pb["D"])[0]
        expect.append(pr)
    assert np.all(np.abs(a[:, 0] - np.array(expect)) <= 4.5 * se[:, 0]), (a[:, 0], expect, se[:, 0])


def test_a0_logistic_1d(oracle_mod):
    w = math.sqrt(2.0)
    pb = dict(dim=1, D=1.0, f_coef=[0.0, -0.25, 1.25, -1.0], u0=("logistic", (0.0, 1.0, 0.0, w)), strategy="B",
              q=0.6, arity_law="uniform")
    x = np.array([[-1.0], [0.0], [2.0]])
    t = 0.6
    a, se = _solve(oracle_mod, pb, x, t, 200_000, 8)
    expect = heat_quadrature_1d(lambda z: 1.0 / (1.0 + np.exp(-z / w)), x[:, 0], t, 1.0)
    assert np.all(np.abs(a[:, 0] - expect) <= 4.5 * se[:, 0]), (a[:, 0], expect, se[:, 0])


@pytest.mark.parametrize("strategy,D,q,lam,c", [("B", 1.0, 0.55, 1.0, 0.0), ("B", 0.3, 0.7, 1.0, 0.0),
                                                ("A", 1.0, 0.5, 1.0, 1.0), ("A", 0.6, 0.5, 1.7, 0.4)])
def test_a1_one_split_closed_form(oracle_mod, strategy, D, q, lam, c):
    A, s, b = 1.3, 0.8, 0.9
    pb = dict(dim=1, D=D, f_coef=[0.0, -c, b], u0=("gauss", (0.0, A, s, 0.0)), strategy=strategy, q=q,
              lam=lam, c_pot=c, arity_law="uniform")
    x = np.array([[0.0], [0.7], [-1.6]])
    t = 0.7
    a, se = _solve(oracle_mod, pb, x, t, 300_000, 6)
    expect = first_order_gauss_1d(x[:, 0], t, D, A, s, b, c_pot=c)
    assert np.all(np.abs(a[:, 1] - expect) <= 4.5 * se[:, 1]), (a[:, 1], expect, se[:, 1])
    e0 = math.exp(-c * t) * heat_gauss(x, t, D, 0.0, A, s, (0.0,))
    assert np.all(np.abs(a[:, 0] - e0) <= 4.5 * se[:, 0])


def test_first_order_checker_against_brute_quadrature():
    # the helper's Gaussian algebra against a direct 2-D quadrature of the same integral
    from scipy import integrate
    D, A, s, b, t, x = 0.8, 1.1, 0.7, 1.0, 0.5, 0.3

    def P(tau, fun, xx):
        return heat_quadrature_1d(fun, xx, tau, D, n=60)[0] if tau > 0 else fun(np.array([xx]))[0]

    def g(z):
        return A * np.exp(-z * z / (2 * s * s))

    def integrand(sp):
        inner = lambda z: np.array([P(t - sp, g, zz) ** 2 for zz in np.atleast_1d(z)])
        return P(sp, inner, x)

    brute = b * integrate.quad(integrand, 0.0, t, epsrel=1e-8)[0]
    assert abs(first_order_gauss_1d([x], t, D, A, s, b)[0] - brute) < 1e-8


def test_a0_axis_gaussian_2d(oracle_mod):
    # g = c0 + A exp(-sum_i w_i (x_i - m_i)^2): each axis convolves separately,
    # (P_t g)(x) = c0 + A prod_i (1 + 4 w_i D t)^{-1/2} exp(-w_i (x_i - m_i)^2 / (1 + 4 w_i D t));
    # w_1 = 0 is the Example 5 initial data (a function of x_0 alone)
    pb = workloads.problem_var_coef_2d()
    c0, A, w0, w1, _, m0, m1, _ = pb["u0"][1]
    x = np.array([[0.0, 0.0], [1.5, -2.0], [-2.5, 0.7]])
    t, D = 0.5, pb["D"]
    pb0 = dict(pb)
    pb0.pop("coef")
    a, se = _solve(oracle_mod, pb0, x, t, 200_000, 4)
    expect = np.full(len(x), c0)
    g = np.ones(len(x)) * A
    for i, (w, m) in enumerate(((w0, m0), (w1, m1))):
        s = 1.0 + 4.0 * w * D * t
        g *= np.exp(-w * (x[:, i] - m) ** 2 / s) / math.sqrt(s)
    expect = expect + g
    assert np.all(np.abs(a[:, 0] - expect) <= 4.5 * se[:, 0]), (a[:, 0], expect, se[:, 0])
