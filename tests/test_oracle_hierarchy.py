"""Pin: spatially constant u0 reduces the PDE to the ODE u' = f(u).

With g = c0 the Brownian paths drop out, and the expected order-n coefficient
is the eps^n coefficient of the ODE's eps-expansion:
  Strategy B (u_t = D Lap u + eps f(u)):  a_n = phi_n t^n, phi' = f(phi), phi(0) = c0;
  Strategy A (u_t = D Lap u - c u + eps F(u), F = f + c u):  U_n(t) of the hierarchy,
  closed form for F = u^2:  a_n = c0^{n+1} e^{-ct} ((1 - e^{-ct})/c)^n
  (McKean's case c = lambda = 1 gives c0^{n+1} e^{-t} (1 - e^{-t})^n).
The oracle's Monte Carlo a_n must lie within 4.5 standard errors of these.
"""
import math

import numpy as np
import pytest

import workloads
from checkers import eps_hierarchy_rk4, ode_taylor


def pooled(oracle_mod, pb, x, t, n_total, K, copies=8, seed=11):
    """Estimate a_n from `copies` independent streams (points 0..copies-1 at the same x)."""
    d = pb["dim"]
    xs = np.tile(np.asarray(x, float).reshape(1, d), (copies, 1))
    r = oracle_mod.solve(pb, xs, np.full(copies, t), np.full(copies, n_total // copies, np.uint64), K,
                         min(K // 2, 4), min(K // 2, 4), seed)
    N = float(n_total // copies * copies)
    S1 = r["s1"].sum(axis=0)
    S2 = r["s2"].sum(axis=0)
    a = S1 / N
    se = np.sqrt(np.maximum(S2 / N - a * a, 0.0) / (N - 1))
    return a, se


def _const_problem(f_coef, strategy, c0, q=0.6, lam=1.0, c_pot=0.0, law="uniform", dim=2):
    return dict(dim=dim, D=0.7, f_coef=list(f_coef), u0=("const", (c0,)), strategy=strategy, lam=lam,
                c_pot=c_pot, q=q, arity_law=law)


def _check(a, se, expect, nsig=4.5):
    for n in range(len(expect)):
        tol = nsig * se[n] + 1e-14 * abs(expect[n])
        assert abs(a[n] - expect[n]) <= tol, (n, a[n], expect[n], se[n])


def test_b_quadratic_geometric_coefficients(oracle_mod):
    c0, t, K = 0.8, 0.9, 8
    pb = _const_problem([0.0, 0.0, 1.0], "B", c0, q=2.0 / 3.0)
    a, se = pooled(oracle_mod, pb, [0.1, 0.2], t, 400_000, K)
    _check(a, se, [c0 ** (n + 1) * t ** n for n in range(K + 1)])


@pytest.mark.parametrize("f_coef,law,c0,t,q", [
    (workloads.SIN9, "abs", 0.9, 1.0, None),
    ((0.0, 1.0, 0.0, -1.0), "uniform", 0.5, 0.8, 2.0 / 3.0),
    ((0.3, 0.0, 1.0), "abs", 0.5, 0.7, 0.6),
])
def test_b_taylor_coefficients_of_the_ode(oracle_mod, f_coef, law, c0, t, q):
    K = 10
    if q is None:
        q = workloads.default_q(f_coef, law)
    pb = _const_problem(f_coef, "B", c0, q=q, law=law)
    a, se = pooled(oracle_mod, pb, [0.0, 0.0], t, 400_000, K)
    phi = ode_taylor(f_coef, c0, K + 1)
    _check(a, se, [phi[n] * t ** n for n in range(K + 1)])


@pytest.mark.parametrize("lam,c", [(1.0, 1.0), (1.5, 0.5)])
def test_a_quadratic_closed_form(oracle_mod, lam, c):
    c0, t, K = 0.7, 0.5, 8
    pb = _const_problem([0.0, -c, 1.0], "A", c0, lam=lam, c_pot=c)
    a, se = pooled(oracle_mod, pb, [0.0, 0.0], t, 300_000, K)
    g = (1 - math.exp(-c * t)) / c
    _check(a, se, [c0 ** (n + 1) * math.exp(-c * t) * g ** n for n in range(K + 1)])


@pytest.mark.parametrize("f_coef,lam,c,c0,t", [
    (workloads.SIN9, 1.0, 0.0, 0.9, 0.6),                 # the paper's u = v e^t change of variables
    ((0.0, 1.0, 0.0, -1.0), 0.8, 0.3, 0.5, 0.7),          # F = 1.3 u - u^3 under a potential
])
def test_a_hierarchy_rk4(oracle_mod, f_coef, lam, c, c0, t):
    K = 8
    pb = _const_problem(f_coef, "A", c0, lam=lam, c_pot=c)
    a, se = pooled(oracle_mod, pb, [0.0, 0.0], t, 300_000, K)
    F = list(f_coef)
    F[1] = F[1] + c
    U = eps_hierarchy_rk4(F, c, c0, t, K)
    _check(a, se, U)


def test_ode_taylor_helper_against_closed_forms():
    # the helper itself: phi' = phi^2 -> c0/(1 - c0 s); phi' = phi - phi^3 -> c0 e^s / sqrt(1 + c0^2 (e^{2s} - 1))
    phi = ode_taylor([0.0, 0.0, 1.0], 0.8, 8)
    assert np.allclose(phi, [0.8 ** (n + 1) for n in range(8)], rtol=1e-14)
    phi = ode_taylor([0.0, 1.0, 0.0, -1.0], 0.5, 12)
    s = 0.3
    exact = 0.5 * math.exp(s) / math.sqrt(1 + 0.25 * (math.exp(2 * s) - 1))
    assert abs(np.polyval(phi[::-1], s) - exact) < 1e-9
    U = eps_hierarchy_rk4([0.0, 0.0, 1.0], 0.5, 0.7, 0.5, 6)
    g = (1 - math.exp(-0.25)) / 0.5
    assert np.allclose(U, [0.7 ** (n + 1) * math.exp(-0.25) * g ** n for n in range(7)], rtol=1e-10)
