"""Pins of general drift and diffusion (Eqs. SDE, green: sigma^2 = a, drift b; Euler
scheme as in Sec. 2.4): per axis dX = (beta - kappa X) dt + (s + r X) dW, m equal
Euler-Maruyama steps per segment.

For this affine family the Euler chain's first two moments follow an exact recursion,
  E[X'] = (1 - kappa h) E[X] + beta h,
  E[X'^2] = E[((1 - kappa h) X + beta h)^2] + h E[(s + r X)^2],
so with quadratic initial data g(x) = c0 + sum_i (l_i x_i + q_i x_i^2) the order-0
coefficient of a tree walk with f = 0 is known exactly; with r = 0 the chain is Gaussian
and the Gaussian initial data's a_0 is a closed form too.  The order-1 coefficient of
f = b u^2 (split at tau S, children from the split position, m steps per segment) is a
one-dimensional integral of Gaussian moments, computed by quadrature.
"""
import math

import numpy as np
import pytest
from scipy import integrate


def _moments(x, m, h, beta, kappa, s, r):
    e1, e2 = float(x), float(x) ** 2
    a = 1.0 - kappa * h
    for _ in range(m):
        n1 = a * e1 + beta * h
        n2 = a * a * e2 + 2.0 * a * beta * h * e1 + (beta * h) ** 2 + h * (s * s + 2.0 * s * r * e1 + r * r * e2)
        e1, e2 = n1, n2
    return e1, e2


def _solve(oracle_mod, pb, x, t, N, K, seed=13, copies=8):
    d = pb["dim"]
    xs = np.tile(np.asarray(x, float).reshape(1, d), (copies, 1))
    r = oracle_mod.solve(pb, xs, np.full(copies, t), np.full(copies, N // copies, np.uint64), K, K // 2, K // 2, seed)
    n = float(N // copies * copies)
    a = r["s1"].sum(axis=0) / n
    se = np.sqrt(np.maximum(r["s2"].sum(axis=0) / n - a * a, 0.0) / (n - 1))
    return a, se


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_order0_quadratic_data_exact_euler_moments(oracle_mod, dim):
    m, t = 5, 0.8
    beta, kappa, s, r = (0.3, -0.2, 0.5)[:dim], (0.7, 1.3, 0.0)[:dim], (0.6, 0.4, 0.9)[:dim], (0.25, -0.3, 0.15)[:dim]
    c0, lin, quad = 0.2, (0.5, -0.7, 0.3), (0.4, 0.25, -0.6)
    pb = dict(dim=dim, D=0.0, f_coef=[0.0], u0=("quadratic", (c0,) + lin + quad), strategy="B", q=0.5,
              sde=(m, beta, kappa, s, r))
    x = (0.4, -0.9, 1.2)[:dim]
    a, se = _solve(oracle_mod, pb, x, t, 400_000, 2)
    expect = c0
    for i in range(dim):
        e1, e2 = _moments(x[i], m, t / m, beta[i], kappa[i], s[i], r[i])
        expect += lin[i] * e1 + quad[i] * e2
    assert abs(a[0] - expect) <= 4.5 * se[0], (a[0], expect, se[0])
    # the wrong step count (one step of t) gives a different value: the pin sees the stepping
    wrong = c0 + sum(lin[i] * _moments(x[i], 1, t, beta[i], kappa[i], s[i], r[i])[0]
                     + quad[i] * _moments(x[i], 1, t, beta[i], kappa[i], s[i], r[i])[1] for i in range(dim))
    assert abs(wrong - expect) > 10 * se[0]


def test_order0_gaussian_data_ou_closed_form(oracle_mod):
    # additive noise (r = 0): the chain is Gaussian with the recursion's mean and variance
    m, t = 7, 1.1
    beta, kappa, s = (0.2, -0.4), (0.9, 0.3), (0.8, 0.5)
    w, c = (0.5, 1.2), (0.3, -0.2)
    pb = dict(dim=2, D=0.0, f_coef=[0.0], u0=("gauss_axes", (0.1, 0.9, w[0], w[1], 0.0, c[0], c[1], 0.0)),
              strategy="A", lam=1.0, c_pot=0.0, sde=(m, beta, kappa, s, (0.0, 0.0)))
    x = (-0.5, 0.7)
    a, se = _solve(oracle_mod, pb, x, t, 400_000, 2)
    val = 0.9
    for i in range(2):
        e1, e2 = _moments(x[i], m, t / m, beta[i], kappa[i], s[i], 0.0)
        v = e2 - e1 * e1
        val *= math.exp(-w[i] * (e1 - c[i]) ** 2 / (1.0 + 2.0 * w[i] * v)) / math.sqrt(1.0 + 2.0 * w[i] * v)
    # Strategy A with f = 0, lambda = 1, c = 0: a_0 = e^{(lambda - c) t} P(S > t) E[g] = E[g]
    expect = 0.1 + val
    assert abs(a[0] - expect) <= 4.5 * se[0], (a[0], expect, se[0])


def test_order1_split_position_and_segments_quadrature(oracle_mod):
    # Strategy B, f = b u^2, 1-D additive OU, quadratic g: a_1 = b int_0^t E[G_{t-s}(X_s)^2] ds with
    # G_tau(y) = E[g(Y)], Y the m-step chain from y over tau, X_s the m-step chain from x over s.
    m, t, b, q = 4, 0.9, 1.3, 0.6
    beta, kappa, s_ = 0.25, 0.8, 0.7
    c0, l, qq = 0.3, 0.6, -0.4
    pb = dict(dim=1, D=0.0, f_coef=[0.0, 0.0, b], u0=("quadratic", (c0, l, 0.0, 0.0, qq, 0.0, 0.0)),
              strategy="B", q=q, sde=(m, (beta,), (kappa,), (s_,), (0.0,)))
    x = 0.35
    a, se = _solve(oracle_mod, pb, [x], t, 800_000, 4)

    def G_coeffs(tau):
        # Y = A y + B0 + noise (variance V): E[g(Y)] = c0 + l (A y + B0) + qq ((A y + B0)^2 + V)
        h = tau / m
        A = (1.0 - kappa * h) ** m
        _, e2_0 = _moments(0.0, m, h, beta, kappa, s_, 0.0)
        B0, _ = _moments(0.0, m, h, beta, kappa, s_, 0.0)
        V = e2_0 - B0 * B0
        # polynomial in y: p0 + p1 y + p2 y^2
        return (c0 + l * B0 + qq * (B0 * B0 + V), l * A + 2.0 * qq * A * B0, qq * A * A)

    def integrand(sv):
        p0, p1, p2 = G_coeffs(t - sv)
        mu, e2 = _moments(x, m, sv / m, beta, kappa, s_, 0.0)
        v = e2 - mu * mu
        M = [1.0, mu, mu * mu + v, mu ** 3 + 3 * mu * v, mu ** 4 + 6 * mu * mu * v + 3 * v * v]
        # (p0 + p1 X + p2 X^2)^2
        c = [p0 * p0, 2 * p0 * p1, p1 * p1 + 2 * p0 * p2, 2 * p1 * p2, p2 * p2]
        return sum(ci * Mi for ci, Mi in zip(c, M))

    a1 = b * integrate.quad(integrand, 0.0, t, epsabs=1e-13, epsrel=1e-12)[0]
    assert abs(a[1] - a1) <= 4.5 * se[1], (a[1], a1, se[1])


def test_invalid_sde_rejected(oracle_mod):
    pb = dict(dim=1, D=0.0, f_coef=[0.0], u0=("const", (1.0,)), strategy="B", q=0.5,
              sde=(0, (0.0,), (0.0,), (1.0,), (0.0,)))
    with pytest.raises(ValueError):
        oracle_mod.trees(pb, [0.0], 0.5, 0, 0, 4, 4, 0)
