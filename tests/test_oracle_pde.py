"""Pins of the whole oracle pipeline (trees -> series -> Pade) on nonlinear PDEs.

* Example 3 (Sec. 2.4) after correcting its misprint: the travelling wave
  u = 1/(1 + exp(-(x + sqrt(2)(1/2 - a) t)/sqrt(2))) solves
  u_t = u_xx - a u + (1+a) u^2 - u^3 exactly (checked symbolically here), not the
  printed u_t = u_xx - (1+a) u^2 - u^3.
* Examples 1 and 2 (Sec. 2.4) and the 1-D KPP workload against a fine
  Crank-Nicolson finite-difference solve, the paper's own check (Sec. 2.4,
  before Example 1).
The Monte Carlo error of a Pade value is estimated by a delete-one jackknife
over independent replicas; the tolerance adds the CN and Pade truncation error.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from checkers import crank_nicolson_1d

A_WAVE = 0.25


def test_example3_corrected_form_is_exact():
    sp = pytest.importorskip("sympy")
    x, t, a = sp.symbols("x t a")
    u = 1 / (1 + sp.exp(-(x + sp.sqrt(2) * (sp.Rational(1, 2) - a) * t) / sp.sqrt(2)))
    corrected = sp.diff(u, t) - sp.diff(u, x, 2) - (-a * u + (1 + a) * u ** 2 - u ** 3)
    assert sp.simplify(corrected) == 0
    printed = sp.diff(u, t) - sp.diff(u, x, 2) - (-(1 + a) * u ** 2 - u ** 3)
    assert abs(float(printed.subs({x: 0.3, t: 0.2, a: A_WAVE}).evalf())) > 0.1


def _replicated_pade(pb, x, t, N, K, L, M, reps=8, seed0=100):
    x = np.asarray(x, float).reshape(-1, pb["dim"])
    R = [oracle.solve(pb, x, np.full(len(x), t), np.full(len(x), N, np.uint64), K, L, M, seed0 + r)["coef"]
         for r in range(reps)]
    C = np.mean(R, axis=0)
    u = np.array([oracle.pade(C[p], L, M)[0] for p in range(len(x))])
    jk = np.array([[oracle.pade(np.mean([R[j][p] for j in range(reps) if j != i], axis=0), L, M)[0]
                    for p in range(len(x))] for i in range(reps)])
    se = np.sqrt((reps - 1) / reps * ((jk - jk.mean(axis=0)) ** 2).sum(axis=0))
    return u, se


@pytest.mark.parametrize("strategy,extra,L", [("A", dict(lam=1.0, c_pot=A_WAVE), 3), ("B", dict(q=0.75), 2)])
def test_travelling_wave(strategy, extra, L):
    w = math.sqrt(2.0)
    pb = dict(dim=1, D=1.0, f_coef=[0.0, -A_WAVE, 1 + A_WAVE, -1.0], u0=("logistic", (0.0, 1.0, 0.0, w)),
              strategy=strategy, arity_law="uniform", **extra)
    xs = np.array([-1.0, 0.0, 0.8])
    t = 0.25
    u, se = _replicated_pade(pb, xs, t, 100_000, 2 * L, L, L)
    exact = 1.0 / (1.0 + np.exp(-(xs + math.sqrt(2) * (0.5 - A_WAVE) * t) / w))
    assert np.all(np.abs(u - exact) <= 4.5 * se + 2e-3), (u, exact, se)


@pytest.mark.parametrize("b,amp,strategy", [(-1.0, 1.0, "B"), (-1.0, 1.0, "A"), (1.0, -6.0, "B")])
def test_examples_1_and_2_against_crank_nicolson(b, amp, strategy):
    T = 0.5

    def g(z):
        return amp * np.exp(-z * z / 4) / math.sqrt(4 * math.pi)

    xg, ug = crank_nicolson_1d(lambda u: b * u * u, lambda u: 2 * b * u, g, 1.0, T, 20.0, 0.02, 5e-4,
                               lambda tt: 0.0)
    ref = float(np.interp(0.0, xg, ug))
    extra = dict(q=2.0 / 3.0) if strategy == "B" else dict(lam=1.0, c_pot=0.0)
    pb = dict(dim=1, D=1.0, f_coef=[0.0, 0.0, b], u0=("gauss", (0.0, amp / math.sqrt(4 * math.pi), math.sqrt(2), 0.0)),
              strategy=strategy, arity_law="uniform", **extra)
    u, se = _replicated_pade(pb, [0.0], T, 100_000, 8, 4, 4, seed0=200)
    assert abs(u[0] - ref) <= 4.5 * se[0] + 2e-4, (u[0], ref, se[0])


def test_kpp_workload_against_crank_nicolson():
    wl = workloads.workload_kpp_1d()
    pb = wl["problem"]
    c0 = 0.5  # u0 -> 0.5 far away: boundary data from the ODE u' = u^2 - u

    def bc(tt):
        return 1.0 / (1.0 + (1.0 / c0 - 1.0) * math.exp(tt))

    xg, ug = crank_nicolson_1d(lambda u: u * u - u, lambda u: 2 * u - 1, lambda z: 0.5 + 0.3 * np.exp(-z * z),
                               pb["D"], 0.5, 12.0, 0.02, 5e-4, bc)
    ref = np.interp(wl["x"][:, 0], xg, ug)
    N = 100_000
    r = oracle.solve(pb, wl["x"], wl["t"], np.full(16, N, np.uint64), wl["K"], wl["L"], wl["M"], 0)
    # the series converges fast here (McKean: weights are products of g <= 0.8), so the standard
    # error of the total tree weight bounds the error of the Pade sum
    S1, S2 = r["s1"].sum(axis=1), r["s2"].sum(axis=1)
    mean = S1 / N
    se = np.sqrt((S2 / N - mean * mean) / (N - 1))
    assert np.all(r["status"] == 0)
    assert np.all(np.abs(r["u"] - ref) <= 4.5 * se + 1e-5), (r["u"] - ref, se)
