"""Pin: the oracle's per-order standard errors SE_n (Sec. 2.4, Eq. simplecase_discrete: a_n is
the sample mean of the trees' order-n contributions, so its error is O(N^{-1/2}) and is estimated
from the same trees).

SE_n^2 is meant to be an unbiased estimate of Var(a_n) = Var(contribution)/N.  Two checks that do
not reuse the oracle's formula:

  * a closed form: with constant initial data c under Strategy B a tree has order 0 with
    probability P(leaf) = q (the word threshold of q) and then contributes g/P(leaf) = c/P(leaf),
    else 0 to order 0.  So Var(a_0) = c^2 (1/P(leaf) - 1)/N exactly, and the mean of SE_0^2 over
    many independent replicas must match it.  Dropping the "- a^2" term of the variance makes the
    mean 4x too large at N = 4, dividing by N instead of N - 1 makes it 0.75x: both fail.
  * calibration: over independent replicas (distinct point streams and 40 seeds) the spread of
    a_n equals the mean of SE_n^2, order by order, for Gaussian initial data in 2-D.
"""
import numpy as np

import workloads


def _replicas(oracle_mod, pb, x, t, ntrees, K, copies, seed):
    d = pb["dim"]
    xs = np.tile(np.asarray(x, float).reshape(1, d), (copies, 1))
    return oracle_mod.solve(pb, xs, np.full(copies, t), np.full(copies, ntrees, np.uint64), K, K // 2,
                            K - K // 2, seed)


def test_order0_standard_error_matches_the_closed_form(oracle_mod):
    c, q, N, P = 0.8, 2.0 / 3.0, 4, 40_000
    pb = dict(dim=1, D=0.5, f_coef=[0.0, 0.0, 1.0], u0=("const", (c,)), strategy="B", lam=1.0, c_pot=0.0, q=q,
              arity_law="uniform")
    r = _replicas(oracle_mod, pb, [0.3], 0.7, N, 4, P, seed=5)
    p_leaf = round(q * 2.0 ** 32) / 2.0 ** 32  # the leaf probability the 32-bit threshold realises
    var_a0 = c * c * (1.0 / p_leaf - 1.0) / N
    mean_se2 = float(np.mean(r["se"][:, 0] ** 2))
    spread = float(np.var(r["coef"][:, 0], ddof=1))
    # the standard error of mean_se2 over P replicas is ~1 % here; 5 % leaves room and still
    # rejects a dropped -a^2 (x4) or a divisor N instead of N - 1 (x0.75)
    assert abs(mean_se2 / var_a0 - 1.0) < 0.05, (mean_se2, var_a0)
    assert abs(spread / var_a0 - 1.0) < 0.05, (spread, var_a0)
    # a_0 itself: mean c (the order-0 term of the eps series of u' = u^2 from c)
    assert abs(np.mean(r["coef"][:, 0]) - c) < 5 * np.sqrt(var_a0 / P)


def test_standard_errors_match_the_spread_over_seeds(oracle_mod):
    pb = dict(workloads.problem_sin_2d(), precision="fp64")
    pb["f_coef"] = [0.0, 0.0, 1.0]
    pb["q"] = 2.0 / 3.0
    pb["arity_law"] = "uniform"
    K, N, P, seeds = 8, 500, 100, 40
    a, se2 = [], []
    for seed in range(seeds):
        r = _replicas(oracle_mod, pb, [0.4, -0.3], 0.6, N, K, P, seed)
        a.append(r["coef"])
        se2.append(r["se"] ** 2)
    a = np.concatenate(a)
    se2 = np.concatenate(se2)
    # binary trees with q = 2/3 have order n with probability Catalan(n) q^{n+1} (1-q)^n: 333, 74, 33,
    # 18 of the 500 trees for n = 0..3, enough for both estimates of Var(a_n) to settle
    for n in range(4):
        ratio = np.var(a[:, n], ddof=1) / np.mean(se2[:, n])
        assert 0.85 < ratio < 1.18, (n, ratio)
