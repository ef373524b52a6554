"""Pins of the oracle's tree topology against the laws the paper and textbook theory fix.

* Strategy B, m-ary trees: P(Ne = n) = q^k (1-q)^n N_D(n, m), k = (m-1) n + 1 leaves,
  N_D(n, m) = C(mn+1, n)/(mn+1) (Fuss-Catalan; Sec. 2.3, Eq. pfinal; Catalan for m = 2).
* Strategy B, several terms: the Galton-Watson generating function
  G(z) = q + (1-q) z sum_k p_k G(z)^k, solved here as a power series.
* Mean number of leaves <k> = q / (1 - m (1-q)) (Sec. 2.3, after Eq. aproxTb).
* Strategy A with binary splitting at rate lambda: the Yule law
  P(Ne = n) = e^{-lambda t} (1 - e^{-lambda t})^n.
Each is checked by a chi-square test on 2e5 trees.
"""
import math

import numpy as np
import pytest
from scipy import stats

N_TREES = 200_000


def _prob(dim=1, f_coef=(0.0, 0.0, 1.0), strategy="B", q=0.6, lam=1.0, c_pot=0.0, law="uniform"):
    return dict(dim=dim, D=1.0, f_coef=list(f_coef), u0=("const", (1.0,)), strategy=strategy, lam=lam,
                c_pot=c_pot, q=q, arity_law=law)


def _chi2_pvalue(counts, probs):
    counts = np.asarray(counts, float)
    e = np.asarray(probs, float) * counts.sum()
    # merge tail bins with small expectation into their left neighbour
    obs, exp = [], []
    co, ce = 0.0, 0.0
    for c_, e_ in zip(counts, e):
        co += c_
        ce += e_
        if ce >= 20:
            obs.append(co)
            exp.append(ce)
            co, ce = 0.0, 0.0
    if ce > 0:
        obs[-1] += co
        exp[-1] += ce
    obs, exp = np.array(obs), np.array(exp)
    chi2 = ((obs - exp) ** 2 / exp).sum()
    return stats.chi2.sf(chi2, len(obs) - 1)


def _order_histogram(oracle_mod, pb, K, t=1.0, seed=7):
    r = oracle_mod.trees(pb, [0.0] * pb["dim"], t, 3, 0, N_TREES, K, seed)
    return np.bincount(r["order"], minlength=K + 2)[: K + 2], r


def _fuss_catalan(n, m):
    return math.comb(m * n + 1, n) / (m * n + 1)


@pytest.mark.parametrize("m,q", [(2, 0.6), (2, 2.0 / 3.0), (3, 0.75)])
def test_strategy_b_mary_law_matches_pfinal(oracle_mod, m, q):
    K = 16
    f = [0.0] * (m + 1)
    f[m] = 1.0
    hist, _ = _order_histogram(oracle_mod, _prob(f_coef=f, q=q), K)
    p = [q ** ((m - 1) * n + 1) * (1 - q) ** n * _fuss_catalan(n, m) for n in range(K + 1)]
    p.append(1.0 - sum(p))
    assert _chi2_pvalue(hist, p) > 1e-4


def _gw_law(q, terms, K):
    """P(Ne = n), n <= K, of the Galton-Watson tree with leaf prob q and term law {k: p_k}."""
    G = np.zeros(K + 1)
    G[0] = q
    for _ in range(K + 2):
        acc = np.zeros(K + 1)
        for k, pk in terms.items():
            pw = np.zeros(K + 1)
            pw[0] = 1.0
            for _ in range(k):
                pw = np.convolve(pw, G)[: K + 1]
            acc += pk * pw
        newG = np.zeros(K + 1)
        newG[0] = q
        newG[1:] = (1 - q) * acc[:K]
        G = newG
    return G


@pytest.mark.parametrize("f_coef,law,q", [
    ((0.0, 0.0, 1.0, 1.0), "uniform", 0.7),          # u^2 + u^3, alpha uniform on {2,3}
    ((0.0, 0.0, 1.0, -3.0), "abs", 0.7),             # p_2 = 1/4, p_3 = 3/4
    ((0.0, 1.0, 0.0, -1.0), "uniform", 2.0 / 3.0),   # u - u^3: an arity-1 term
    ((0.5, 0.0, 1.0), "abs", 0.55),                  # constant term: arity-0 internal nodes
])
def test_strategy_b_multiterm_law_matches_generating_function(oracle_mod, f_coef, law, q):
    K = 12
    terms = {k: abs(b) for k, b in enumerate(f_coef) if b != 0.0}
    s = sum(terms.values())
    if law == "uniform":
        terms = {k: 1.0 / len(terms) for k in terms}
    else:
        terms = {k: v / s for k, v in terms.items()}
    hist, _ = _order_histogram(oracle_mod, _prob(f_coef=f_coef, q=q, law=law), K)
    G = _gw_law(q, terms, K)
    p = list(G) + [1.0 - G.sum()]
    assert _chi2_pvalue(hist, p) > 1e-4


def test_mean_leaves_matches_closed_form(oracle_mod):
    q, m = 0.85, 2
    _, r = _order_histogram(oracle_mod, _prob(f_coef=(0.0, 0.0, 1.0), q=q), 16)
    kept = r["order"] <= 16
    assert kept.sum() >= len(kept) - 2  # P(Ne > 16) ~ 1e-7 at q = 0.85
    leaves = r["nodes"][kept].astype(float) - r["order"][kept]
    mean = leaves.mean()
    se = leaves.std() / math.sqrt(len(leaves))
    expect = q / (1 - m * (1 - q))
    assert abs(mean - expect) < 4.5 * se


@pytest.mark.parametrize("lam,t", [(1.0, 0.5), (1.3, 0.8)])
def test_strategy_a_binary_yule_law(oracle_mod, lam, t):
    K = 16
    # F = f + c u = u^2 with f = u^2 - c u: binary splitting at rate lambda
    pb = _prob(f_coef=(0.0, -0.7, 1.0), strategy="A", lam=lam, c_pot=0.7)
    hist, _ = _order_histogram(oracle_mod, pb, K, t=t)
    e = math.exp(-lam * t)
    p = [e * (1 - e) ** n for n in range(K + 1)]
    p.append(1.0 - sum(p))
    assert _chi2_pvalue(hist, p) > 1e-4


def test_tree_records_do_not_depend_on_the_range_split(oracle_mod):
    pb = _prob(dim=2, f_coef=(0.0, 1.0, 0.0, -1.0), q=0.6)
    pb["u0"] = ("gauss", (0.1, 1.0, 0.7, 0.2, -0.3))
    full = oracle_mod.trees(pb, [0.3, -0.2], 0.9, 5, 0, 3000, 10, 42)
    part = oracle_mod.trees(pb, [0.3, -0.2], 0.9, 5, 1234, 1000, 10, 42)
    for key in ("order", "w", "nodes", "hash"):
        assert np.array_equal(full[key][1234:2234], part[key])
    other_point = oracle_mod.trees(pb, [0.3, -0.2], 0.9, 6, 1234, 1000, 10, 42)
    assert not np.array_equal(other_point["hash"], part["hash"])
    other_seed = oracle_mod.trees(pb, [0.3, -0.2], 0.9, 5, 1234, 1000, 10, 43)
    assert not np.array_equal(other_seed["hash"], part["hash"])


def test_branching_thresholds_realise_the_law(oracle_mod):
    pb = _prob(f_coef=(0.0, 1.0, 0.0, -1.0 / 6.0, 0.0, 1.0 / 120.0), q=0.49, law="abs")
    tb = oracle_mod.setup_tables(pb)
    thr = tb["thr"].astype(np.float64) / 2**32
    assert list(tb["arity"]) == [1, 3, 5]
    assert thr[-1] == 1.0
    assert abs(thr[0] - 0.49) < 2**-32
    sabs = 1 + 1 / 6 + 1 / 120
    assert abs(thr[1] - (0.49 + 0.51 / sabs)) < 2**-31
    # weights are b_k / P_k with the realised probabilities: unbiased for any threshold rounding
    P = np.diff(np.concatenate([[0.0], thr]))
    assert np.allclose(tb["term_factor"] * P[1:], tb["coef"], rtol=1e-15, atol=0)
    assert abs(tb["leaf_factor"] * P[0] - 1.0) < 1e-15


def test_cost_versus_final_time(oracle_mod):
    """Sec. 2.4 / Fig. 6: Strategy B's work does not grow with t the way Strategy A's does.  Here
    segments are exact, so under Strategy B a tree's topology (coin and term draws) does not
    depend on t at all -- the same streams give the same trees and node counts for every t --
    while under Strategy A the expected number of splits grows with t (Yule: e^{lambda t} - 1
    for binary trees before pruning)."""
    import numpy as np

    pb_b = dict(dim=1, D=0.5, f_coef=[0.0, 0.0, 1.0], u0=("const", (0.5,)), strategy="B", q=2.0 / 3.0)
    ref = oracle_mod.trees(pb_b, [0.0], 0.1, 0, 0, 4000, 12, 3)
    for t in (0.5, 1.0, 4.0):
        r = oracle_mod.trees(pb_b, [0.0], t, 0, 0, 4000, 12, 3)
        assert np.array_equal(r["hash"], ref["hash"]) and np.array_equal(r["nodes"], ref["nodes"])
    pb_a = dict(pb_b, strategy="A", lam=1.0, c_pot=0.0)
    means = [oracle_mod.trees(pb_a, [0.0], t, 0, 0, 4000, 16, 3)["nodes"].mean() for t in (0.25, 0.5, 1.0)]
    assert means[0] < means[1] < means[2]
