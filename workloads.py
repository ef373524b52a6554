"""Seeded synthetic workloads for the generalized-random-tree point solve.

This module holds the problem descriptions and the seeded point sets only: no
step of the method's arithmetic.  Both the CUDA path (through its binding) and
the CPU oracle take their inputs from here; neither side imports the other.

A problem is a plain dict:
    dim, D, f_coef=[b_0..b_deg], u0=(kind, params), strategy "A"|"B",
    lam, c_pot (Strategy A), q (Strategy B), arity_law "uniform"|"abs",
    precision "fp32"|"fp64".
A workload adds the points: x [n, dim], t [n], ntrees [n], K, L, M, seed.

The five workloads below follow the paper's test problems and its
probabilistic-domain-decomposition set-up (Sec. 2.4 Examples 1-3, Sec. 3):
    kpp_1d     u_t = u_xx + u^2 - u (McKean's KPP case, Eq. KPP-1D), 1-D, FP64
    sin_2d     u_t = 0.5 Lap u + sin(u) (sin as its degree-9 Taylor polynomial)
    uneven_2d  u_t = Lap u + u^2 on PDD interface points, uneven tree budgets
    pdd_3d     u_t = 0.1 Lap u + u - u^3 on the 9 interior planes of a 4x4x4 split
    var_coef_2d  u_t = Lap u - e^{-x^2}/(t + 0.1) u^2 (Sec. 3 Example 5: a variable
               coefficient on the nonlinear term), u0 = e^{-x^2/4}/sqrt(4 pi), t = 0.5
    drift_2d   u_t = L u + u^2 - u with a general operator
               L = sum_i (s_i^2 / 2) d_ii - kappa_i x_i d_i (anisotropic Ornstein-Uhlenbeck
               paths, Euler-Maruyama, Eqs. green and SDE), t = 0.5
"""
from __future__ import annotations

import math

import numpy as np


def mean_arity(f_coef, arity_law: str, extra_linear: float = 0.0) -> float:
    """E_p[k] of the branching law over the nonzero terms of f (+ c u)."""
    terms = []
    for k, b in enumerate(f_coef):
        b = b + (extra_linear if k == 1 else 0.0)
        if b != 0.0:
            terms.append((k, abs(b)))
    if not terms:
        return 0.0
    if arity_law == "abs":
        s = sum(a for _, a in terms)
        return sum(k * a for k, a in terms) / s
    return sum(k for k, _ in terms) / len(terms)


def default_q(f_coef, arity_law: str) -> float:
    """Leaf probability giving a Galton-Watson mean offspring of 2/3.

    The tree is a Galton-Watson process with mean offspring (1-q) E_p[k]; the
    paper's admissibility bound (Sec. 2.3, Eqs. q and qgen) is the boundary
    (1-q) E_p[k] = 1.  Choosing 2/3 gives q = 2/3 for binary trees, a value the
    paper itself uses (Fig. 6).
    """
    m = mean_arity(f_coef, arity_law)
    return 1.0 - 2.0 / (3.0 * m) if m > 0 else 0.5


SIN9 = [0.0, 1.0, 0.0, -1.0 / 6.0, 0.0, 1.0 / 120.0, 0.0, -1.0 / 5040.0, 0.0, 1.0 / 362880.0]


def problem_kpp_1d() -> dict:
    return dict(dim=1, D=1.0, f_coef=[0.0, -1.0, 1.0], u0=("gauss", (0.5, 0.3, 1.0 / math.sqrt(2.0), 0.0)),
                strategy="A", lam=1.0, c_pot=1.0, q=0.5, arity_law="uniform", precision="fp64")


def problem_sin_2d() -> dict:
    return dict(dim=2, D=0.5, f_coef=list(SIN9), u0=("gauss", (0.0, 1.2, 1.0, 0.0, 0.0)), strategy="B",
                lam=1.0, c_pot=0.0, q=default_q(SIN9, "abs"), arity_law="abs", precision="fp32")


def problem_uneven_2d() -> dict:
    return dict(dim=2, D=1.0, f_coef=[0.0, 0.0, 1.0], u0=("cos_prod", (1.5, 0.5, 1.0, 1.0)), strategy="B",
                lam=1.0, c_pot=0.0, q=2.0 / 3.0, arity_law="uniform", precision="fp32")


def problem_pdd_3d() -> dict:
    return dict(dim=3, D=0.1, f_coef=[0.0, 1.0, 0.0, -1.0], u0=("tanh_prod", (0.0, 1.0, 2.0, 2.0, 2.0)),
                strategy="B", lam=1.0, c_pot=0.0, q=2.0 / 3.0, arity_law="uniform", precision="fp32")


def problem_var_coef_2d(strategy: str = "B", precision: str = "fp32") -> dict:
    """Example 5: c_2(x, t) = -e^{-x_0^2} / (t + 0.1), binary trees, u0 a function of x_0 alone."""
    return dict(dim=2, D=1.0, f_coef=[0.0, 0.0, -1.0], u0=("gauss_axes", (0.0, 1.0 / math.sqrt(4.0 * math.pi),
                                                                       0.25, 0.0, 0.0, 0.0, 0.0, 0.0)),
                coef=("gauss_over_t", (1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.1), [2]), strategy=strategy, lam=1.0,
                c_pot=0.0, q=2.0 / 3.0, arity_law="uniform", precision=precision)


def problem_drift_2d(strategy: str = "B", precision: str = "fp32", steps: int = 8) -> dict:
    """General drift and diffusion: OU paths dX_i = -kappa_i X_i dt + s_i dW_i, kappa = (1, 0.5), s = (1, 0.7)."""
    return dict(dim=2, D=0.0, f_coef=[0.0, -1.0, 1.0], u0=("gauss", (0.0, 1.0, 0.8, 0.5, -0.3)),
                sde=(steps, (0.0, 0.0), (1.0, 0.5), (1.0, 0.7), (0.0, 0.0)), strategy=strategy, lam=1.0, c_pot=0.0,
                q=default_q([0.0, -1.0, 1.0], "uniform"), arity_law="uniform", precision=precision)


def workload_kpp_1d() -> dict:
    x = np.linspace(-2.0, 2.0, 16).reshape(-1, 1)
    n = x.shape[0]
    return dict(name="kpp_1d", problem=problem_kpp_1d(), x=x, t=np.full(n, 0.5), ntrees=np.full(n, 10_000, np.uint64),
                K=8, L=4, M=4, seed=0)


def workload_sin_2d() -> dict:
    g = np.linspace(-3.0, 3.0, 16)
    X, Y = np.meshgrid(g, g, indexing="ij")
    xy = np.stack([X.ravel(), Y.ravel()], axis=1)
    x = np.concatenate([xy, xy], axis=0)
    t = np.concatenate([np.full(len(xy), 0.25), np.full(len(xy), 1.0)])
    return dict(name="sin_2d", problem=problem_sin_2d(), x=x, t=t, ntrees=np.full(len(t), 100_000, np.uint64),
                K=10, L=5, M=5, seed=0)


def interface_segments_8x8() -> list:
    """The 112 interior unit segments of the 8x8 unit-square split of [0,8]^2."""
    segs = []
    for i in range(1, 8):          # vertical interfaces x = i
        for j in range(8):
            segs.append(((float(i), float(j)), (float(i), float(j + 1))))
    for j in range(1, 8):          # horizontal interfaces y = j
        for i in range(8):
            segs.append(((float(i), float(j)), (float(i + 1), float(j))))
    return segs


def workload_uneven_2d(seed: int = 0) -> dict:
    rng = np.random.default_rng(seed)
    segs = interface_segments_8x8()
    pick = rng.choice(len(segs), size=64, replace=False)
    pts = []
    for s in sorted(pick):
        (x0, y0), (x1, y1) = segs[s]
        f = (np.arange(64) + 0.5) / 64.0
        pts.append(np.stack([x0 + f * (x1 - x0), y0 + f * (y1 - y0)], axis=1))
    x = np.concatenate(pts, axis=0)
    n = x.shape[0]
    t = rng.uniform(0.1, 2.0, size=n)
    ntrees = np.exp(rng.uniform(math.log(1e3), math.log(1e6), size=n)).astype(np.uint64)
    # u0 lies in [1, 2] and f = u^2: by comparison with the ODE u' = u^2 from 1 and from 2 the
    # solution blows up somewhere in t in [1/2, 1] and everywhere by t = 1, so points at t >= 1/2
    # may lie past blow-up, where the Pade value continues the series and no PDE value exists
    past_blowup = t >= 0.5
    return dict(name="uneven_2d", problem=problem_uneven_2d(), x=x, t=t, ntrees=ntrees, K=16, L=8, M=8, seed=0,
                past_blowup=past_blowup)


def workload_pdd_3d() -> dict:
    c = (np.arange(32) + 0.5) / 8.0
    A, B = np.meshgrid(c, c, indexing="ij")
    a, b = A.ravel(), B.ravel()
    pts = []
    for axis in range(3):
        for plane in (1.0, 2.0, 3.0):
            p = np.empty((a.size, 3))
            others = [i for i in range(3) if i != axis]
            p[:, axis] = plane
            p[:, others[0]] = a
            p[:, others[1]] = b
            pts.append(p)
    x = np.concatenate(pts, axis=0)
    n = x.shape[0]
    return dict(name="pdd_3d", problem=problem_pdd_3d(), x=x, t=np.full(n, 1.0), ntrees=np.full(n, 100_000, np.uint64),
                K=12, L=6, M=6, seed=0)


def workload_var_coef_2d() -> dict:
    g = np.linspace(-3.0, 3.0, 16)
    X, Y = np.meshgrid(g, g, indexing="ij")
    x = np.stack([X.ravel(), Y.ravel()], axis=1)
    n = x.shape[0]
    return dict(name="var_coef_2d", problem=problem_var_coef_2d(), x=x, t=np.full(n, 0.5),
                ntrees=np.full(n, 100_000, np.uint64), K=8, L=4, M=4, seed=0)


def workload_drift_2d() -> dict:
    g = np.linspace(-3.0, 3.0, 16)
    X, Y = np.meshgrid(g, g, indexing="ij")
    x = np.stack([X.ravel(), Y.ravel()], axis=1)
    n = x.shape[0]
    return dict(name="drift_2d", problem=problem_drift_2d(), x=x, t=np.full(n, 0.5),
                ntrees=np.full(n, 100_000, np.uint64), K=8, L=4, M=4, seed=0)


WORKLOADS = {
    "kpp_1d": workload_kpp_1d,
    "sin_2d": workload_sin_2d,
    "uneven_2d": workload_uneven_2d,
    "pdd_3d": workload_pdd_3d,
    "var_coef_2d": workload_var_coef_2d,
    "drift_2d": workload_drift_2d,
}


def subsample(wl: dict, npoints: int, ntrees: int | None = None, stride: int | None = None) -> dict:
    """A smaller copy of a workload: every `stride`-th point, optionally fewer trees per point.

    Point indices of the subsample are its own 0..n-1; callers that want the
    full workload's random streams pass point_base / index lists themselves.
    """
    n = wl["x"].shape[0]
    if stride is None:
        stride = max(1, n // max(npoints, 1))
    idx = np.arange(0, n, stride)[:npoints]
    out = dict(wl)
    out["x"] = wl["x"][idx].copy()
    out["t"] = wl["t"][idx].copy()
    nt = wl["ntrees"][idx].copy()
    if ntrees is not None:
        nt = np.minimum(nt, np.uint64(ntrees)).astype(np.uint64)
    out["ntrees"] = nt
    out["index"] = idx
    if "past_blowup" in wl:
        out["past_blowup"] = np.asarray(wl["past_blowup"])[idx].copy()
    return out


def random_points(rng: np.random.Generator, n: int, dim: int, lo: float = -3.0, hi: float = 3.0) -> np.ndarray:
    return rng.uniform(lo, hi, size=(n, dim))


# ----------------------------------------------------------------------------
# serving trace: Poisson arrivals of point-solve requests
# ----------------------------------------------------------------------------
def serving_problems(precision: str = "fp32") -> dict:
    """The nine request problems: f in {u^2 - u, sin u, u - u^3} x d in {1, 2, 3} (Strategy B).

    Diffusion constants 1, 0.5, 0.1 for the three f; u0 as in the other workloads.
    Series shapes: K = 8 [4/4], 10 [5/5], 12 [6/6].
    """
    out = {}
    fs = {
        "u2-u": ([0.0, -1.0, 1.0], "uniform", 1.0, lambda d: ("gauss", (0.5, 0.3) + (1 / math.sqrt(2.0),) + (0.0,) * d), 8),
        "sin": (list(SIN9), "abs", 0.5, lambda d: ("gauss", (0.0, 1.2, 1.0) + (0.0,) * d), 10),
        "u-u3": ([0.0, 1.0, 0.0, -1.0], "uniform", 0.1, lambda d: ("tanh_prod", (0.0, 1.0) + (0.3,) * d), 12),
    }
    for fname, (coef, law, D, u0, K) in fs.items():
        for d in (1, 2, 3):
            out[(fname, d)] = dict(problem=dict(dim=d, D=D, f_coef=list(coef), u0=u0(d), strategy="B",
                                                q=default_q(coef, law), arity_law=law, precision=precision),
                                   K=K, L=K // 2, M=K // 2)
    return out


def serving_trace(n_requests: int, rate_per_s: float, seed: int = 0, max_points: int = 4096,
                  trees_lo: float = 1e3, trees_hi: float = 1e7) -> list:
    """Seeded Poisson arrivals; points per request log-uniform in [1, max_points], tree budgets
    per point log-uniform in [trees_lo, trees_hi], problem uniform over serving_problems().
    The requests draw from one service-wide stream key (Philox key = the trace's seed) and get
    disjoint point streams (point_base = the points of the requests before them), so requests
    of the same problem and orders may share a walk launch."""
    rng = np.random.default_rng(seed)
    keys = sorted(serving_problems().keys())
    t_arr = 0.0
    out = []
    base = 0
    for k in range(n_requests):
        t_arr += rng.exponential(1.0 / rate_per_s)
        key = keys[int(rng.integers(0, len(keys)))]
        n = int(np.clip(np.exp(rng.uniform(0.0, math.log(max_points))), 1, max_points))
        d = key[1]
        x = rng.uniform(-3.0, 3.0, size=(n, d))
        t = rng.uniform(0.1, 1.0, size=n)
        nt = np.exp(rng.uniform(math.log(trees_lo), math.log(trees_hi), size=n)).astype(np.uint64)
        out.append(dict(arrival=t_arr, key=key, x=x, t=t, ntrees=nt, seed=seed, point_base=base))
        base += n
    return out


def serving_mean_trees(max_points: int = 4096, trees_lo: float = 1e3, trees_hi: float = 1e7) -> float:
    """Expected trees per request of serving_trace (log-uniform points x log-uniform budgets)."""
    mp = (max_points - 1) / math.log(max_points)
    mt = (trees_hi - trees_lo) / math.log(trees_hi / trees_lo)
    return mp * mt
