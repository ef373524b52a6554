"""FP64 CPU oracle of the generalized-random-tree point solve.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import this package.  The
product library never imports, links or calls it, and this package imports
nothing from the product package: it has its own C walker, its own Philox and
its own Pade solver (``grt_oracle.c``), and its own marshalling of the problem
description below.

Problem descriptions are plain dicts (see ``workloads.py``):

    dim        d in {1, 2, 3}
    D          diffusion constant (L = D * Laplacian)
    f_coef     [b_0, ..., b_deg], f(u) = sum_k b_k u^k, deg <= 15
    u0         (kind, params): "const" (c,), "gauss" (c0, A, s, x0...),
               "cos_prod" (c0, A, w_0, w_1, w_2), "tanh_prod" (c0, A, s_0, s_1, s_2),
               "logistic" (c0, A, x0, width), "gauss_axes" (c0, A, w_0, w_1, w_2, m_0, m_1, m_2):
               c0 + A exp(-sum_i w_i (x_i - m_i)^2)
    strategy   "A" (exponential clock, Sec. 2.1) or "B" (coin + uniform split, Sec. 2.2)
    lam, c_pot Strategy A clock rate and pulled-out potential
    q          Strategy B leaf probability
    arity_law  "uniform" (paper, Sec. 2.1 after Eq. probexp2) or "abs" (p_k ~ |b_k|)
    coef       optional (kind, params, powers): variable coefficients c_k(x, t) = b_k gamma(x, t)
               for k in powers (Sec. 1, Eq. nonlinear_new; Example 5); kinds
               "gauss_over_t" exp(-sum w_i (x_i - m_i)^2) / (t + t0), params (w0, w1, w2, m0, m1, m2, t0),
               and "gauss" exp(-sum w_i (x_i - m_i)^2), params (w0, w1, w2, m0, m1, m2)
    sde        optional (steps, beta, kappa, s, r): paths of dX_i = (beta_i - kappa_i X_i) dt
               + (s_i + r_i X_i) dW_i by Euler-Maruyama, `steps` equal steps per segment
               (D is then unused); u0 kind "quadratic" (c0, l_0, l_1, l_2, q_0, q_1, q_2):
               c0 + sum_i (l_i x_i + q_i x_i^2)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "grt_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

MAX_DEG = 15
MAX_K = 16

STATUS_PADE_SINGULAR = 1
STATUS_PADE_POLE_NEAR = 2
STATUS_SERIES_PARTIAL = 4
STATUS_HIGH_PRUNE = 8

_U0_KINDS = {"const": 0, "gauss": 1, "cos_prod": 2, "tanh_prod": 3, "logistic": 4, "gauss_axes": 5, "quadratic": 6}
_COEF_KINDS = {"const": 0, "gauss_over_t": 1, "gauss": 2}


class _OrProblem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32),
        ("D", ctypes.c_double),
        ("f_deg", ctypes.c_int32),
        ("f_coef", ctypes.c_double * (MAX_DEG + 1)),
        ("u0_kind", ctypes.c_int32),
        ("u0_param", ctypes.c_double * 8),
        ("strategy", ctypes.c_int32),
        ("lam", ctypes.c_double),
        ("c_pot", ctypes.c_double),
        ("q", ctypes.c_double),
        ("arity_law", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("coef_kind", ctypes.c_int32),
        ("coef_param", ctypes.c_double * 8),
        ("coef_mask", ctypes.c_uint32),
        ("sde_kind", ctypes.c_int32),
        ("sde_steps", ctypes.c_int32),
        ("sde_param", ctypes.c_double * 12),
    ]


def build(force: bool = False) -> str:
    """Compile ``grt_oracle.c`` into ``liboracle.so`` with gcc (plain -O2, IEEE math)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER
        u32p, u64p, i32p, f64p = P(ctypes.c_uint32), P(ctypes.c_uint64), P(ctypes.c_int32), P(ctypes.c_double)
        lib.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
        lib.oracle_philox4x32_10.restype = None
        lib.oracle_uniform.argtypes = [ctypes.c_uint32]
        lib.oracle_uniform.restype = ctypes.c_double
        lib.oracle_trees.argtypes = [P(_OrProblem), f64p, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64,
                                     ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64, i32p, f64p, u32p, u64p]
        lib.oracle_trees.restype = ctypes.c_int
        lib.oracle_pade.argtypes = [ctypes.c_int, ctypes.c_int, f64p, f64p, i32p, i32p]
        lib.oracle_pade.restype = ctypes.c_int
        lib.oracle_solve.argtypes = [P(_OrProblem), ctypes.c_int64, f64p, f64p, u64p, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, f64p, f64p,
                                     f64p, i32p, f64p, f64p, f64p, u64p, u64p]
        lib.oracle_solve.restype = ctypes.c_int
        lib.oracle_setup_tables.argtypes = [P(_OrProblem), i32p, i32p, f64p, u64p, f64p, f64p]
        lib.oracle_setup_tables.restype = ctypes.c_int
        lib.oracle_u0.argtypes = [P(_OrProblem), f64p]
        lib.oracle_u0.restype = ctypes.c_double
        _lib = lib
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype)) if a is not None else None


def _problem(pb: dict) -> _OrProblem:
    s = _OrProblem()
    s.dim = int(pb["dim"])
    s.D = float(pb["D"])
    fc = [float(v) for v in pb["f_coef"]]
    if len(fc) > MAX_DEG + 1:
        raise ValueError("f degree above 15")
    s.f_deg = max(len(fc) - 1, 0)
    for i, v in enumerate(fc):
        s.f_coef[i] = v
    kind, params = pb["u0"]
    s.u0_kind = _U0_KINDS[kind]
    for i, v in enumerate(params):
        s.u0_param[i] = float(v)
    s.strategy = {"A": 0, "B": 1}[pb["strategy"]]
    s.lam = float(pb.get("lam", 1.0))
    s.c_pot = float(pb.get("c_pot", 0.0))
    s.q = float(pb.get("q", 0.5))
    s.arity_law = {"uniform": 0, "abs": 1}[pb.get("arity_law", "uniform")]
    if "coef" in pb:
        kind, params, powers = pb["coef"]
        s.coef_kind = _COEF_KINDS[kind]
        for i, v in enumerate(params):
            s.coef_param[i] = float(v)
        s.coef_mask = sum(1 << int(k) for k in powers)
    if "sde" in pb:
        steps, beta, kappa, sd, rr = pb["sde"]
        s.sde_kind = 1
        s.sde_steps = int(steps)
        for blk, vals in enumerate((beta, kappa, sd, rr)):
            for i, v in enumerate(vals):
                s.sde_param[3 * blk + i] = float(v)
    return s


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one 128-bit counter under a 64-bit key (two u32 words)."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.oracle_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return out


def uniform(w: int) -> float:
    return _load().oracle_uniform(ctypes.c_uint32(w))


def u0(pb: dict, x) -> float:
    xs = np.ascontiguousarray(x, dtype=np.float64)
    s = _problem(pb)
    return _load().oracle_u0(ctypes.byref(s), _ptr(xs, ctypes.c_double))


def setup_tables(pb: dict) -> dict:
    """The branching-law tables: terms (arity, coefficient), thresholds, weight factors."""
    lib = _load()
    s = _problem(pb)
    nt = ctypes.c_int32(0)
    ar = np.zeros(16, np.int32)
    co = np.zeros(16, np.float64)
    thr = np.zeros(17, np.uint64)
    lf = ctypes.c_double(0)
    tf = np.zeros(16, np.float64)
    ncat = lib.oracle_setup_tables(ctypes.byref(s), ctypes.byref(nt), _ptr(ar, ctypes.c_int32),
                                   _ptr(co, ctypes.c_double), _ptr(thr, ctypes.c_uint64), ctypes.byref(lf),
                                   _ptr(tf, ctypes.c_double))
    if ncat < 0:
        raise ValueError("invalid problem")
    n = nt.value
    return dict(nterms=n, arity=ar[:n].copy(), coef=co[:n].copy(), thr=thr[:ncat].copy(),
                leaf_factor=lf.value, term_factor=tf[:n].copy())


def trees(pb: dict, x, t: float, point_index: int, first_tree: int, ntrees: int, K: int, seed: int) -> dict:
    """Per-tree records: order (Ne, K+1 if pruned), weight W, nodes visited, topology hash."""
    lib = _load()
    s = _problem(pb)
    xs = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    order = np.zeros(ntrees, np.int32)
    w = np.zeros(ntrees, np.float64)
    nodes = np.zeros(ntrees, np.uint32)
    h = np.zeros(ntrees, np.uint64)
    rc = lib.oracle_trees(ctypes.byref(s), _ptr(xs, ctypes.c_double), float(t), point_index, first_tree, ntrees,
                          K, seed, _ptr(order, ctypes.c_int32), _ptr(w, ctypes.c_double),
                          _ptr(nodes, ctypes.c_uint32), _ptr(h, ctypes.c_uint64))
    if rc != 0:
        raise ValueError("oracle_trees: invalid arguments")
    return dict(order=order, w=w, nodes=nodes, hash=h)


def pade(a, L: int, M: int):
    """[L/M] Pade of sum a_n eps^n at eps = 1. Returns (value, status, (L_used, M_used))."""
    lib = _load()
    av = np.zeros(MAX_K + 1, np.float64)
    a = np.asarray(a, np.float64)
    av[: len(a)] = a
    u = ctypes.c_double(0)
    st = ctypes.c_int32(0)
    lm = np.zeros(2, np.int32)
    if lib.oracle_pade(L, M, _ptr(av, ctypes.c_double), ctypes.byref(u), ctypes.byref(st),
                       _ptr(lm, ctypes.c_int32)) != 0:
        raise ValueError("oracle_pade: invalid L, M")
    return u.value, st.value, (int(lm[0]), int(lm[1]))


def solve(pb: dict, x, t, ntrees, K: int, L: int, M: int, seed: int, point_base: int = 0,
          nthreads: int | None = None) -> dict:
    """Point solve of n points: Pade value u, coefficients a_n, standard errors, status, raw sums."""
    lib = _load()
    s = _problem(pb)
    d = int(pb["dim"])
    xs = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, d)
    n = xs.shape[0]
    ts = np.ascontiguousarray(np.broadcast_to(np.asarray(t, np.float64), (n,)))
    nt = np.ascontiguousarray(np.broadcast_to(np.asarray(ntrees, np.uint64), (n,)))
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    u = np.zeros(n, np.float64)
    coef = np.zeros((n, K + 1), np.float64)
    se = np.zeros((n, K + 1), np.float64)
    st = np.zeros(n, np.int32)
    s1 = np.zeros((n, K + 1), np.float64)
    s2 = np.zeros((n, K + 1), np.float64)
    sa = np.zeros((n, K + 1), np.float64)
    cnt = np.zeros((n, K + 2), np.uint64)
    nodes = np.zeros(n, np.uint64)
    rc = lib.oracle_solve(ctypes.byref(s), n, _ptr(xs, ctypes.c_double), _ptr(ts, ctypes.c_double),
                          _ptr(nt, ctypes.c_uint64), K, L, M, seed, point_base, int(nthreads),
                          _ptr(u, ctypes.c_double), _ptr(coef, ctypes.c_double), _ptr(se, ctypes.c_double),
                          _ptr(st, ctypes.c_int32), _ptr(s1, ctypes.c_double), _ptr(s2, ctypes.c_double),
                          _ptr(sa, ctypes.c_double), _ptr(cnt, ctypes.c_uint64), _ptr(nodes, ctypes.c_uint64))
    if rc != 0:
        raise ValueError("oracle_solve: invalid arguments")
    return dict(u=u, coef=coef, se=se, status=st, s1=s1, s2=s2, sa=sa, cnt=cnt, nodes=nodes,
                nthreads=int(min(nthreads, max(n, 1))))


def pade_error(coef, se, L: int, M: int) -> np.ndarray:
    """Per-result first-order error of the [L/M] Pade value: sqrt(sum_j (du/da_j SE_j)^2), j = 0..L+M,
    the derivatives by central differences of this oracle's Pade with steps
    h_j = 1e-6 max(|a_j|, 1e-12 max_i |a_i|) (the Pade value is Lipschitz in the coefficients,
    Sec. 2.4); +inf where an evaluation is not finite."""
    coef = np.atleast_2d(np.asarray(coef, np.float64))
    se = np.atleast_2d(np.asarray(se, np.float64))
    out = np.zeros(coef.shape[0])
    nn = L + M
    for i in range(coef.shape[0]):
        a = coef[i, : nn + 1].copy()
        amax = np.abs(a).max() if a.size else 0.0
        acc, ok = 0.0, True
        for j in range(nn + 1):
            s = se[i, j]
            if s == 0.0:
                continue
            h = 1e-6 * max(abs(a[j]), 1e-12 * amax, 1e-300)
            ap, am = a.copy(), a.copy()
            ap[j] += h
            am[j] -= h
            up, _, _ = pade(ap, L, M)
            um, _, _ = pade(am, L, M)
            d = (up - um) / (2.0 * h) * s
            if not np.isfinite(d):
                ok = False
            acc += d * d
        out[i] = np.sqrt(acc) if ok else np.inf
    return out
