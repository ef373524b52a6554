"""ctypes binding of libgrt (include/grt.h): argument marshalling only.

Every step of a solve runs in the library's CUDA kernels; this module only
converts Python/numpy/torch arguments to the C ABI and raises on errors.
There is no CPU fallback: if libgrt.so is missing or no GPU is present, the
calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgrt.so")

MAX_DIM = 3
MAX_DEG = 15
MAX_K = 16

OK, EINVAL, ENOMEM, EDEVICE, ENOTSUP, EAGAIN = 0, -1, -2, -3, -5, 1
STRATEGY = {"A": 0, "B": 1}
ARITY_LAW = {"uniform": 0, "abs": 1}
PRECISION = {"fp32": 0, "fp64": 1}
U0_KIND = {"const": 0, "gauss": 1, "cos_prod": 2, "tanh_prod": 3, "logistic": 4, "gauss_axes": 5, "quadratic": 6}
COEF_KIND = {"const": 0, "gauss_over_t": 1, "gauss": 2}
STATUS_PADE_SINGULAR, STATUS_PADE_POLE_NEAR, STATUS_SERIES_PARTIAL, STATUS_HIGH_PRUNE = 1, 2, 4, 8


class GrtError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"libgrt error {code}: {message}")
        self.code = code


class grt_problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32),
        ("D", ctypes.c_double),
        ("f_deg", ctypes.c_int32),
        ("f_coef", ctypes.c_double * (MAX_DEG + 1)),
        ("u0_kind", ctypes.c_int32),
        ("u0_param", ctypes.c_double * 8),
        ("strategy", ctypes.c_int32),
        ("lambda_", ctypes.c_double),
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


class grt_request_info(ctypes.Structure):
    _fields_ = [
        ("latency_s", ctypes.c_double),
        ("shared_launches", ctypes.c_uint64),
        ("shared_steps", ctypes.c_uint64),
        ("cancelled", ctypes.c_int32),
    ]


class grt_pdd_grid(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("sub", ctypes.c_int32 * 3),
        ("cells", ctypes.c_int32 * 3),
        ("nodes", ctypes.c_int32 * 3),
        ("t_nodes", ctypes.c_int32),
        ("T", ctypes.c_double),
        ("nsteps", ctypes.c_int32),
    ]


_P = ctypes.POINTER
_vp = ctypes.c_void_p
_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libgrt.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    i64, u64, i32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int
    # host arrays go in as plain addresses (`_ptr`): an int converts to a void pointer far faster
    # than a typed ctypes pointer is built (a per-call cost of the synchronous solves)
    f64p = u64p = i32p = u32p = _vp
    sig = {
        "grt_create": ([_P(grt_problem), i32, _P(_vp)], i32),
        "grt_destroy": ([_vp], None),
        "grt_last_error": ([_vp], ctypes.c_char_p),
        "grt_solve": ([_vp, i64, f64p, f64p, u64p, i32, i32, i32, u64, u64, f64p, f64p, f64p, i32p], i32),
        "grt_solve_plain": ([_vp, i64, f64p, f64p, u64p, i32, i32, i32, u64, u64, f64p, f64p, f64p, i32p], i32),
        "grt_plan_create": ([_vp, i64, u64p, i32, i32, i32, _P(_vp)], i32),
        "grt_plan_execute": ([_vp, _vp, _vp, u64, u64, _vp, _vp, _vp, _vp, _vp], i32),
        "grt_plan_counters": ([_vp, u64p, u64p, u64p], i32),
        "grt_plan_set_timing": ([_vp, i32], i32),
        "grt_plan_timing": ([_vp, _P(ctypes.c_float), _P(ctypes.c_float)], i32),
        "grt_plan_launches": ([_vp], i32),
        "grt_plan_set_config": ([_vp, i32p], i32),
        "grt_set_solve_config": ([_vp, i32p], i32),
        "grt_plan_get_config": ([_vp, i32p], i32),
        "grt_plan_autotune": ([_vp, _vp, _vp, u64, u64, _vp, _vp, _vp, _vp, _vp, i32p], i32),
        "grt_plan_graph_capture": ([_vp, _vp, _vp, u64, u64, _vp, _vp, _vp, _vp], i32),
        "grt_plan_graph_launch": ([_vp, _vp], i32),
        "grt_plan_destroy": ([_vp], None),
        "grt_pade": ([_vp, i64, i32, i32, i32, f64p, f64p, i32p], i32),
        "grt_pade_error": ([_vp, i64, i32, i32, i32, _vp, _vp, _vp, _vp], i32),
        "grt_plan_kappa": ([_vp, _vp, _vp], i32),
        "grt_trees": ([_vp, f64p, ctypes.c_double, u64, u64, u64, i32, u64, i32p, f64p, u32p, u64p], i32),
        "grt_solve_noalloc": ([_vp, i64, _vp, _vp, u64p, i32, i32, i32, u64, u64, _vp, _vp, _vp, _vp, _vp], i32),
        "grt_server_sizes": ([u64, u64p, u64p], i32),
        "grt_server_create": ([i32, u64, u64, _P(_vp)], i32),
        "grt_server_destroy": ([_vp], None),
        "grt_server_last_error": ([_vp], ctypes.c_char_p),
        "grt_submit": ([_vp, _vp, i64, f64p, f64p, u64p, i32, i32, i32, u64, u64, u64p], i32),
        "grt_poll": ([_vp, u64, i32, f64p, f64p, f64p, i32p, f64p], i32),
        "grt_poll_ex": ([_vp, u64, i32, f64p, f64p, f64p, i32p, u64p, _P(grt_request_info)], i32),
        "grt_cancel": ([_vp, u64], i32),
        "grt_server_stats": ([_vp, u64p, u64p, u64p, u64p, u64p, u64p, u64p, u64p], i32),
        "grt_spline_grid": ([_vp, i32, i32p, f64p, f64p, i32p, f64p, i64, _vp, _vp, _vp], i32),
        "grt_pdd_points": ([_P(grt_pdd_grid), i64, f64p, f64p, _P(ctypes.c_int64)], i32),
        "grt_pdd_solve": ([_vp, _P(grt_pdd_grid), _vp, _vp, _vp], i32),
        "grt_pdd_solve_range": ([_vp, _P(grt_pdd_grid), i64, i64, _vp, _vp, _vp], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def library_path() -> str:
    return LIB_PATH


def _ptr(a, ctype):
    """The address of a host array (ctype names its element type for the reader), None for None."""
    return None if a is None else a.ctypes.data


def _vec(a, dtype, n: int):
    """a as a contiguous length-n array of dtype (a scalar is broadcast), without a copy when it
    already is one."""
    if isinstance(a, np.ndarray) and a.dtype == dtype and a.ndim == 1 and a.shape[0] == n and a.flags.c_contiguous:
        return a
    return np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype), (n,)))


def _devptr(obj):
    """A device address from a torch tensor, an int or None."""
    if obj is None:
        return None
    if hasattr(obj, "data_ptr"):
        return obj.data_ptr()
    return int(obj)


def problem_struct(pb: dict) -> grt_problem:
    """Marshal a problem dict (see workloads.py) into the C struct."""
    s = grt_problem()
    s.dim = int(pb["dim"])
    s.D = float(pb["D"])
    fc = [float(v) for v in pb["f_coef"]]
    if len(fc) > MAX_DEG + 1:
        raise ValueError("f degree above 15")
    s.f_deg = max(len(fc) - 1, 0)
    for i, v in enumerate(fc):
        s.f_coef[i] = v
    kind, params = pb["u0"]
    s.u0_kind = U0_KIND[kind]
    for i, v in enumerate(params):
        s.u0_param[i] = float(v)
    s.strategy = STRATEGY[pb["strategy"]]
    s.lambda_ = float(pb.get("lam", 1.0))
    s.c_pot = float(pb.get("c_pot", 0.0))
    s.q = float(pb.get("q", 0.5))
    s.arity_law = ARITY_LAW[pb.get("arity_law", "uniform")]
    s.precision = PRECISION[pb.get("precision", "fp32")]
    if "coef" in pb:
        kind, params, powers = pb["coef"]
        s.coef_kind = COEF_KIND[kind]
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


class Context:
    """A libgrt context (grt_ctx) for one problem on one device."""

    def __init__(self, handle, problem: dict):
        self._h = handle
        self.problem = dict(problem)
        self.dim = int(problem["dim"])

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("context is closed")
        return self._h

    def close(self):
        if self._h:
            _load().grt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Plan:
    """A libgrt plan (grt_plan): fixed points budgets and K, L, M; device-resident execution."""

    def __init__(self, handle, ctx: Context, n: int, K: int, L: int, M: int, ntrees):
        self._h = handle
        self.ctx = ctx
        self.n, self.K, self.L, self.M = n, K, L, M
        self.ntrees = np.array(ntrees, dtype=np.uint64)

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("plan is closed")
        return self._h

    def close(self):
        if self._h:
            _load().grt_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check(rc: int, ctx_handle=None):
    if rc != OK:
        msg = _load().grt_last_error(ctx_handle)
        raise GrtError(rc, msg.decode() if msg else "")


def grt_server_last_error(server: Server) -> str:
    msg = _load().grt_server_last_error(server.handle)
    return msg.decode() if msg else ""


def grt_last_error(ctx: Context | None) -> str:
    msg = _load().grt_last_error(ctx.handle if ctx is not None else None)
    return msg.decode() if msg else ""


def grt_create(problem: dict, device: int = 0) -> Context:
    lib = _load()
    s = problem_struct(problem)
    h = _vp()
    _check(lib.grt_create(ctypes.byref(s), int(device), ctypes.byref(h)), None)
    return Context(h.value, problem)


def grt_destroy(ctx: Context) -> None:
    ctx.close()


def grt_solve(ctx: Context, x, t, ntrees, K: int, L: int, M: int, seed: int, point_base: int = 0,
              want_coef: bool = True, want_se: bool = True, want_status: bool = True, out: dict | None = None) -> dict:
    """Synchronous point solve with host arrays. Returns u [n], coef/se [n, K+1], status [n]."""
    lib = _load()
    d = ctx.dim
    xs = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, d)
    n = xs.shape[0]
    ts = _vec(t, np.float64, n)
    nt = _vec(ntrees, np.uint64, n)
    if out is None:
        out = {}
    u = out.get("u")
    if u is None:
        u = np.empty(n, np.float64)
    coef = out.get("coef") if want_coef else None
    if want_coef and coef is None:
        coef = np.empty((n, K + 1), np.float64)
    se = out.get("se") if want_se else None
    if want_se and se is None:
        se = np.empty((n, K + 1), np.float64)
    st = out.get("status") if want_status else None
    if want_status and st is None:
        st = np.empty(n, np.int32)
    rc = lib.grt_solve(ctx.handle, n, _ptr(xs, ctypes.c_double), _ptr(ts, ctypes.c_double),
                       _ptr(nt, ctypes.c_uint64), K, L, M, int(seed), int(point_base), _ptr(u, ctypes.c_double),
                       _ptr(coef, ctypes.c_double), _ptr(se, ctypes.c_double), _ptr(st, ctypes.c_int32))
    _check(rc, ctx.handle)
    return dict(u=u, coef=coef, se=se, status=st)


def grt_solve_plain(ctx: Context, x, t, ntrees, K: int, L: int, M: int, seed: int, point_base: int = 0,
                    want_coef: bool = True, want_se: bool = True) -> dict:
    """The plain FP64 solve, one kernel launch per point (host arrays, synchronous)."""
    lib = _load()
    d = ctx.dim
    xs = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, d)
    n = xs.shape[0]
    ts = _vec(t, np.float64, n)
    nt = _vec(ntrees, np.uint64, n)
    u = np.empty(n, np.float64)
    coef = np.empty((n, K + 1), np.float64) if want_coef else None
    se = np.empty((n, K + 1), np.float64) if want_se else None
    st = np.empty(n, np.int32)
    rc = lib.grt_solve_plain(ctx.handle, n, _ptr(xs, ctypes.c_double), _ptr(ts, ctypes.c_double),
                             _ptr(nt, ctypes.c_uint64), K, L, M, int(seed), int(point_base), _ptr(u, ctypes.c_double),
                             _ptr(coef, ctypes.c_double), _ptr(se, ctypes.c_double), _ptr(st, ctypes.c_int32))
    _check(rc, ctx.handle)
    return dict(u=u, coef=coef, se=se, status=st)


def grt_plan_create(ctx: Context, ntrees, K: int, L: int, M: int) -> Plan:
    lib = _load()
    nt = np.ascontiguousarray(np.asarray(ntrees, np.uint64).reshape(-1))
    h = _vp()
    _check(lib.grt_plan_create(ctx.handle, nt.size, _ptr(nt, ctypes.c_uint64), K, L, M, ctypes.byref(h)), ctx.handle)
    return Plan(h.value, ctx, nt.size, K, L, M, nt)


def grt_plan_execute(plan: Plan, x, t, seed: int, point_base: int, u, coef=None, se=None, status=None,
                     stream=None) -> None:
    """Enqueue a solve on `stream` (torch.cuda.Stream, a raw handle, or None).

    x, t, u, coef, se, status are device buffers: torch CUDA tensors (float64 /
    int32, contiguous) or raw device addresses.
    """
    lib = _load()
    sh = None
    if stream is not None:
        sh = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    rc = lib.grt_plan_execute(plan.handle, _devptr(x), _devptr(t), int(seed), int(point_base), _devptr(u),
                              _devptr(coef), _devptr(se), _devptr(status), sh)
    _check(rc, plan.ctx.handle)


def grt_plan_counters(plan: Plan):
    """(nodes visited, splitting events, trees pruned) of the plan's last execution."""
    lib = _load()
    a, b, c = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(lib.grt_plan_counters(plan.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), plan.ctx.handle)
    return int(a.value), int(b.value), int(c.value)


def grt_plan_set_timing(plan: Plan, on: bool) -> None:
    _check(_load().grt_plan_set_timing(plan.handle, 1 if on else 0), plan.ctx.handle)


def grt_plan_timing(plan: Plan):
    """(walk kernel ms, finalize kernel ms) of the last execution, from CUDA events on its stream."""
    a, b = ctypes.c_float(0), ctypes.c_float(0)
    _check(_load().grt_plan_timing(plan.handle, ctypes.byref(a), ctypes.byref(b)), plan.ctx.handle)
    return float(a.value), float(b.value)


def grt_plan_set_config(plan: Plan, cfg) -> None:
    """Walk launch shape [warps, smem stack levels, blocks per SM, trees per queue chunk]."""
    c = np.ascontiguousarray(cfg, dtype=np.int32)
    _check(_load().grt_plan_set_config(plan.handle, _ptr(c, ctypes.c_int32)), plan.ctx.handle)


def grt_set_solve_config(ctx: Context, cfg) -> None:
    """Launch shape [warps, smem_levels, blocks_per_sm, tile] of the context's grt_solve walks."""
    c = np.ascontiguousarray(np.asarray(cfg, np.int32).reshape(4))
    _check(_load().grt_set_solve_config(ctx.handle, _ptr(c, ctypes.c_int32)), ctx.handle)


def grt_plan_get_config(plan: Plan) -> list:
    c = np.zeros(4, np.int32)
    _check(_load().grt_plan_get_config(plan.handle, _ptr(c, ctypes.c_int32)), plan.ctx.handle)
    return [int(v) for v in c]


def grt_plan_autotune(plan: Plan, x, t, seed: int, point_base: int, u, coef=None, se=None, status=None,
                      stream=None) -> list:
    """Time the candidate launch shapes on this plan's workload and keep the fastest; returns it."""
    sh = None
    if stream is not None:
        sh = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    c = np.zeros(4, np.int32)
    _check(_load().grt_plan_autotune(plan.handle, _devptr(x), _devptr(t), int(seed), int(point_base), _devptr(u),
                                     _devptr(coef), _devptr(se), _devptr(status), sh, _ptr(c, ctypes.c_int32)),
           plan.ctx.handle)
    return [int(v) for v in c]


def grt_plan_graph_capture(plan: Plan, x, t, seed: int, point_base: int, u, coef=None, se=None, status=None) -> None:
    _check(_load().grt_plan_graph_capture(plan.handle, _devptr(x), _devptr(t), int(seed), int(point_base), _devptr(u),
                                          _devptr(coef), _devptr(se), _devptr(status)), plan.ctx.handle)


def grt_plan_graph_launch(plan: Plan, stream=None) -> None:
    sh = None
    if stream is not None:
        sh = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    _check(_load().grt_plan_graph_launch(plan.handle, sh), plan.ctx.handle)


def grt_plan_launches(plan: Plan) -> int:
    return int(_load().grt_plan_launches(plan.handle))


def grt_plan_destroy(plan: Plan) -> None:
    plan.close()


def grt_pade(ctx: Context, coef, L: int, M: int):
    """FP64 [L/M] Pade at eps = 1 of each row of coef [n, K+1], on the GPU. Returns (u, status)."""
    lib = _load()
    c = np.ascontiguousarray(coef, dtype=np.float64)
    if c.ndim == 1:
        c = c.reshape(1, -1)
    n, K1 = c.shape
    u = np.empty(n, np.float64)
    st = np.empty(n, np.int32)
    _check(lib.grt_pade(ctx.handle, n, K1 - 1, L, M, _ptr(c, ctypes.c_double), _ptr(u, ctypes.c_double),
                        _ptr(st, ctypes.c_int32)), ctx.handle)
    return u, st


def grt_plan_kappa(plan: Plan, kappa, stream=None) -> None:
    """Cancellation factors SA_n / |S1_n| of the plan's last execution into the device buffer kappa [n][K+1]."""
    lib = _load()
    sh = None
    if stream is not None:
        sh = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    _check(lib.grt_plan_kappa(plan.handle, _devptr(kappa), sh), plan.ctx.handle)


def grt_pade_error(ctx: Context, coef, se, L: int, M: int, err, stream=None) -> None:
    """Per-result first-order error of the Pade value from the coefficient standard errors.
    coef, se: device [n][K+1] float64; err: device [n] float64 (torch tensors or raw addresses)."""
    lib = _load()
    n = int(coef.shape[0]) if hasattr(coef, "shape") else None
    K = int(coef.shape[1]) - 1 if hasattr(coef, "shape") else None
    if n is None:
        raise ValueError("coef must carry its shape (a torch tensor)")
    sh = None
    if stream is not None:
        sh = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    _check(lib.grt_pade_error(ctx.handle, n, K, L, M, _devptr(coef), _devptr(se), _devptr(err), sh), ctx.handle)


def grt_trees(ctx: Context, x, t: float, point_index: int, first_tree: int, ntrees: int, K: int, seed: int) -> dict:
    """Per-tree records (order, weight, nodes, topology hash) of one point's trees, from the GPU."""
    lib = _load()
    xs = np.ascontiguousarray(np.asarray(x, np.float64).reshape(-1))
    order = np.empty(ntrees, np.int32)
    w = np.empty(ntrees, np.float64)
    nodes = np.empty(ntrees, np.uint32)
    h = np.empty(ntrees, np.uint64)
    _check(lib.grt_trees(ctx.handle, _ptr(xs, ctypes.c_double), float(t), int(point_index), int(first_tree),
                         int(ntrees), K, int(seed), _ptr(order, ctypes.c_int32), _ptr(w, ctypes.c_double),
                         _ptr(nodes, ctypes.c_uint32), _ptr(h, ctypes.c_uint64)), ctx.handle)
    return dict(order=order, w=w, nodes=nodes, hash=h)


NOALLOC_MAX_POINTS = 4096
NOALLOC_MAX_TREES = 524288


def grt_solve_noalloc(ctx: Context, x, t, ntrees, K: int, L: int, M: int, seed: int, point_base: int, u, coef=None,
                      se=None, status=None, stream=None) -> None:
    """Point solve that allocates no device memory (for callers that cannot allocate when they solve).

    x, t, u, coef, se, status are the caller's device buffers (torch CUDA tensors or raw
    addresses); ntrees is a host array.  The solve's work area is a fixed ~7 MB array the
    library keeps on the device; calls whose GPU work overlaps in time race on it.
    """
    lib = _load()
    nt = np.ascontiguousarray(np.asarray(ntrees, np.uint64).reshape(-1))
    sh = None
    if stream is not None:
        sh = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    rc = lib.grt_solve_noalloc(ctx.handle, nt.size, _devptr(x), _devptr(t), _ptr(nt, ctypes.c_uint64), K, L, M,
                               int(seed), int(point_base), _devptr(u), _devptr(coef), _devptr(se), _devptr(status), sh)
    _check(rc, ctx.handle)


class Server:
    """A libgrt serving instance (grt_server): scheduler thread + device-memory budget."""

    def __init__(self, handle):
        self._h = handle
        self.requests = {}  # request id -> (n, K)

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("server is closed")
        return self._h

    def close(self):
        if self._h:
            _load().grt_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check_server(rc: int, server: "Server"):
    if rc != OK:
        msg = _load().grt_server_last_error(server._h)
        raise GrtError(rc, msg.decode() if msg else "")


def grt_server_sizes(step_trees: int = 0) -> dict:
    """Step-buffer bytes of a server with steps of step_trees trees and resident bytes per admitted point."""
    sb, pb = ctypes.c_uint64(0), ctypes.c_uint64(0)
    rc = _load().grt_server_sizes(int(step_trees), ctypes.byref(sb), ctypes.byref(pb))
    if rc != OK:
        raise GrtError(rc, "grt_server_sizes: step_trees must be in [8192, 2^31]")
    return {"step_bytes": int(sb.value), "point_bytes": int(pb.value)}


def grt_server_create(device: int = 0, mem_budget_bytes: int = 2 << 30, step_trees: int = 0) -> Server:
    h = _vp()
    rc = _load().grt_server_create(int(device), int(mem_budget_bytes), int(step_trees), ctypes.byref(h))
    if rc != OK:
        raise GrtError(rc, "grt_server_create failed")
    return Server(h.value)


def grt_server_destroy(server: Server) -> None:
    server.close()


def grt_submit(server: Server, ctx: Context, x, t, ntrees, K: int, L: int, M: int, seed: int,
               point_base: int = 0) -> int:
    """Queue a point-solve request (host arrays are copied); returns its id at once."""
    lib = _load()
    d = ctx.dim
    xs = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, d)
    n = xs.shape[0]
    ts = _vec(t, np.float64, n)
    nt = _vec(ntrees, np.uint64, n)
    rid = ctypes.c_uint64(0)
    _check_server(lib.grt_submit(server.handle, ctx.handle, n, _ptr(xs, ctypes.c_double), _ptr(ts, ctypes.c_double),
                                 _ptr(nt, ctypes.c_uint64), K, L, M, int(seed), int(point_base),
                                 ctypes.byref(rid)), server)
    server.requests[rid.value] = (n, K)
    return rid.value


def grt_poll(server: Server, request_id: int, timeout_ms: int = -1):
    """Results of a request (dict with u, coef, se, status, latency_s), or None if not finished."""
    lib = _load()
    n, K = server.requests[request_id]
    u = np.empty(n, np.float64)
    coef = np.empty((n, K + 1), np.float64)
    se = np.empty((n, K + 1), np.float64)
    st = np.empty(n, np.int32)
    lat = ctypes.c_double(0)
    rc = lib.grt_poll(server.handle, int(request_id), int(timeout_ms), _ptr(u, ctypes.c_double),
                      _ptr(coef, ctypes.c_double), _ptr(se, ctypes.c_double), _ptr(st, ctypes.c_int32),
                      ctypes.byref(lat))
    if rc == EAGAIN:
        return None
    del server.requests[request_id]
    _check_server(rc, server)
    return dict(u=u, coef=coef, se=se, status=st, latency_s=lat.value)


def grt_poll_ex(server: Server, request_id: int, timeout_ms: int = -1):
    """grt_poll plus the trees each point's estimate used (ntrees_done) and the request's sharing figures."""
    lib = _load()
    n, K = server.requests[request_id]
    u = np.empty(n, np.float64)
    coef = np.empty((n, K + 1), np.float64)
    se = np.empty((n, K + 1), np.float64)
    st = np.empty(n, np.int32)
    nd = np.empty(n, np.uint64)
    info = grt_request_info()
    rc = lib.grt_poll_ex(server.handle, int(request_id), int(timeout_ms), _ptr(u, ctypes.c_double),
                         _ptr(coef, ctypes.c_double), _ptr(se, ctypes.c_double), _ptr(st, ctypes.c_int32),
                         _ptr(nd, ctypes.c_uint64), ctypes.byref(info))
    if rc == EAGAIN:
        return None
    del server.requests[request_id]
    _check_server(rc, server)
    return dict(u=u, coef=coef, se=se, status=st, ntrees_done=nd, latency_s=info.latency_s,
                shared_launches=int(info.shared_launches), shared_steps=int(info.shared_steps),
                cancelled=bool(info.cancelled))


def grt_cancel(server: Server, request_id: int) -> None:
    """Stop a request early: unfinished points end with the trees binned so far (SERIES_PARTIAL)."""
    _check_server(_load().grt_cancel(server.handle, int(request_id)), server)


def grt_server_stats(server: Server) -> dict:
    vals = [ctypes.c_uint64(0) for _ in range(8)]
    _check_server(_load().grt_server_stats(server.handle, *[ctypes.byref(v) for v in vals]), server)
    keys = ["steps", "trees", "launches", "resident_bytes", "pending", "active", "shared_launches", "cancelled"]
    return {k: int(v.value) for k, v in zip(keys, vals)}


# ---------------------------------------------------------------------------
# probabilistic domain decomposition (Sec. 3)
# ---------------------------------------------------------------------------
def pdd_grid_struct(g: dict) -> grt_pdd_grid:
    """Marshal a PDD grid dict (dim, lo, hi, sub, cells, nodes, t_nodes, T, nsteps) into the C struct."""
    s = grt_pdd_grid()
    d = int(g["dim"])
    s.dim = d
    for a in range(d):
        s.lo[a] = float(g["lo"][a])
        s.hi[a] = float(g["hi"][a])
        s.sub[a] = int(g["sub"][a])
        s.cells[a] = int(g["cells"][a])
        s.nodes[a] = int(g["nodes"][a]) if "nodes" in g else 0
    s.t_nodes = int(g["t_nodes"])
    s.T = float(g["T"])
    s.nsteps = int(g["nsteps"])
    return s


def grt_pdd_points(grid: dict):
    """The probabilistic nodal points (x [n][dim], t [n]) of a PDD grid, in the order grt_pdd_solve reads."""
    lib = _load()
    gs = pdd_grid_struct(grid)
    n = ctypes.c_int64(0)
    _check(lib.grt_pdd_points(ctypes.byref(gs), 0, None, None, ctypes.byref(n)))
    x = np.zeros((n.value, gs.dim), np.float64)
    t = np.zeros(n.value, np.float64)
    _check(lib.grt_pdd_points(ctypes.byref(gs), n.value, _ptr(x, ctypes.c_double), _ptr(t, ctypes.c_double),
                              ctypes.byref(n)))
    return x, t


def grt_pdd_solve(ctx: Context, grid: dict, u_nodes, u_out, stream=None, subdomains=None) -> None:
    """Enqueue the PDD solution at T on the global grid into the device buffer u_out (N[0] x ... row-major).
    u_nodes: device values at grt_pdd_points.  subdomains=(begin, end) solves only that range of the
    row-major subdomain numbering (grt_pdd_solve_range)."""
    lib = _load()
    gs = pdd_grid_struct(grid)
    sh = None
    if stream is not None:
        sh = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    if subdomains is None:
        rc = lib.grt_pdd_solve(ctx.handle, ctypes.byref(gs), _devptr(u_nodes), _devptr(u_out), sh)
    else:
        rc = lib.grt_pdd_solve_range(ctx.handle, ctypes.byref(gs), int(subdomains[0]), int(subdomains[1]),
                                     _devptr(u_nodes), _devptr(u_out), sh)
    _check(rc, ctx.handle)


def grt_pdd_solve_range(ctx: Context, grid: dict, sub_begin: int, sub_end: int, u_nodes, u_out,
                        stream=None) -> None:
    """grt_pdd_solve for the row-major subdomains [sub_begin, sub_end) only (all plane nodes written)."""
    grt_pdd_solve(ctx, grid, u_nodes, u_out, stream=stream, subdomains=(sub_begin, sub_end))


def grt_spline_grid(ctx: Context, n_nodes, lo, hi, targets, values, out, batch: int = 1, stream=None) -> None:
    """Tensor-product not-a-knot spline on a uniform grid: values (device, [batch][n_nodes...]) at the grid
    of target coordinates (a list of 1-D host arrays, one per axis) into out (device, [batch][n_targets...])."""
    lib = _load()
    nd = len(n_nodes)
    nn = np.ascontiguousarray(n_nodes, np.int32)
    lo_ = np.ascontiguousarray(lo, np.float64)
    hi_ = np.ascontiguousarray(hi, np.float64)
    nt = np.ascontiguousarray([len(v) for v in targets], np.int32)
    tg = np.ascontiguousarray(np.concatenate([np.asarray(v, np.float64) for v in targets]))
    sh = None
    if stream is not None:
        sh = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    rc = lib.grt_spline_grid(ctx.handle, nd, _ptr(nn, ctypes.c_int32), _ptr(lo_, ctypes.c_double),
                             _ptr(hi_, ctypes.c_double), _ptr(nt, ctypes.c_int32), _ptr(tg, ctypes.c_double),
                             int(batch), _devptr(values), _devptr(out), sh)
    _check(rc, ctx.handle)


EXPORTED = ["grt_create", "grt_destroy", "grt_last_error", "grt_solve", "grt_solve_plain", "grt_plan_create",
            "grt_plan_execute",
            "grt_plan_counters", "grt_plan_set_timing", "grt_plan_timing", "grt_plan_launches", "grt_plan_destroy",
            "grt_plan_set_config", "grt_plan_get_config", "grt_set_solve_config", "grt_plan_autotune", "grt_plan_graph_capture",
            "grt_plan_graph_launch",
            "grt_pade", "grt_pade_error", "grt_plan_kappa", "grt_trees", "grt_solve_noalloc", "grt_server_sizes", "grt_server_create",
            "grt_server_destroy",
            "grt_server_last_error", "grt_submit", "grt_poll", "grt_poll_ex", "grt_cancel", "grt_server_stats",
            "grt_spline_grid",
            "grt_pdd_points", "grt_pdd_solve", "grt_pdd_solve_range"]
