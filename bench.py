"""Benchmark of the generalized-random-tree point solve on GB300.

Workload (N=1): sin_2d -- u_t = 0.5 Lap u + sin(u) in 2-D (sin as its degree-9
Taylor polynomial, offspring k drawn with p_k ~ |b_k|, Strategy B), u0 =
1.2 exp(-|x|^2/2), a 16x16 grid on [-3,3]^2 at t in {0.25, 1.0} (512 point
solves), 1e5 trees per point, series order K = 10, FP64 Pade [5/5], FP32
walk.  One step = one full point solve of that batch (walk + finalize) with
the inputs resident in device memory; the L2 is flushed between steps.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl grt|reference]
Under torchrun (N > 1) every rank solves its own batch of 512 point solves
(point streams keyed by rank * 512 + i): weak scaling, no collective on the
data path; the timed region is bracketed by barriers and the max over ranks
is taken.  Rank 0 prints one compact JSON line (the last line of stdout); the
per-result error list, the other workloads' and the serving trace's full
figures go to a side JSON file (--details, default bench_details.json).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "trees/s, points/s at 1e-5 rel vs oracle; p50/p99 served latency vs plain path"
WORKLOAD = "sin_2d"
L2_FLUSH_BYTES = 256 << 20
ISSUE_PER_SM_PER_CLK = 4 * 32   # 4 schedulers x 1 warp-instruction x 32 threads
FP32_WEIGHT_RTOL = 3e-5        # per-tree FP32 weight vs its FP64 value (the per-tree parity bound)


def _walk_profile():
    """(DRAM bytes per full-size walk launch, ncu figures of the walk kernel) from the committed
    ncu summary, or (None, None) when the walk kernel's sources changed since that capture."""
    import hashlib
    import re
    try:
        text = open(os.path.join(ROOT, "profiles", "walk_kernel_sin2d.md")).read()
        want = re.search(r"source_sha256_16: ([0-9a-f]+)", text).group(1)
        traffic = int(re.search(r"traffic_bytes_per_launch: (\d+)", text).group(1))

        def num(key):
            m = re.search(key + r": ([0-9.]+)", text)
            return float(m.group(1)) if m else None

        issue, alu, fma, lanes = (num("issue_active_pct"), num("alu_pipe_pct"), num("fma_pipe_pct"),
                                  num("active_lanes_per_inst"))
        figs = {"issue_active": issue / 100.0 if issue is not None else None,
                "alu_pipe": alu / 100.0 if alu is not None else None,
                "fma_pipe": fma / 100.0 if fma is not None else None,
                "lane_efficiency": lanes / 32.0 if lanes is not None else None}
        h = hashlib.sha256()
        for f in ("grt_device.cuh", "grt_walk.cuh", "grt_walk_u0.cu"):
            with open(os.path.join(ROOT, "paper_2402_06491_gb300", "csrc", f), "rb") as fh:
                h.update(fh.read())
        return (traffic, figs) if h.hexdigest()[:16] == want else (None, None)
    except Exception:
        return None, None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# ---------------------------------------------------------------------------
# algorithmic instruction model of the node body (FP32 walk), per unit of work
# ---------------------------------------------------------------------------
def instruction_model(problem: dict, K: int) -> dict:
    """Minimal thread-instructions the method needs per node / leaf / split / tree.

    Node (every node): Philox4x32-10 = 10 rounds x (2 IMAD.WIDE + 2 LOP3) = 40
    per call (1 call for d <= 2, 2 for d = 3); 2 per uniform word (shift-or,
    add); Box-Muller pair = 8 (lg2, mul, rsqrt, mul, sin, cos, 2 mul); decision
    1; segment = 4 + d (select, 2 mul, sqrt = rsqrt + mul, d FFMA); weight
    multiply 1; node count 1.
    Leaf: g(y) (gauss 3 + 2d, cos/tanh product 3d, logistic 5, const 0), leaf
    factor 1, continue with the next sibling = d + 5 (frame loads, test,
    update).
    Split: term search 2 per finite threshold past the leaf's, tau(1-S) 2,
    factor 3 (two table loads, mul), Ne check 2, child label 3, push d + 4.
    Tree: start 8, record 2, refill 6.
    """
    d = int(problem["dim"])
    kind = problem["u0"][0]
    nterms = sum(1 for b in problem["f_coef"] if b != 0.0)
    calls = 2 if d == 3 else 1
    words = 3 + (2 if d == 3 else 0)
    pairs = 2 if d == 3 else 1
    node = 40 * calls + 2 * words + 8 * pairs + 1 + (4 + d) + 1 + 1
    g = {"gauss": 3 + 2 * d, "cos_prod": 3 * d, "tanh_prod": 3 * d, "logistic": 5, "const": 0}[kind]
    leaf = g + 1 + (d + 5)
    split = 2 * max(nterms - 1, 0) + 2 + 3 + 2 + 3 + (d + 4)
    tree = 16
    return dict(node=node, leaf=leaf, split=split, tree=tree)


def algorithmic_instructions(model: dict, nodes: int, splits: int, trees: int) -> float:
    leaves = nodes - splits
    return float(model["node"] * nodes + model["leaf"] * leaves + model["split"] * splits + model["tree"] * trees)


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = (bus_id or "").lower()  # e.g. "00000009:01:00.0"; empty = only GPU of the box
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            bus = parts[1].lower()
            if self.bus_id and bus[-7:] != self.bus_id[-7:]:
                continue
            try:
                self.samples.append(dict(t=time.time(), sm=float(parts[2]), sm_max=float(parts[3]),
                                         hw=parts[6], hw_thermal=parts[7], sw_thermal=parts[8], sw_power=parts[9]))
            except ValueError:
                continue

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self, t0: float, t1: float) -> dict:
        inside = [s for s in self.samples if t0 <= s["t"] <= t1]
        window = "timed region"
        if len(inside) < 3:  # short timed region: take the samples nearest to it
            inside = sorted(self.samples, key=lambda s: min(abs(s["t"] - t0), abs(s["t"] - t1)))[:5]
            window = "nearest samples to a short timed region"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}
        reasons = set()
        for s in inside:
            for key, name in (("hw", "hw_slowdown"), ("hw_thermal", "hw_thermal_slowdown"),
                              ("sw_thermal", "sw_thermal_slowdown"), ("sw_power", "sw_power_cap")):
                if s[key].lower() in ("active", "1", "yes"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(s["sm"] for s in inside), "sm_max_mhz": max(s["sm_max"] for s in inside),
                "reasons": sorted(reasons), "samples": len(inside), "window": window}


# ---------------------------------------------------------------------------
# CPU oracle arms
# ---------------------------------------------------------------------------
def oracle_sample(wl: dict, target_s: float, nthreads: int):
    """Time the oracle on a bounded leading slice of the workload's points (all their trees)."""
    import oracle

    oracle.build()
    n = wl["x"].shape[0]
    probe = min(4, n)
    t0 = time.perf_counter()
    oracle.solve(wl["problem"], wl["x"][:probe], wl["t"][:probe], wl["ntrees"][:probe], wl["K"], wl["L"], wl["M"],
                 wl["seed"], nthreads=min(nthreads, probe))
    per_point_thread = (time.perf_counter() - t0) * min(nthreads, probe) / probe
    npts = int(max(1, min(n, target_s * nthreads / max(per_point_thread, 1e-6))))
    npts = max(min(npts, n), min(nthreads, n))
    return npts


def run_oracle(wl: dict, npts: int, nthreads: int):
    import oracle

    t0 = time.perf_counter()
    r = oracle.solve(wl["problem"], wl["x"][:npts], wl["t"][:npts], wl["ntrees"][:npts], wl["K"], wl["L"], wl["M"],
                     wl["seed"], nthreads=nthreads)
    return time.perf_counter() - t0, r


def cpu_baseline(wl: dict, target_s: float, gpu=None) -> dict:
    """The oracle, as it stands, on all host cores over the leading points of the workload.

    Whole passes over the chosen points are repeated until about target_s of wall time.  When the
    GPU's results for the same points (same streams) are given as gpu = (u, coef), the error of
    each sampled result against the FP64 oracle is stated beside the timing.
    """
    nthreads = os.cpu_count() or 1
    npts = oracle_sample(wl, target_s, nthreads)
    trees = float(np.sum(wl["ntrees"][:npts]))
    total, reps, r = 0.0, 0, None
    while reps == 0 or (total < 0.5 * target_s and reps < 20):
        dt, r = run_oracle(wl, npts, nthreads)
        total += dt
        reps += 1
    n = wl["x"].shape[0]
    out = {"value": trees * reps / total, "unit": "trees/s", "cores": nthreads, "kind": "oracle",
           "sample": f"{npts} of {n} {WORKLOAD} points, all trees, x {reps}, {total:.1f} s"}
    if gpu is not None:
        gu, gc = gpu
        du = np.abs(gu[:npts] - r["u"])
        scale = np.maximum(np.abs(r["u"]), np.abs(r["coef"]).sum(axis=1))  # the 1e-5 bar's scale
        rel = du / np.maximum(scale, 1e-300)
        out["error_vs_oracle"] = {
            "points": npts, "bar": "|u_gpu - u_oracle| <= 1e-5 max(|u|, sum_n |a_n|)",
            "max_rel": float(rel.max()), "median_rel": float(np.median(rel)),
            "within_bar": int((rel <= 1e-5).sum()),
            "per_result_rel": [float(v) for v in rel],
            "max_abs_coef": float(np.abs(gc[:npts] - r["coef"]).max()),
        }
    return out


def reference_arm(args) -> int:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = workloads.WORKLOADS[WORKLOAD]()
    nthreads = os.cpu_count() or 1
    # a bounded sample per step, sized so that the whole run (warm-up + timed steps) takes about two
    # minutes of host time whatever --steps is (at least one point per host thread per step)
    budget_s = float(os.environ.get("GRT_REFERENCE_BUDGET_S", "120"))
    per_step_s = float(os.environ.get("GRT_REFERENCE_STEP_S", str(min(2.0, budget_s / max(args.steps + args.warmup, 1)))))
    npts = oracle_sample(wl, per_step_s, nthreads)
    trees = float(np.sum(wl["ntrees"][:npts]))
    for _ in range(args.warmup):
        run_oracle(wl, npts, nthreads)
    times = []
    for _ in range(args.steps):
        dt, _ = run_oracle(wl, npts, nthreads)
        times.append(dt)
    total = sum(times)
    value = trees * args.steps / total
    sample = f"first {npts} of {wl['x'].shape[0]} point solves of {WORKLOAD}, all 1e5 trees each, per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "trees/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "points_per_s": npts * args.steps / total,
        "config": {"workload": f"{WORKLOAD} (FP64 CPU oracle: the plain reference of the method; no upstream code exists)",
                   "points_per_step": npts, "trees_per_point": int(wl["ntrees"][0]), "K": wl["K"], "L": wl["L"],
                   "M": wl["M"], "parallelism": f"{nthreads} host threads"},
        "cpu_baseline": {"value": value, "unit": "trees/s", "cores": nthreads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "trees/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# the other workloads: uneven budgets (4096 interface points) and the 3-D PDD planes
# ---------------------------------------------------------------------------
def pade_health(grt, ctx, plan, x, t, seed: int, K: int, L: int, M: int, tmask=None) -> dict:
    """How many point values the Pade has spoiled: points flagged PADE_POLE_NEAR (|Q(1)| < 1e-8) or
    PADE_SINGULAR, and points whose first-order statistical error (grt_pade_error from the standard
    errors) exceeds 1e-2 -- over all points, or over those of `tmask` (a boolean mask)."""
    import torch

    dev = x.device
    n = x.shape[0]
    u = torch.empty(n, dtype=torch.float64, device=dev)
    coef = torch.empty((n, K + 1), dtype=torch.float64, device=dev)
    se = torch.empty((n, K + 1), dtype=torch.float64, device=dev)
    st = torch.empty(n, dtype=torch.int32, device=dev)
    err = torch.empty(n, dtype=torch.float64, device=dev)
    grt.grt_plan_execute(plan, x, t, seed, 0, u, coef, se, st)
    grt.grt_pade_error(ctx, coef, se, L, M, err)
    torch.cuda.synchronize(dev)
    sth, eh = st.cpu().numpy(), err.cpu().numpy()
    m = np.ones(n, bool) if tmask is None else np.asarray(tmask, bool)
    return {"points": int(m.sum()), "pole_near": int(((sth & 2) != 0)[m].sum()),
            "singular": int(((sth & 1) != 0)[m].sum()), "err_over_1e-2": int((~(eh <= 1e-2))[m].sum()),
            "err_median": float(np.median(eh[m])) if m.any() else None}

def workload_bench(grt, dev_index: int, name: str, steps: int) -> dict:
    import torch

    dev = torch.device("cuda", dev_index)
    wl = workloads.WORKLOADS[name]()
    n, K = wl["x"].shape[0], wl["K"]
    ctx = grt.grt_create(wl["problem"], dev_index)
    plan = grt.grt_plan_create(ctx, wl["ntrees"], K, wl["L"], wl["M"])
    x = torch.from_numpy(wl["x"]).to(dev)
    t = torch.from_numpy(wl["t"]).to(dev)
    u = torch.empty(n, dtype=torch.float64, device=dev)
    coef = torch.empty((n, K + 1), dtype=torch.float64, device=dev)
    st = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    s = torch.cuda.Stream(device=dev)
    cfg = grt.grt_plan_autotune(plan, x, t, wl["seed"], 0, u, coef, None, st, stream=s)
    grt.grt_plan_set_timing(plan, True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    wms, fms = [], []
    for a, b in ev:
        with torch.cuda.stream(s):
            flush.zero_()
        a.record(s)
        grt.grt_plan_execute(plan, x, t, wl["seed"], 0, u, coef, None, st, stream=s)
        b.record(s)
        wm, fm = grt.grt_plan_timing(plan)
        wms.append(wm)
        fms.append(fm)
    torch.cuda.synchronize(dev)
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    nodes, splits, pruned = grt.grt_plan_counters(plan)
    trees = float(np.sum(wl["ntrees"]))
    finite = bool(torch.isfinite(u).all().item())
    health = pade_health(grt, ctx, plan, x, t, wl["seed"], K, wl["L"], wl["M"])
    plan.close()
    ctx.close()
    return {"trees_per_s": trees / (ms / 1e3), "points_per_s": n / (ms / 1e3), "ms_per_step": ms, "steps": steps,
            "pade_health": health,
            "walk_ms": float(np.mean(wms)), "finalize_ms": float(np.mean(fms)), "points": n, "trees": trees,
            "nodes": nodes, "pruned_trees": pruned, "K": K, "L": wl["L"], "M": wl["M"],
            "walk_config": dict(zip(["warps", "smem_levels", "blocks_per_sm", "tile"], cfg)), "finite_output": finite}


# ---------------------------------------------------------------------------
# PDD pipeline: interface point solves -> spline -> subdomain Crank-Nicolson
# ---------------------------------------------------------------------------
PDD_GRID = dict(dim=3, lo=[0.0] * 3, hi=[4.0] * 3, sub=[4] * 3, cells=[16] * 3, nodes=[17] * 3, t_nodes=4, T=1.0,
                nsteps=100)


def pdd_flops(g: dict) -> float:
    """Algorithmic FP64 flops of grt_pdd_solve (FMA = 2): per subdomain step, 2 d sine-transform passes of
    m_a flops-pairs per unknown plus the right-hand side (~40 flops per unknown: stencil, reaction, ring
    terms); the spline's three contractions per plane family."""
    d = g["dim"]
    m = [c - 1 for c in g["cells"][:d]]
    mloc = int(np.prod(m))
    nsub = int(np.prod(g["sub"][:d]))
    per_step = sum(2 * 2 * mloc * ma for ma in m) + 40 * mloc
    cn = float(nsub) * g["nsteps"] * per_step
    N = [g["sub"][a] * g["cells"][a] + 1 for a in range(d)]
    spl = 0.0
    tn = g["t_nodes"] + 1
    for a in range(d):
        np_ = g["sub"][a] + 1
        oth = [b for b in range(d) if b != a]
        pn = int(np.prod([g["nodes"][b] for b in oth])) if oth else 1
        spl += 2.0 * np_ * g["nsteps"] * pn * tn
        if len(oth) >= 1:
            nc = g["nodes"][oth[1]] if len(oth) > 1 else 1
            spl += 2.0 * np_ * g["nsteps"] * N[oth[0]] * nc * g["nodes"][oth[0]]
        if len(oth) == 2:
            spl += 2.0 * np_ * g["nsteps"] * N[oth[0]] * N[oth[1]] * g["nodes"][oth[1]]
    return cn + spl


def pdd_bench(grt, dev_index: int, steps: int) -> dict:
    """The 3-D interface problem end to end on the GPU: point solves at every plane's nodal points (the
    outer faces included) and time levels, then grt_pdd_solve (spline + 64 independent subdomain solves)."""
    import torch

    dev = torch.device("cuda", dev_index)
    wl = workloads.workload_pdd_3d()
    g = PDD_GRID
    x, t = grt.grt_pdd_points(g)
    n = x.shape[0]
    ctx = grt.grt_create(wl["problem"], dev_index)
    plan = grt.grt_plan_create(ctx, np.full(n, 100_000, np.uint64), wl["K"], wl["L"], wl["M"])
    dx, dtt = torch.from_numpy(x).to(dev), torch.from_numpy(t).to(dev)
    u = torch.empty(n, dtype=torch.float64, device=dev)
    N = [g["sub"][a] * g["cells"][a] + 1 for a in range(3)]
    out = torch.empty(N, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    s = torch.cuda.Stream(device=dev)
    grt.grt_plan_autotune(plan, dx, dtt, 0, 0, u, stream=s)
    grt.grt_pdd_solve(ctx, g, u, out, stream=s)  # warm-up
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    for e0, e1, e2 in ev:
        with torch.cuda.stream(s):
            flush.zero_()
        e0.record(s)
        grt.grt_plan_execute(plan, dx, dtt, 0, 0, u, stream=s)
        e1.record(s)
        grt.grt_pdd_solve(ctx, g, u, out, stream=s)
        e2.record(s)
    torch.cuda.synchronize(dev)
    mc = float(np.mean([a.elapsed_time(b) for a, b, _ in ev]))
    pd = float(np.mean([b.elapsed_time(c) for _, b, c in ev]))
    finite = bool(torch.isfinite(out).all().item())
    # the interface values the Pade has spoiled, at the last time level (t = T = 1) and over all levels
    health_T = pade_health(grt, ctx, plan, dx, dtt, 0, wl["K"], wl["L"], wl["M"], tmask=np.isclose(t, g["T"]))
    health_all = pade_health(grt, ctx, plan, dx, dtt, 0, wl["K"], wl["L"], wl["M"])
    plan.close()
    ctx.close()
    nsub = int(np.prod(g["sub"]))
    flops = pdd_flops(g)
    fp64_peak = 1.25  # TFLOP/s, nominal GB300 FP64 (not a tensor path)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    # blocks per subdomain: a cluster pair when half of the subdomain's four vectors fits in 200 KB
    m = [c - 1 for c in g["cells"]]
    half = 4 * ((m[0] + 1) // 2) * int(np.prod(m[1:])) * 8
    per_sub = 2 if m[0] >= 2 and half <= 200 * 1024 else 1
    return {"points": n, "trees": 100_000 * n, "grid_nodes": int(np.prod(N)), "subdomains": nsub,
            "pdd_flops": flops, "pdd_fp64_tflops": flops / (pd / 1e3) / 1e12,
            "pdd_roofline": {"bound": "fp64", "achieved": flops / (pd / 1e3) / 1e12, "peak": fp64_peak,
                             "unit": "TFLOP/s", "frac": flops / (pd / 1e3) / 1e12 / fp64_peak,
                             "frac_of_used_sms": flops / (pd / 1e3) / 1e12
                             / (fp64_peak * min(per_sub * nsub, sms) / sms),
                             "blocks_per_subdomain": per_sub,
                             "peak_basis": f"nominal GB300 FP64 rate (no measured FP64 peak is available); "
                                           f"the subdomain blocks run on min(blocks, {sms}) SMs"},
            "subdomain_unknowns": int(np.prod([c - 1 for c in g["cells"]])), "cn_steps": g["nsteps"],
            "point_solve_ms": mc, "pdd_stage_ms": pd, "total_ms": mc + pd, "steps": steps,
            "finite_output": finite, "pade_health_at_T": health_T, "pade_health_all_levels": health_all,
            "description": ("u_t = 0.1 Lap u + u - u^3, u0 = prod tanh(x_i - 2) on [0,4]^3 cut into 4x4x4 subdomains; "
                            "15 planes (outer faces = probabilistic artificial boundaries) x 17^2 nodes x 4 time levels "
                            "= 17340 point solves of 1e5 trees, K = 12 [6/6]; not-a-knot tensor spline to the 65^3 "
                            "finite-difference grid at 100 Crank-Nicolson steps, 64 subdomains of 15^3 unknowns")}


# ---------------------------------------------------------------------------
# serving: Poisson trace through the continuous-batching server vs the plain path
# ---------------------------------------------------------------------------
def _pct(v, q):
    return float(np.percentile(np.asarray(v, float), q)) if len(v) else None


def _serve_trace(grt, dev: int, probs: dict, ctxs: dict, trace: list) -> dict:
    """Replay a trace in real time through a fresh server: latency per request, wall time, steps."""
    server = grt.grt_server_create(dev, mem_budget_bytes=16 << 30, step_trees=1 << 26)
    # warm-up: one small request per problem (first launch of every kernel instantiation)
    warm = []
    for k, v in probs.items():
        d = v["problem"]["dim"]
        warm.append(grt.grt_submit(server, ctxs[k], np.zeros((4, d)), np.full(4, 0.5), np.full(4, 20000, np.uint64),
                                   v["K"], v["L"], v["M"], 99))
    for rid in warm:
        grt.grt_poll(server, rid, -1)
    st0 = grt.grt_server_stats(server)
    ids = [None] * len(trace)
    t0 = time.perf_counter()

    def submitter():
        for k, r in enumerate(trace):
            delay = t0 + r["arrival"] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            v = probs[r["key"]]
            ids[k] = grt.grt_submit(server, ctxs[r["key"]], r["x"], r["t"], r["ntrees"], v["K"], v["L"], v["M"],
                                    r["seed"], r["point_base"])

    th = threading.Thread(target=submitter)
    th.start()
    lat = [None] * len(trace)
    for k in range(len(trace)):
        while ids[k] is None:
            time.sleep(0.0005)
        res = grt.grt_poll(server, ids[k], -1)
        lat[k] = res["latency_s"]
    t_end = time.perf_counter()
    th.join()
    st1 = grt.grt_server_stats(server)
    server.close()
    points = int(sum(len(r["t"]) for r in trace))
    shared = st1["shared_launches"] - st0["shared_launches"]
    trees = float(sum(float(r["ntrees"].sum()) for r in trace))
    wall = t_end - t0
    return {"lat": lat, "requests": len(trace), "p50_ms": 1e3 * _pct(lat, 50), "p99_ms": 1e3 * _pct(lat, 99),
            "mean_ms": 1e3 * float(np.mean(lat)), "points_per_s": points / wall, "trees_per_s": trees / wall,
            "wall_s": wall, "steps": st1["steps"] - st0["steps"], "launches": st1["launches"] - st0["launches"],
            "shared_launches": shared}


def serving_bench(grt, dev: int, capacity_trees_per_s: float, n_requests: int, plain_requests: int,
                  plain_cap_s: float, overload_requests: int = 2000) -> dict:
    probs = workloads.serving_problems("fp32")
    ctxs = {k: grt.grt_create(v["problem"], dev) for k, v in probs.items()}
    mean_trees = workloads.serving_mean_trees()
    rate = 0.7 * capacity_trees_per_s / mean_trees
    trace = workloads.serving_trace(n_requests, rate, seed=0)
    run = _serve_trace(grt, dev, probs, ctxs, trace)
    lat = run.pop("lat")
    out = dict(trace=(f"{len(trace)} Poisson requests at {rate:.1f} req/s (0.7 x the measured sin_2d capacity / mean "
                      f"request of {mean_trees:.3g} trees); 1-4096 points log-uniform, 1e3-1e7 trees per point "
                      f"log-uniform; f in (u^2-u, sin u, u-u^3) x d in (1, 2, 3); one service-wide seed, "
                      f"disjoint point streams per request; 16 GB admission budget; 2^26-tree steps"), **run)
    if overload_requests > 0:
        # the configured arrival rate, 2000 req/s: ~20x what one GPU serves at these budgets, so the
        # requests queue (admission by memory, smallest remaining work first)
        over = _serve_trace(grt, dev, probs, ctxs, workloads.serving_trace(overload_requests, 2000.0, seed=0))
        over.pop("lat")
        out["at_configured_rate"] = dict(trace=f"the first {overload_requests} Poisson arrivals at 2000 req/s "
                                               f"(seed 0), same mix", **over)
    # plain path: one FP64 launch per point (grt_solve_plain), requests first come first served, same arrivals
    ctx64 = {k: grt.grt_create(dict(v["problem"], precision="fp64"), dev) for k, v in probs.items()}
    for k, v in probs.items():  # warm-up
        d = v["problem"]["dim"]
        grt.grt_solve_plain(ctx64[k], np.zeros((2, d)), np.full(2, 0.5), np.full(2, 1000, np.uint64), v["K"], v["L"],
                            v["M"], 99, want_coef=False, want_se=False)
    plat, ppoints, ptrees = [], 0, 0.0
    t0 = time.perf_counter()
    for r in trace[:plain_requests]:
        now = time.perf_counter() - t0
        if now < r["arrival"]:
            time.sleep(r["arrival"] - now)
        v = probs[r["key"]]
        grt.grt_solve_plain(ctx64[r["key"]], r["x"], r["t"], r["ntrees"], v["K"], v["L"], v["M"], r["seed"],
                            r["point_base"], want_coef=False, want_se=False)
        plat.append(time.perf_counter() - t0 - r["arrival"])
        ppoints += len(r["t"])
        ptrees += float(r["ntrees"].sum())
        if time.perf_counter() - t0 > plain_cap_s:
            break
    pwall = time.perf_counter() - t0
    m = len(plat)
    out["plain"] = {
        "kind": "grt_solve_plain: one FP64 kernel launch per point (walk, block reductions and Pade in the launch), "
                "requests first come first served, same arrivals",
        "requests": m, "p50_ms": 1e3 * _pct(plat, 50), "p99_ms": 1e3 * _pct(plat, 99),
        "points_per_s": ppoints / pwall, "trees_per_s": ptrees / pwall,
        "batched_p50_ms_same_requests": 1e3 * _pct(lat[:m], 50),
        "batched_p99_ms_same_requests": 1e3 * _pct(lat[:m], 99),
    }
    for c in list(ctxs.values()) + list(ctx64.values()):
        c.close()
    return out


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def gpu_arm(args) -> int:
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    # NCCL across the node's GPUs; GRT_DIST_BACKEND=gloo runs the same path with host-side collectives
    # (used to exercise the multi-rank code on a single GPU: ranks share it, no kernel waits on another)
    backend = os.environ.get("GRT_DIST_BACKEND", "nccl")
    gpu = local % max(torch.cuda.device_count(), 1)
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
        torch.cuda.set_device(gpu)
        if backend == "nccl":
            dist.init_process_group("nccl", device_id=torch.device("cuda", gpu))
        else:
            dist.init_process_group(backend)
    dev = torch.device("cuda", gpu)
    torch.cuda.set_device(dev)
    red_dev = dev if backend == "nccl" else torch.device("cpu")

    import __graft_entry__

    if rank == 0:
        __graft_entry__.build()
    if dist is not None:
        dist.barrier()
    import paper_2402_06491_gb300 as grt

    wl = workloads.WORKLOADS[WORKLOAD]()
    if args.trees:
        wl["ntrees"] = np.full_like(wl["ntrees"], args.trees)
    n, K, L, M = wl["x"].shape[0], wl["K"], wl["L"], wl["M"]
    point_base = rank * n
    trees_per_step = float(np.sum(wl["ntrees"]))
    ctx = grt.grt_create(wl["problem"], gpu)
    plan = grt.grt_plan_create(ctx, wl["ntrees"], K, L, M)
    grt.grt_plan_set_timing(plan, True)
    x = torch.from_numpy(wl["x"]).to(dev)
    t = torch.from_numpy(wl["t"]).to(dev)
    u = torch.empty(n, dtype=torch.float64, device=dev)
    coef = torch.empty((n, K + 1), dtype=torch.float64, device=dev)
    status = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def step():
        grt.grt_plan_execute(plan, x, t, wl["seed"], point_base, u, coef, None, status, stream=stream)

    if args.walk_config:
        walk_cfg = tuple(int(v) for v in args.walk_config.split(","))
        grt.grt_plan_set_config(plan, list(walk_cfg))
    else:
        walk_cfg = grt.grt_plan_autotune(plan, x, t, wl["seed"], point_base, u, coef, None, status, stream=stream)
    stream.synchronize()

    for _ in range(max(args.warmup, 0)):
        with torch.cuda.stream(stream):
            flush.zero_()
        step()
    stream.synchronize()
    nodes, splits, pruned = grt.grt_plan_counters(plan)

    props = torch.cuda.get_device_properties(dev)
    bus, devid = getattr(props, "pci_bus_id", None), getattr(props, "pci_device_id", None)
    bus_str = f"{bus:02x}:{devid:02x}.0" if isinstance(bus, int) and isinstance(devid, int) else None
    if torch.cuda.device_count() == 1 and not os.environ.get("CUDA_VISIBLE_DEVICES"):
        bus_str = None
    sampler = ClockSampler(bus_str)
    sampler.start()
    time.sleep(0.3)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    walk_ms, fin_ms = [], []
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t_wall0 = time.time()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        starts[k].record(stream)
        step()
        ends[k].record(stream)
        wm, fm = grt.grt_plan_timing(plan)
        walk_ms.append(wm)
        fin_ms.append(fm)
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    t_wall1 = time.time()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = float(sum(step_ms))
    if dist is not None:
        tt = torch.tensor([total_ms], dtype=torch.float64, device=red_dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    time.sleep(0.3)
    sampler.stop()
    clocks = sampler.summary(t_wall0 - 0.05, t_wall1 + 0.05)

    # the same step replayed from a CUDA graph of one execution
    grt.grt_plan_graph_capture(plan, x, t, wl["seed"], point_base, u, coef, None, status)
    g_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in g_ev:
        with torch.cuda.stream(stream):
            flush.zero_()
        a.record(stream)
        grt.grt_plan_graph_launch(plan, stream)
        b.record(stream)
    torch.cuda.synchronize(dev)
    graph_ms = float(np.mean([a.elapsed_time(b) for a, b in g_ev]))

    # parity spot check of this run's output (rank 0's first points) is in the test suite; here the
    # result must at least be finite
    u_host = u.cpu().numpy()
    finite = bool(np.all(np.isfinite(u_host)))
    # each result's statistical error: one more execute with standard errors, then grt_pade_error
    se_d = torch.empty((n, K + 1), dtype=torch.float64, device=dev)
    grt.grt_plan_execute(plan, x, t, wl["seed"], point_base, u, coef, se_d, status, stream=stream)
    err_d = torch.empty(n, dtype=torch.float64, device=dev)
    grt.grt_pade_error(ctx, coef, se_d, L, M, err_d, stream=stream)
    stream.synchronize()
    err_h = err_d.cpu().numpy()
    rel_err = err_h / np.maximum(np.abs(u_host), 1e-300)
    stat_err = {"median_abs": float(np.median(err_h)), "max_abs": float(np.max(err_h)),
                "median_rel": float(np.median(rel_err)),
                "note": "first-order spread of the Pade value from the coefficients' standard errors "
                        "(grt_pade_error), per point at this run's tree budget"}
    # FP32 rounding of each result.  Every tree weight is within eps = 3e-5 of its FP64 value
    # (per-tree parity), so S1_n moves by at most eps SA_n: |da_n| <= eps kappa_n |a_n| with
    # kappa_n = SA_n/|S1_n| (worst case: all trees' errors of one sign).  Rounding errors of
    # independent trees add like noise instead, sqrt(sum W^2) eps = eps sqrt(S2_n): da_n ~ eps
    # sqrt(SE_n^2 + a_n^2/N).  Both propagate through the Pade by its first-order sensitivities
    # (grt_pade_error; sqrt(L+M+1) x its quadrature sum bounds the linear sum of the worst case).
    kap_d = torch.empty((n, K + 1), dtype=torch.float64, device=dev)
    grt.grt_plan_kappa(plan, kap_d, stream=stream)
    stream.synchronize()
    coef_h, kap_h, se_h = coef.cpu().numpy(), kap_d.cpu().numpy(), se_d.cpu().numpy()
    Nt = np.maximum(np.asarray(wl["ntrees"], np.float64), 1.0)[:, None]
    da_worst = np.where(np.isfinite(kap_h), FP32_WEIGHT_RTOL * kap_h * np.abs(coef_h), 0.0)
    da_noise = FP32_WEIGHT_RTOL * np.sqrt(se_h * se_h + coef_h * coef_h / Nt)
    scale = np.maximum(np.abs(u_host), np.abs(coef_h).sum(axis=1))
    rel = {}
    for name, da, mult in (("worst", da_worst, math.sqrt(L + M + 1)), ("noise", da_noise, 1.0)):
        da_dev = torch.from_numpy(np.ascontiguousarray(da)).to(dev)
        rb_d = torch.empty(n, dtype=torch.float64, device=dev)
        grt.grt_pade_error(ctx, coef, da_dev, L, M, rb_d, stream=stream)
        stream.synchronize()
        rel[name] = rb_d.cpu().numpy() * mult / np.maximum(scale, 1e-300)
    over = np.where(~(rel["worst"] <= 1e-5))[0]
    fin = np.isfinite(kap_h)
    fp32_bound = {
        "worst_case_median_rel": float(np.median(rel["worst"])), "worst_case_max_rel": float(np.max(rel["worst"])),
        "worst_case_over_1e-5": int(over.size), "worst_case_over_1e-5_first": [int(i) + point_base for i in over[:20]],
        "independent_median_rel": float(np.median(rel["noise"])), "independent_max_rel": float(np.max(rel["noise"])),
        "kappa_max": float(np.max(kap_h[fin])) if fin.any() else None,
        "note": "FP32 walk rounding on each Pade value relative to max(|u|, sum |a_n|), per-tree weights within "
                "3e-5 (tested): worst case 3e-5 kappa_n |a_n| per coefficient (kappa_n = SA_n/|S1_n|, "
                "grt_plan_kappa), and independent per-tree errors 3e-5 sqrt(SE_n^2 + a_n^2/N)"}

    # end to end through the public host-buffer call: H2D of the step's inputs, D2H of its result;
    # the one-shot solve takes the plan's launch shape
    grt.grt_set_solve_config(ctx, grt.grt_plan_get_config(plan))
    e2e_steps = 0 if args.no_e2e else max(args.steps, 1)
    xh = torch.from_numpy(wl["x"]).pin_memory().numpy()
    th = torch.from_numpy(wl["t"]).pin_memory().numpy()
    nth = torch.from_numpy(wl["ntrees"].astype(np.int64)).pin_memory().numpy().view(np.uint64)
    uh = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
    sth = torch.empty(n, dtype=torch.int32).pin_memory().numpy()
    out = {"u": uh, "status": sth}
    for _ in range(max(args.warmup, 1) if e2e_steps else 0):
        grt.grt_solve(ctx, xh, th, nth, K, L, M, wl["seed"], point_base, want_coef=False, want_se=False, out=out)
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        grt.grt_solve(ctx, xh, th, nth, K, L, M, wl["seed"], point_base, want_coef=False, want_se=False, out=out)
    e2e_s = max(time.perf_counter() - t0, 1e-9)
    if dist is not None:
        te = torch.tensor([e2e_s], dtype=torch.float64, device=red_dev)
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e_s = float(te.item())
    same = bool(np.array_equal(uh, u_host)) if e2e_steps else None
    h2d = xh.nbytes + th.nbytes
    d2h = uh.nbytes + sth.nbytes

    launches_per_step = grt.grt_plan_launches(plan)
    plan.close()
    ctx.close()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    value = world * trees_per_step * args.steps / (total_ms / 1e3)
    points_per_s = world * n * args.steps / (total_ms / 1e3)
    model = instruction_model(wl["problem"], K)
    inst = algorithmic_instructions(model, nodes, splits, int(trees_per_step))
    walk_avg_ms = float(np.mean(walk_ms))
    achieved = inst / (walk_avg_ms / 1e3) / 1e12
    peaks = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sms = int(props.multi_processor_count)
    peak = n_sms * ISSUE_PER_SM_PER_CLK * sm_max * 1e6 / 1e12
    walk_prof = _walk_profile()
    ncu_figs = walk_prof[1] or {}
    line = {
        "metric": METRIC, "value": value, "unit": "trees/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "points_per_s": points_per_s,
        "config": {
            "workload": "sin_2d: 2-D u_t = 0.5 Lap u + sin u (degree-9 Taylor), u0 = 1.2 exp(-|x|^2/2), "
                        "16x16 grid x t in {0.25, 1}, FP32 walk, FP64 Pade",
            "points": n, "trees_per_point": int(wl["ntrees"][0]), "K": K, "L": L, "M": M,
            "q": round(wl["problem"]["q"], 6), "seed": wl["seed"],
            "l2": "flushed between steps (256 MiB write)",
            "parallelism": f"{world} GPU(s), points sharded (weak), no collective",
        },
        "roofline": {
            "bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tinst/s", "frac": achieved / peak,
            "traffic": walk_prof[0] if not args.trees else None,
            "issue_active_ncu": ncu_figs.get("issue_active"),
            "lane_efficiency_ncu": ncu_figs.get("lane_efficiency"),
            "walk_ms": walk_avg_ms, "finalize_ms": float(np.mean(fin_ms)), "graph_ms_per_step": graph_ms,
            "peak_basis": f"{n_sms} SMs x 128 thread-inst/clk x {sm_max:.0f} MHz; achieved = algorithmic "
                          f"inst / walk event time",
        },
        "e2e": ({"value": world * trees_per_step * e2e_steps / e2e_s, "unit": "trees/s", "h2d_bytes_per_step": h2d,
                 "d2h_bytes_per_step": d2h, "matches_device_run": same} if e2e_steps else None),
        "gpu_launches": launches_per_step * args.steps,
        "clocks": {k: clocks.get(k) for k in ("sm_mhz", "sm_max_mhz", "reasons", "samples")},
    }
    # everything else goes to the side file (the headline line stays short enough for log tails)
    details = {
        "roofline": {
            "ncu": walk_prof[1], "walk_config": dict(zip(["warps", "smem_levels", "blocks_per_sm", "tile"], walk_cfg)),
            "work": f"{inst:.4g} algorithmic thread-instructions per launch = {model['node']}/node x {nodes} nodes"
                    f" + {model['leaf']}/leaf x {nodes - splits} + {model['split']}/split x {splits}"
                    f" + {model['tree']}/tree x {int(trees_per_step)}",
            "issue_note": "smsp__issue_active of the walk kernel (ncu --set full, small case; "
                          "profiles/walk_kernel_sin2d.md): the hardware's SM issue-slot utilisation, beside the "
                          "stricter algorithmic fraction `frac`",
            "traffic_note": "ncu dram__bytes_read+write of one full-size walk launch (profiles/walk_kernel_sin2d.md)",
        },
        "clocks": clocks,
        "work_counters": {"nodes": nodes, "splits": splits, "pruned_trees": pruned, "trees": int(trees_per_step)},
        "statistical_error": stat_err,
        "fp32_rounding_bound": fp32_bound,
        "finite_output": finite,
    }
    # the single-GPU lines (other workloads, serving, CPU baseline) are measured at N = 1 only: at N > 1
    # the run is about the sharded main workload, and the other GPUs would idle meanwhile
    if not args.no_workloads and world == 1:
        wls = {
            "uneven_2d": dict(workload_bench(grt, gpu, "uneven_2d", 5), description=(
                "2-D u_t = Lap u + u^2, u0 = 1.5 + 0.5 cos x cos y, 4096 points on 64 interface segments of the 8x8 "
                "split of [0,8]^2, t ~ U[0.1, 2], budgets log-uniform in [1e3, 1e6] (5.9e8 trees), K = 16, [8/8]")),
            "pdd_3d": dict(workload_bench(grt, gpu, "pdd_3d", 3), description=(
                "3-D u_t = 0.1 Lap u + u - u^3, u0 = prod tanh(x_i - 2), 9 interior planes x 32^2 nodes of the "
                "4x4x4 split of [0,4]^3, t = 1, 1e5 trees per point (9.2e8 trees), K = 12, [6/6]")),
            "pdd_3d_pipeline": pdd_bench(grt, gpu, 3),
            "drift_2d": dict(workload_bench(grt, gpu, "drift_2d", 10), description=(
                "general drift and diffusion: u_t = sum_i (s_i^2/2) d_ii u - kappa_i x_i d_i u + u^2 - u, kappa = (1, 0.5), "
                "s = (1, 0.7) (OU paths by Euler-Maruyama, 8 steps per segment), u0 = exp(-|x - (0.5,-0.3)|^2/1.28), "
                "t = 0.5, 16x16 grid in [-3,3]^2, 1e5 trees per point, K = 8, [4/4]")),
            "var_coef_2d": dict(workload_bench(grt, gpu, "var_coef_2d", 10), description=(
                "Example 5: 2-D u_t = Lap u - e^{-x^2}/(t + 0.1) u^2 (variable coefficient), u0 = e^{-x^2/4}/sqrt(4 pi), "
                "t = 0.5, 16x16 grid in [-3,3]^2, 1e5 trees per point, binary trees q = 2/3, K = 8, [4/4]")),
        }
        details["workloads"] = wls
        line["workloads_trees_per_s"] = {k: float(f"{v['trees_per_s']:.4g}") for k, v in wls.items()
                                         if "trees_per_s" in v}
        pp = wls["pdd_3d_pipeline"]
        line["pdd_3d_pipeline_ms"] = {"point_solves": round(pp["point_solve_ms"], 3),
                                      "pdd_stage": round(pp["pdd_stage_ms"], 3)}
        h = wls["pdd_3d"]["pade_health"]
        line["pdd_3d_pade_at_t1"] = {"points": h["points"], "pole_near": h["pole_near"],
                                     "err_over_1e-2": h["err_over_1e-2"]}
    if not args.no_serving and world == 1:
        srv = serving_bench(grt, gpu, value / world, args.serving_requests, args.plain_requests,
                            float(os.environ.get("GRT_PLAIN_CAP_S", "30")), args.overload_requests)
        details["serving"] = srv
        line["serving"] = serving_summary(srv)
    if world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(wl, float(os.environ.get("GRT_CPU_BASELINE_S", "10")),
                          gpu=(u_host, coef.cpu().numpy()) if point_base == 0 else None)
        details["cpu_baseline"] = cb
        short = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        ev = cb.get("error_vs_oracle")
        if ev is not None:
            short["error_vs_oracle"] = {k: ev[k] for k in ("points", "max_rel", "median_rel", "within_bar")}
        line["cpu_baseline"] = short
    if args.details:
        try:
            with open(args.details, "w") as fh:
                json.dump(dict(line=line, **details), fh, indent=1)
            line["details"] = args.details
        except OSError as exc:
            print(f"bench: could not write {args.details}: {exc}", file=sys.stderr)
    print(headline_json(line))
    sys.stdout.flush()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def serving_summary(srv: dict) -> dict:
    """The serving figures the headline metric names: p50/p99 latency and points/s of the batched
    server against the plain one-launch-per-point FP64 path, on the same requests."""
    out = {k: srv.get(k) for k in ("requests", "p50_ms", "p99_ms", "points_per_s", "trees_per_s", "shared_launches")}
    pl = srv.get("plain") or {}
    out["plain"] = {k: pl.get(k) for k in ("requests", "p50_ms", "p99_ms", "points_per_s",
                                           "batched_p50_ms_same_requests", "batched_p99_ms_same_requests")}
    for key in ("shared_launch_steps", "at_configured_rate"):
        if key in srv:
            v = srv[key]
            out[key] = ({k: v.get(k) for k in ("p50_ms", "p99_ms", "points_per_s", "shared_launches")}
                        if isinstance(v, dict) else v)
    return out


HEADLINE_MAX_BYTES = 2400
# optional keys dropped, in this order, should the headline line outgrow HEADLINE_MAX_BYTES (all of them
# stay in the side file)
HEADLINE_OPTIONAL = (("serving", "at_configured_rate"), ("pdd_3d_pade_at_t1",), ("pdd_3d_pipeline_ms",),
                     ("workloads_trees_per_s",),
                     ("roofline", "graph_ms_per_step"), ("serving",))


def headline_json(line: dict) -> str:
    """The one-line JSON record: floats to 5 significant digits, optional keys dropped while it is
    longer than HEADLINE_MAX_BYTES."""
    out = _compact(line)
    text = json.dumps(out, separators=(",", ":"))
    for path in HEADLINE_OPTIONAL:
        if len(text) <= HEADLINE_MAX_BYTES:
            break
        d = out
        for key in path[:-1]:
            d = d.get(key, {}) if isinstance(d, dict) else {}
        if isinstance(d, dict) and path[-1] in d:
            del d[path[-1]]
            text = json.dumps(out, separators=(",", ":"))
    return text


def _compact(obj, digits: int = 5):
    """Floats to `digits` significant digits (the headline line is read from a log tail)."""
    if isinstance(obj, float):
        return float(f"{obj:.{digits}g}") if math.isfinite(obj) else None
    if isinstance(obj, dict):
        return {k: _compact(v, digits) for k, v in obj.items()}
    if isinstance(obj, (list, tuple)):
        return [_compact(v, digits) for v in obj]
    return obj


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="grt", choices=["grt", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer measurement")
    ap.add_argument("--trees", type=int, default=0, help="trees per point (profiling cases; default: the workload's)")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving trace")
    ap.add_argument("--no-workloads", action="store_true", help="skip the uneven_2d and pdd_3d lines")
    ap.add_argument("--walk-config", default="",
                    help="fixed walk launch shape 'warps,smem_levels,blocks_per_sm,tile' instead of the autotuner")
    ap.add_argument("--serving-requests", type=int, default=150)
    ap.add_argument("--plain-requests", type=int, default=20)
    ap.add_argument("--overload-requests", type=int, default=2000,
                    help="requests of the trace replayed at the configured 2000 req/s (0: skip it)")
    ap.add_argument("--details", default="bench_details.json",
                    help="side JSON file for the per-result and per-workload figures ('' = none)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
