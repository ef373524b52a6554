"""Serving: continuous batching of point-solve requests (grt_server / grt_submit / grt_poll).

Each request's result must equal, bit for bit, the one-shot grt_solve of the
same points (same stream indices and seed) -- alone or in any mix of concurrent
requests, and however the scheduler split its trees over steps.
"""
import threading
import time

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def grt():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2402_06491_gb300 as pkg

    return pkg


def _requests(rng):
    """A mix of problems, dimensions, series shapes, sizes and budgets (some split over many steps)."""
    specs = []
    for name, npts, lo, hi in [("sin_2d", 7, 1000, 40000), ("kpp_1d", 5, 500, 9000), ("pdd_3d", 4, 2000, 30000),
                               ("uneven_2d", 3, 100, 70000), ("sin_2d", 1, 0, 1), ("sin_2d", 2, 8192, 8193),
                               ("var_coef_2d", 3, 5000, 30000), ("drift_2d", 2, 3000, 20000)]:
        wl = workloads.WORKLOADS[name]()
        idx = rng.choice(wl["x"].shape[0], size=npts, replace=False)
        nt = rng.integers(lo, hi, size=npts).astype(np.uint64)
        specs.append(dict(name=name, problem=wl["problem"], x=wl["x"][idx], t=wl["t"][idx], ntrees=nt, K=wl["K"],
                          L=wl["L"], M=wl["M"], seed=int(rng.integers(0, 3)), point_base=int(rng.integers(0, 1000))))
    return specs


def test_results_equal_one_shot_solves_in_a_concurrent_mix(grt):
    rng = np.random.default_rng(5)
    specs = _requests(rng)
    ctxs = {}
    for s in specs:
        if s["name"] not in ctxs:
            ctxs[s["name"]] = grt.grt_create(s["problem"], 0)
    server = grt.grt_server_create(0, mem_budget_bytes=512 << 20, step_trees=1 << 16)
    ids = [None] * len(specs)

    def submit(k):
        s = specs[k]
        ids[k] = grt.grt_submit(server, ctxs[s["name"]], s["x"], s["t"], s["ntrees"], s["K"], s["L"], s["M"],
                                s["seed"], s["point_base"])

    threads = [threading.Thread(target=submit, args=(k,)) for k in range(len(specs))]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    results = [grt.grt_poll(server, rid, -1) for rid in ids]
    stats = grt.grt_server_stats(server)
    assert stats["steps"] > 5 and stats["active"] == 0 and stats["pending"] == 0
    from test_parity_gpu import _assert_fp32_parity

    for s, r in zip(specs, results):
        ref = grt.grt_solve(ctxs[s["name"]], s["x"], s["t"], s["ntrees"], s["K"], s["L"], s["M"], s["seed"],
                            s["point_base"])
        assert np.array_equal(r["coef"], ref["coef"]), s["name"]
        assert np.array_equal(r["se"], ref["se"]), s["name"]
        assert np.array_equal(r["status"], ref["status"]), s["name"]
        assert np.array_equal(r["u"], ref["u"]) or np.allclose(r["u"], ref["u"], equal_nan=True, rtol=0, atol=0)
        assert r["latency_s"] >= 0.0
        # and against the FP64 oracle on the same streams (two points of every request)
        for i in range(min(2, len(s["t"]))):
            o = oracle.solve(s["problem"], s["x"][i:i + 1], s["t"][i:i + 1], s["ntrees"][i:i + 1], s["K"], s["L"],
                             s["M"], s["seed"], point_base=s["point_base"] + i)
            gi = {k: r[k][i:i + 1] for k in ("u", "coef", "status")}
            if s["problem"]["precision"] == "fp64":
                assert np.allclose(gi["coef"], o["coef"], rtol=1e-12, atol=1e-15), s["name"]
            else:
                ctol = 1.5e-4 if s["name"] == "pdd_3d" else 3e-5
                blow = np.array([s["name"] == "uneven_2d" and s["t"][i] >= 0.5])
                _assert_fp32_parity(gi, o, s["ntrees"][i:i + 1], ctol=ctol, L=s["L"], M=s["M"], unpinned=blow)
    server.close()
    for c in ctxs.values():
        c.close()


def _min_budget(grt, step):
    """The smallest budget a server with this step size accepts, and the points it holds resident."""
    sz = grt.grt_server_sizes(step)
    return sz["step_bytes"] + (1 << 20), (1 << 20) // sz["point_bytes"]


def test_admission_waits_for_memory(grt):
    wl = workloads.workload_sin_2d()
    ctx = grt.grt_create(wl["problem"], 0)
    step = 1 << 16
    budget, cap = _min_budget(grt, step)
    # each request below has 200 points, each point one resident accumulator and result row: at most
    # three requests are admitted at a time
    assert 600 <= cap < 800
    server = grt.grt_server_create(0, mem_budget_bytes=budget, step_trees=step)
    rng = np.random.default_rng(5)
    x, t = rng.uniform(-3.0, 3.0, (2400, 2)), rng.uniform(0.1, 1.0, 2400)
    nt = np.full(200, 20 * 8192, np.uint64)
    ids = []
    for k in range(12):
        sl = slice(k * 200, k * 200 + 200)
        ids.append(grt.grt_submit(server, ctx, x[sl], t[sl], nt, wl["K"], wl["L"], wl["M"], 0, k * 200))
    peak_active = 0
    res = {}
    while len(res) < len(ids):
        st = grt.grt_server_stats(server)
        peak_active = max(peak_active, st["active"])
        for rid in ids:
            if rid not in res:
                r = grt.grt_poll(server, rid, 0)
                if r is not None:
                    res[rid] = r
    assert 1 <= peak_active <= 3
    ref = grt.grt_solve(ctx, x, t, np.full(2400, 20 * 8192, np.uint64), wl["K"], wl["L"], wl["M"], 0)
    assert np.array_equal(np.concatenate([res[rid]["coef"] for rid in ids]), ref["coef"])
    server.close()
    ctx.close()


def test_errors_and_empty_requests(grt):
    wl = workloads.workload_sin_2d()
    ctx = grt.grt_create(wl["problem"], 0)
    with pytest.raises(grt.GrtError):
        grt.grt_server_create(0, mem_budget_bytes=1 << 20, step_trees=1 << 16)  # budget below the step buffers
    budget, cap = _min_budget(grt, 1 << 16)
    server = grt.grt_server_create(0, mem_budget_bytes=budget, step_trees=1 << 16)
    rid = grt.grt_submit(server, ctx, np.zeros((0, 2)), np.zeros(0), np.zeros(0, np.uint64), 10, 5, 5, 0)
    r = grt.grt_poll(server, rid, 0)
    assert r is not None and r["u"].shape == (0,)
    with pytest.raises(grt.GrtError):
        grt.grt_submit(server, ctx, np.zeros((1, 2)), [1.0], [10], 10, 6, 5, 0)
    with pytest.raises(grt.GrtError):  # more points than the whole budget holds resident
        grt.grt_submit(server, ctx, np.zeros((cap + 1, 2)), np.ones(cap + 1), np.ones(cap + 1, np.uint64), 10, 5, 5, 0)
    with pytest.raises(grt.GrtError):
        grt.grt_server_sizes(4096)  # steps below one 8192-tree chunk
    rid = grt.grt_submit(server, ctx, np.zeros((3, 2)), [0.5, 1.0, 0.25], [20000, 1, 0], 10, 5, 5, 7)
    assert grt.grt_poll(server, rid, -1)["u"].shape == (3,)
    server.close()
    ctx.close()


def test_requests_that_arrive_while_another_runs_share_its_launches(grt):
    """A request submitted while another of the same problem, series shape and seed is on the GPU joins
    the running request's walk launches (its points are batched into the same launch); one with another
    seed runs in the same steps, in a launch of its own on another stream.  Each result is still the
    one-shot solve's, bit for bit."""
    wl = workloads.workload_sin_2d()
    ctx = grt.grt_create(wl["problem"], 0)
    server = grt.grt_server_create(0, mem_budget_bytes=512 << 20, step_trees=1 << 16)
    K, L, M = wl["K"], wl["L"], wl["M"]
    big = grt.grt_submit(server, ctx, wl["x"][:16], wl["t"][:16], np.full(16, 200_000, np.uint64), K, L, M, 1, 0)
    t0 = time.time()
    while grt.grt_server_stats(server)["steps"] < 2 and time.time() - t0 < 30:
        time.sleep(0.001)
    # small requests: the scheduler takes smallest remaining work first, so both fit in the next step
    # beside a range of the big request
    same = grt.grt_submit(server, ctx, wl["x"][16:20], wl["t"][16:20], np.full(4, 3000, np.uint64), K, L, M, 1, 16)
    other = grt.grt_submit(server, ctx, wl["x"][20:24], wl["t"][20:24], np.full(4, 3000, np.uint64), K, L, M, 2, 20)
    rb, rs, ro = (grt.grt_poll_ex(server, rid, -1) for rid in (big, same, other))
    stats = grt.grt_server_stats(server)
    assert rs["shared_launches"] >= 1 and rb["shared_launches"] >= 1 and stats["shared_launches"] >= 1
    assert ro["shared_steps"] >= 1 and rb["shared_steps"] >= 1
    for r, sl, seed in ((rb, slice(0, 16), 1), (rs, slice(16, 20), 1), (ro, slice(20, 24), 2)):
        n = sl.stop - sl.start
        ref = grt.grt_solve(ctx, wl["x"][sl], wl["t"][sl], r["ntrees_done"], K, L, M, seed, sl.start)
        assert np.array_equal(r["coef"], ref["coef"]) and np.array_equal(r["u"], ref["u"])
        assert not r["cancelled"] and np.all(r["status"] & grt.STATUS_SERIES_PARTIAL == 0) and n == len(r["u"])
    server.close()
    ctx.close()


def test_cancelled_request_ends_with_the_trees_binned_so_far(grt):
    """grt_cancel mid-request: every point that had not received all its trees ends with N_done (a
    multiple of 8192, below N) and SERIES_PARTIAL; its coefficients, standard errors and Pade value are
    grt_solve's with N = N_done, bit for bit, and agree with the FP64 oracle over those N_done trees.
    A request still waiting for admission ends with N_done = 0."""
    wl = workloads.workload_sin_2d()
    ctx = grt.grt_create(wl["problem"], 0)
    K, L, M = wl["K"], wl["L"], wl["M"]
    step = 1 << 16
    budget, cap = _min_budget(grt, step)
    server = grt.grt_server_create(0, mem_budget_bytes=budget, step_trees=step)
    nt = np.array([8 * 8192 + 5, 300_000, 1000, 500_000, 2 * 8192, 777_777], np.uint64)
    x, t = wl["x"][100:106], wl["t"][100:106]
    rid = grt.grt_submit(server, ctx, x, t, nt, K, L, M, 9, 100)
    # a second request with more points than the budget has rows left waits for admission
    nw = cap - len(nt) + 1
    rng = np.random.default_rng(3)
    waiting = grt.grt_submit(server, ctx, rng.uniform(-3.0, 3.0, (nw, 2)), rng.uniform(0.1, 1.0, nw),
                             np.full(nw, 8192, np.uint64), K, L, M, 9, 1000)
    t0 = time.time()
    while grt.grt_server_stats(server)["steps"] < 4 and time.time() - t0 < 30:
        time.sleep(0.0005)
    grt.grt_cancel(server, waiting)
    grt.grt_cancel(server, rid)
    r = grt.grt_poll_ex(server, rid, -1)
    w = grt.grt_poll_ex(server, waiting, -1)
    stats = grt.grt_server_stats(server)
    server.close()
    assert r["cancelled"] and w["cancelled"] and stats["cancelled"] == 2
    nd = r["ntrees_done"]
    partial = nd < nt
    assert partial.any() and np.all(nd <= nt)
    assert np.all(nd[partial] % 8192 == 0)
    assert np.all((r["status"] & grt.STATUS_SERIES_PARTIAL != 0) == partial)
    ref = grt.grt_solve(ctx, x, t, nd, K, L, M, 9, 100)
    assert np.array_equal(r["coef"], ref["coef"]) and np.array_equal(r["se"], ref["se"])
    assert np.array_equal(r["u"], ref["u"], equal_nan=True)
    assert np.array_equal(r["status"] & ~grt.STATUS_SERIES_PARTIAL, ref["status"])
    i = int(np.argmax(partial & (nd > 0))) if np.any(partial & (nd > 0)) else None
    if i is not None:
        from test_parity_gpu import _assert_fp32_parity

        o = oracle.solve(wl["problem"], x[i:i + 1], t[i:i + 1], nd[i:i + 1], K, L, M, 9, point_base=100 + i)
        gi = {k: r[k][i:i + 1] for k in ("u", "coef")}
        gi["status"] = r["status"][i:i + 1] & ~grt.STATUS_SERIES_PARTIAL
        _assert_fp32_parity(gi, o, nd[i:i + 1], L=L, M=M)
    assert np.all(w["ntrees_done"] == 0) and np.all(w["u"] == 0.0) and np.all(w["coef"] == 0.0)
    assert np.all(w["status"] & grt.STATUS_SERIES_PARTIAL)
    zero = grt.grt_solve(ctx, wl["x"][:1], wl["t"][:1], np.zeros(1, np.uint64), K, L, M, 9, 0)
    assert np.all((w["status"] & ~grt.STATUS_SERIES_PARTIAL) == zero["status"][0])
    ctx.close()
