"""Serving: continuous batching of point-solve requests (grt_server / grt_submit / grt_poll).

Each request's result must equal, bit for bit, the one-shot grt_solve of the
same points (same stream indices and seed) -- alone or in any mix of concurrent
requests, and however the scheduler split its trees over steps.
"""
import threading

import numpy as np
import pytest

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
    for s, r in zip(specs, results):
        ref = grt.grt_solve(ctxs[s["name"]], s["x"], s["t"], s["ntrees"], s["K"], s["L"], s["M"], s["seed"],
                            s["point_base"])
        assert np.array_equal(r["coef"], ref["coef"]), s["name"]
        assert np.array_equal(r["se"], ref["se"]), s["name"]
        assert np.array_equal(r["status"], ref["status"]), s["name"]
        assert np.array_equal(r["u"], ref["u"]) or np.allclose(r["u"], ref["u"], equal_nan=True, rtol=0, atol=0)
        assert r["latency_s"] >= 0.0
    server.close()
    for c in ctxs.values():
        c.close()


def test_admission_waits_for_memory(grt):
    wl = workloads.workload_sin_2d()
    ctx = grt.grt_create(wl["problem"], 0)
    # resident part of the budget: 1 MB = ~1365 chunk rows of 8192 trees; each request below
    # needs 20 points x 20 chunks = 400 rows, so at most three are admitted at a time
    step = 1 << 16
    budget = step * 9 + 64 * 1024 + 4096 * 80 + (1 << 20)
    server = grt.grt_server_create(0, mem_budget_bytes=budget, step_trees=step)
    nt = np.full(20, 20 * 8192, np.uint64)
    ids = []
    for k in range(12):
        sl = slice(k * 20, k * 20 + 20)
        ids.append(grt.grt_submit(server, ctx, wl["x"][sl], wl["t"][sl], nt, wl["K"], wl["L"], wl["M"], 0, k * 20))
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
    ref = grt.grt_solve(ctx, wl["x"][:240], wl["t"][:240], np.full(240, 20 * 8192, np.uint64), wl["K"], wl["L"],
                        wl["M"], 0)
    assert np.array_equal(np.concatenate([res[rid]["coef"] for rid in ids]), ref["coef"])
    server.close()
    ctx.close()


def test_errors_and_empty_requests(grt):
    wl = workloads.workload_sin_2d()
    ctx = grt.grt_create(wl["problem"], 0)
    with pytest.raises(grt.GrtError):
        grt.grt_server_create(0, mem_budget_bytes=1 << 20, step_trees=1 << 16)  # budget below the step buffers
    # 64 MB: ~86K resident chunk rows; a point of 2^31 - 1 trees needs 262144
    server = grt.grt_server_create(0, mem_budget_bytes=64 << 20, step_trees=1 << 16)
    rid = grt.grt_submit(server, ctx, np.zeros((0, 2)), np.zeros(0), np.zeros(0, np.uint64), 10, 5, 5, 0)
    r = grt.grt_poll(server, rid, 0)
    assert r is not None and r["u"].shape == (0,)
    with pytest.raises(grt.GrtError):
        grt.grt_submit(server, ctx, np.zeros((1, 2)), [1.0], [10], 10, 6, 5, 0)
    with pytest.raises(grt.GrtError):  # more resident state than the whole budget
        grt.grt_submit(server, ctx, np.zeros((1, 2)), [1.0], [2**31 - 1], 10, 5, 5, 0)
    rid = grt.grt_submit(server, ctx, np.zeros((3, 2)), [0.5, 1.0, 0.25], [20000, 1, 0], 10, 5, 5, 7)
    assert grt.grt_poll(server, rid, -1)["u"].shape == (3,)
    server.close()
    ctx.close()
