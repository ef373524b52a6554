"""grt_solve_noalloc: the point solve for callers that cannot allocate device memory.

Such callers (an application whose own pool allocator has reserved the device
memory, or a latency-critical path where a possibly synchronising cudaMalloc is
not acceptable) get a solve whose whole work area is a fixed array the library
keeps on the device.
This file is collected last so that a run stopping at its first failure has
already run every other test; it also passes alone in a fresh process.
"""
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


def test_noalloc_matches_the_allocating_solve_on_two_calls(grt):
    torch = pytest.importorskip("torch")
    wl = workloads.subsample(workloads.workload_sin_2d(), 40, ntrees=6000)
    wl["ntrees"][3] = 0          # an empty point
    wl["ntrees"][7] = 9000       # a point spanning two binning chunks
    n, K, L, M = wl["x"].shape[0], wl["K"], wl["L"], wl["M"]
    ctx = grt.grt_create(wl["problem"], 0)
    ref = grt.grt_solve(ctx, wl["x"], wl["t"], wl["ntrees"], K, L, M, wl["seed"], 11)
    dev = torch.device("cuda:0")
    x = torch.from_numpy(wl["x"]).to(dev)
    t = torch.from_numpy(wl["t"]).to(dev)
    for call in range(2):  # the work area keeps the previous call's contents
        u = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
        coef = torch.full((n, K + 1), float("nan"), dtype=torch.float64, device=dev)
        se = torch.full((n, K + 1), float("nan"), dtype=torch.float64, device=dev)
        st = torch.full((n,), -1, dtype=torch.int32, device=dev)
        grt.grt_solve_noalloc(ctx, x, t, wl["ntrees"], K, L, M, wl["seed"], 11, u, coef, se, st)
        torch.cuda.synchronize()
        scale = np.maximum(np.abs(ref["u"]), np.abs(ref["coef"]).sum(axis=1))
        assert np.all(np.abs(u.cpu().numpy() - ref["u"]) <= 1e-12 * scale), call
        assert np.allclose(coef.cpu().numpy(), ref["coef"], rtol=1e-12, atol=1e-300), call
        assert np.allclose(se.cpu().numpy(), ref["se"], rtol=1e-12, atol=1e-300), call
        assert np.array_equal(st.cpu().numpy(), ref["status"]), call
    ctx.close()


def test_noalloc_at_its_limits_matches_the_allocating_solve(grt):
    """Exactly at both limits: 4096 points holding 524288 trees, most of them one-tree points (the
    most record padding, each point's records starting on a multiple of 4) plus points of 8193
    trees (two binning chunks each for 8193 trees: the most chunks), in two consecutive calls."""
    torch = pytest.importorskip("torch")
    n = grt.NOALLOC_MAX_POINTS
    nt = np.ones(n, np.uint64)
    nt[:63] = 8193
    nt[-1] += grt.NOALLOC_MAX_TREES - int(nt.sum())
    assert int(nt.sum()) == grt.NOALLOC_MAX_TREES and nt[-1] >= 1
    rng = np.random.default_rng(4)
    x = rng.uniform(-3.0, 3.0, size=(n, 2))
    t = rng.uniform(0.1, 1.0, size=n)
    pb = workloads.problem_sin_2d()
    K, L, M = 10, 5, 5
    ctx = grt.grt_create(pb, 0)
    ref = grt.grt_solve(ctx, x, t, nt, K, L, M, 21, 0)
    dev = torch.device("cuda:0")
    xd, td = torch.from_numpy(x).to(dev), torch.from_numpy(t).to(dev)
    for call in range(2):
        u = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
        coef = torch.full((n, K + 1), float("nan"), dtype=torch.float64, device=dev)
        st = torch.full((n,), -1, dtype=torch.int32, device=dev)
        grt.grt_solve_noalloc(ctx, xd, td, nt, K, L, M, 21, 0, u, coef, None, st)
        torch.cuda.synchronize()
        assert np.array_equal(coef.cpu().numpy(), ref["coef"]), call
        assert np.array_equal(u.cpu().numpy(), ref["u"], equal_nan=True), call
        assert np.array_equal(st.cpu().numpy(), ref["status"]), call
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_limits(grt):
    torch = pytest.importorskip("torch")
    ctx = grt.grt_create(workloads.problem_sin_2d(), 0)
    dev = torch.device("cuda:0")
    n = grt.NOALLOC_MAX_POINTS + 1
    x = torch.zeros((n, 2), dtype=torch.float64, device=dev)
    t = torch.ones(n, dtype=torch.float64, device=dev)
    u = torch.empty(n, dtype=torch.float64, device=dev)
    with pytest.raises(grt.GrtError, match="GRT_NOALLOC_MAX_POINTS"):
        grt.grt_solve_noalloc(ctx, x, t, np.full(n, 10, np.uint64), 10, 5, 5, 0, 0, u)
    with pytest.raises(grt.GrtError, match="GRT_NOALLOC_MAX_TREES"):
        grt.grt_solve_noalloc(ctx, x[:2], t[:2], [grt.NOALLOC_MAX_TREES, 1], 10, 5, 5, 0, 0, u[:2])
    ctx.close()
