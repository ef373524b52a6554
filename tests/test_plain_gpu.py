"""The plain FP64 path (grt_solve_plain: one kernel launch per point) against the FP64 oracle.

The walk is the same FP64 node arithmetic on the same random streams as the oracle's; the
differences are the last-ulp differences of the two math libraries (exp, log, tanh, sin / cos)
and the order in which tree weights are added (per thread, warp butterfly, blocks).  Initial data
that change sign (the tanh product on its zero planes) make a weight's relative error grow near
the zeros, so the coefficients are held to 1e-11 of the mean |W| of each order, and the Pade value
to 1e-11 of max(|u|, sum |a_n|) (the Pade amplifies coefficient rounding by its condition number,
small at these points).
"""
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


def _check(g, o, nt, ctol=1e-11, rtol=1e-11):
    N = np.maximum(np.asarray(nt, float), 1.0)[:, None]
    scale_c = o["sa"] / N
    assert np.all(np.abs(g["coef"] - o["coef"]) <= ctol * scale_c + 1e-300), np.max(
        np.abs(g["coef"] - o["coef"]) / np.maximum(scale_c, 1e-300))
    se_ok = np.abs(g["se"] - o["se"]) <= 1e-9 * np.maximum(o["se"], 1e-300) + 1e-15 * scale_c
    assert np.all(se_ok)
    scale_u = np.maximum(np.abs(o["u"]), np.abs(o["coef"]).sum(axis=1))
    ok = np.abs(g["u"] - o["u"]) <= rtol * scale_u
    ok |= (np.asarray(o["status"]) & 3) != 0  # flagged Pade: compared through the coefficients above
    assert np.all(ok), (g["u"], o["u"])
    assert np.array_equal(g["status"] & 8, o["status"] & 8)


@pytest.mark.parametrize("name,npts,ntrees", [("kpp_1d", 16, 10_000), ("sin_2d", 12, 20_000), ("pdd_3d", 6, 8_000),
                                             ("var_coef_2d", 6, 6_000), ("drift_2d", 4, 3_000),
                                             ("uneven_2d", 8, 5_000)])
def test_plain_path_matches_the_oracle(grt, name, npts, ntrees):
    wl = workloads.subsample(workloads.WORKLOADS[name](), npts, ntrees=ntrees)
    pb = dict(wl["problem"], precision="fp64")
    ctx = grt.grt_create(wl["problem"], 0)  # the plain path walks in FP64 whatever the context's precision
    g = grt.grt_solve_plain(ctx, wl["x"], wl["t"], wl["ntrees"], wl["K"], wl["L"], wl["M"], wl["seed"], 5)
    ctx.close()
    o = oracle.solve(pb, wl["x"], wl["t"], wl["ntrees"], wl["K"], wl["L"], wl["M"], wl["seed"], point_base=5)
    _check(g, o, wl["ntrees"])


def test_plain_path_edge_budgets_and_grids(grt):
    """Budgets around the block size and a grid of many blocks whose threads walk several trees each."""
    pb = workloads.problem_sin_2d()
    nt = np.array([0, 1, 127, 128, 129, 4097, 300_000], np.uint64)
    x = np.linspace(-1.5, 1.5, 2 * nt.size).reshape(-1, 2)
    t = np.linspace(0.2, 1.0, nt.size)
    ctx = grt.grt_create(pb, 0)
    g = grt.grt_solve_plain(ctx, x, t, nt, 10, 5, 5, 3)
    again = grt.grt_solve_plain(ctx, x, t, nt, 10, 5, 5, 3)
    ctx.close()
    assert np.array_equal(g["coef"], again["coef"]) and np.array_equal(g["u"], again["u"], equal_nan=True)
    assert g["u"][0] == 0.0 and np.all(g["coef"][0] == 0.0)
    o = oracle.solve(dict(pb, precision="fp64"), x, t, nt, 10, 5, 5, 3)
    _check(g, o, nt)


def test_plain_path_agrees_with_the_batched_fp64_solve(grt):
    """One launch per point versus the persistent walk and the binning kernel on an FP64 context:
    the same trees, summed in another order."""
    wl = workloads.subsample(workloads.workload_kpp_1d(), 16)
    ctx = grt.grt_create(wl["problem"], 0)
    args = (wl["x"], wl["t"], wl["ntrees"], wl["K"], wl["L"], wl["M"], wl["seed"])
    a = grt.grt_solve_plain(ctx, *args)
    b = grt.grt_solve(ctx, *args)
    ctx.close()
    assert np.allclose(a["coef"], b["coef"], rtol=1e-12, atol=1e-15)
    assert np.allclose(a["u"], b["u"], rtol=1e-11, atol=1e-14)
    assert np.array_equal(a["status"], b["status"])


def test_plain_path_rejects_bad_arguments(grt):
    ctx = grt.grt_create(workloads.problem_sin_2d(), 0)
    with pytest.raises(grt.GrtError):
        grt.grt_solve_plain(ctx, np.zeros((1, 2)), [-1.0], [10], 10, 5, 5, 0)
    with pytest.raises(grt.GrtError):
        grt.grt_solve_plain(ctx, np.zeros((1, 2)), [1.0], [10], 10, 6, 5, 0)
    r = grt.grt_solve_plain(ctx, np.zeros((0, 2)), np.zeros(0), np.zeros(0, np.uint64), 10, 5, 5, 0)
    assert r["u"].shape == (0,)
    ctx.close()
