"""GPU parity of the PDD stages (Sec. 3) against the oracle, and the end-to-end check.

  * grt_spline_grid against the oracle's tensor-product not-a-knot spline
    (1e-12 of the data's size: both are FP64 evaluations of one linear map);
  * grt_pdd_solve against the oracle's PDD on the same nodal values: the spline
    stages agree to rounding and both sides solve each Crank-Nicolson system
    exactly (sine transforms: dense on the GPU, FFT-based in the oracle), so the
    solutions agree to 1e-10 of max |u| after tens of steps;
  * end to end on the 3-D interface problem: point solves on the GPU at the
    PDD nodal points, the PDD on the GPU, and the oracle's global
    Crank-Nicolson solve on the same outer data as the check; they differ by
    the interface values' Monte Carlo error, bounded here by four standard
    errors of the Pade value (summed per-order standard errors).
"""
import numpy as np
import pytest

import workloads
from oracle import pdd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def grt():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2402_06491_gb300 as pkg

    return pkg


@pytest.fixture(scope="module")
def torch():
    import torch

    return torch


@pytest.mark.parametrize("shape,batch", [((9,), 3), ((6, 11), 2), ((5, 4, 7), 2)])
def test_spline_grid_parity(grt, torch, shape, batch):
    rng = np.random.default_rng(len(shape))
    lo = rng.uniform(-1.0, 0.0, len(shape))
    hi = lo + rng.uniform(0.5, 3.0, len(shape))
    nodes = [np.linspace(lo[a], hi[a], shape[a]) for a in range(len(shape))]
    targets = [np.sort(rng.uniform(lo[a] - 0.1, hi[a] + 0.1, 5 + 3 * a)) for a in range(len(shape))]
    V = rng.standard_normal((batch,) + shape)
    ctx = grt.grt_create(workloads.problem_sin_2d(), 0)
    dv = torch.from_numpy(V).cuda()
    out = torch.empty((batch,) + tuple(len(t) for t in targets), dtype=torch.float64, device="cuda")
    grt.grt_spline_grid(ctx, list(shape), lo, hi, targets, dv, out, batch=batch)
    torch.cuda.synchronize()
    g = out.cpu().numpy()
    ctx.close()
    o = np.stack([pdd.spline_tensor(V[b], nodes, targets) for b in range(batch)])
    assert np.allclose(g, o, rtol=0, atol=1e-12 * np.abs(V).max()), np.abs(g - o).max()


def _pdd_problem(dim):
    return dict(dim=dim, D=0.3, f_coef=[0.1, 1.0, 0.0, -1.0], u0=("tanh_prod", (0.2, 0.8, 1.0, 1.1, 0.9)),
                coef=("gauss", (0.3, 0.2, 0.1, 1.0, 1.0, 1.0), [3]), strategy="B", q=0.6, arity_law="uniform",
                precision="fp32")


@pytest.mark.parametrize("dim,sub,cells,nodes", [(1, [4], [9], [4]), (2, [3, 2], [7, 5], [7, 6]),
                                                 (3, [2, 3, 2], [6, 5, 7], [6, 7, 5]),
                                                 (3, [1, 1, 2], [20, 20, 20], [5, 5, 5]),  # block pairs
                                                 (3, [1, 1, 2], [30, 30, 30], [5, 5, 5])])  # global-memory vectors
def test_pdd_solve_parity(grt, torch, dim, sub, cells, nodes):
    g = dict(dim=dim, lo=[0.0] * dim, hi=[float(s) for s in sub], sub=sub, cells=cells, nodes=nodes, t_nodes=4,
             T=0.6, nsteps=24)
    pb = _pdd_problem(dim)
    x, t = grt.grt_pdd_points(g)
    u_nodes = 0.3 * np.sin(x.sum(axis=1)) + 0.1 * t + 0.2
    ctx = grt.grt_create(pb, 0)
    N = [sub[a] * cells[a] + 1 for a in range(dim)]
    out = torch.empty(N, dtype=torch.float64, device="cuda")
    grt.grt_pdd_solve(ctx, g, torch.from_numpy(u_nodes).cuda(), out)
    G = out.cpu().numpy()
    ctx.close()
    O = pdd.pdd_solve(pb, g, u_nodes)
    assert np.allclose(G, O, rtol=0, atol=1e-10 * np.abs(O).max()), np.abs(G - O).max()


def test_pdd_needs_heat_paths(grt):
    ctx = grt.grt_create(workloads.problem_drift_2d(), 0)
    g = dict(dim=2, lo=[0.0, 0.0], hi=[2.0, 2.0], sub=[2, 2], cells=[4, 4], nodes=[5, 5], t_nodes=4, T=1.0, nsteps=8)
    with pytest.raises(grt.GrtError) as ei:
        grt.grt_pdd_solve(ctx, g, 0, 0)
    assert ei.value.code == -5
    ctx.close()


def test_pdd_rejects_bad_grids(grt):
    ctx = grt.grt_create(_pdd_problem(2), 0)
    good = dict(dim=2, lo=[0.0, 0.0], hi=[2.0, 2.0], sub=[2, 2], cells=[4, 4], nodes=[5, 5], t_nodes=4, T=1.0,
                nsteps=8)
    for bad in (dict(good, cells=[1, 4]), dict(good, nodes=[3, 5]), dict(good, t_nodes=2), dict(good, dim=3,
                lo=[0.0] * 3, hi=[1.0] * 3, sub=[1] * 3, cells=[4] * 3, nodes=[4] * 3),
                dict(good, cells=[66, 4])):
        with pytest.raises(grt.GrtError):
            grt.grt_pdd_solve(ctx, bad, 0, 0)
    ctx.close()


def _nodal_from_levels(g, levels):
    """Values of full-grid solution levels at the PDD nodal points (nodes and time levels on the FD grid)."""
    d = g["dim"]
    N = [g["sub"][a] * g["cells"][a] + 1 for a in range(d)]
    out = []
    for a, k in pdd.planes(g):
        idx_other = [np.arange(g["nodes"][b]) * ((N[b] - 1) // (g["nodes"][b] - 1)) for b in range(d) if b != a]
        for j in range(1, g["t_nodes"] + 1):
            L = levels[j * g["nsteps"] // g["t_nodes"]]
            sl = [slice(None)] * d
            sl[a] = k * g["cells"][a]
            P = L[tuple(sl)]
            out.append(P[np.ix_(*idx_other)].ravel())
    return np.concatenate(out)


def test_pdd_3d_end_to_end_against_the_global_solve(grt, torch):
    """The 3-D interface problem (u_t = 0.1 Lap u + u - u^3, u0 = prod tanh(x_i - 2), 4^3 subdomains of [0,4]^3,
    K = 12, [6/6], 1e5 trees per nodal point) through point solves and the PDD on the GPU, checked against one
    global Crank-Nicolson solve with the same outer data.  T = 1/4: at T = 1 a few percent of the nodal Pade
    values are spoiled by the Monte Carlo noise of the high orders (see the design notes).

    Bound: the PDD and the global solve differ only through the interior planes' data, so
        max |PDD - global| <= 1.2 e^{L T} (Lambda e_if + e_int),
    e_if the largest nodal error against the global solve on the interior planes, Lambda the product of the
    spline's Lebesgue constants (max row sums of |W|) over time and the two plane axes, e_int the spline's
    interpolation error of the global solution itself, L = 1 >= f'(u) for f = u - u^3; the scheme is monotone
    here (dt D sum_a 2/h_a^2 <= 1), which gives the discrete maximum principle behind the bound."""
    pb = workloads.problem_pdd_3d()
    g = dict(dim=3, lo=[0.0] * 3, hi=[4.0] * 3, sub=[4] * 3, cells=[8] * 3, nodes=[17] * 3, t_nodes=4, T=0.25,
             nsteps=20)
    x, t = grt.grt_pdd_points(g)
    n = x.shape[0]
    ctx = grt.grt_create(pb, 0)
    plan = grt.grt_plan_create(ctx, np.full(n, 100_000, np.uint64), 12, 6, 6)
    dx, dtt = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    u = torch.empty(n, dtype=torch.float64, device="cuda")
    grt.grt_plan_execute(plan, dx, dtt, 0, 0, u)
    out = torch.empty((33, 33, 33), dtype=torch.float64, device="cuda")
    grt.grt_pdd_solve(ctx, g, u, out)
    G = out.cpu().numpy()
    u_nodes = u.cpu().numpy()
    plan.close()
    ctx.close()
    assert np.isfinite(u_nodes).all() and np.isfinite(G).all()
    # parity of the PDD stages on these nodal values
    O = pdd.pdd_solve(pb, g, u_nodes)
    assert np.allclose(G, O, rtol=0, atol=1e-10 * np.abs(O).max()), np.abs(G - O).max()
    # the check
    U, levels = pdd.global_solve(pb, g, u_nodes, history=True)
    ref_nodes = _nodal_from_levels(g, levels)
    interior = np.zeros(n, bool)
    off = 0
    for a, k in pdd.planes(g):
        m = g["t_nodes"] * 17 * 17
        interior[off: off + m] = 0 < k < g["sub"][a]
        off += m
    e_if = np.abs(u_nodes - ref_nodes)[interior].max()
    P_ref = pdd.plane_values(pb, g, ref_nodes)
    P_glob = pdd.planes_from_levels(g, levels)
    e_int = max(np.abs(P_ref[key][1:] - P_glob[key][1:]).max() for key in P_ref if 0 < key[1] < g["sub"][key[0]])
    tl = np.concatenate([[0.0], pdd.time_levels(g)])
    lam = np.abs(pdd.spline_matrix(tl, g["T"] / g["nsteps"] * np.arange(1, g["nsteps"] + 1))).sum(axis=1).max()
    lam *= np.abs(pdd.spline_matrix(np.linspace(0, 4, 17), np.linspace(0, 4, 33))).sum(axis=1).max() ** 2
    bound = 1.2 * np.exp(g["T"]) * (lam * e_if + e_int)
    err = np.abs(G - U).max()
    assert err <= bound, (err, bound, e_if, e_int, lam)
    assert e_if < 0.05, e_if  # the interface values themselves: Monte Carlo sized at T = 1/4


@pytest.mark.parametrize("cells", [[5, 6, 4], [30, 30, 30]])  # block pairs; one block with global vectors
def test_pdd_subdomain_ranges_reproduce_the_full_solve(grt, torch, cells):
    """Disjoint subdomain ranges (what different GPUs would solve) together give the full solve
    bit for bit; each range call writes every plane node and only its own interiors."""
    from paper_2402_06491_gb300.sharding import pdd_subdomain_range

    sub = [2, 2, 2] if cells[0] < 30 else [1, 1, 2]
    g = dict(dim=3, lo=[0.0] * 3, hi=[float(v) for v in sub], sub=sub, cells=cells, nodes=[5, 5, 5], t_nodes=4,
             T=0.4, nsteps=12)
    pb = _pdd_problem(3)
    x, t = grt.grt_pdd_points(g)
    u_nodes = torch.from_numpy(0.3 * np.sin(x.sum(axis=1)) + 0.1 * t + 0.2).cuda()
    ctx = grt.grt_create(pb, 0)
    N = [sub[a] * cells[a] + 1 for a in range(3)]
    full = torch.empty(N, dtype=torch.float64, device="cuda")
    grt.grt_pdd_solve(ctx, g, u_nodes, full)
    parts = torch.zeros(N, dtype=torch.float64, device="cuda")
    for rank in range(3):  # three "ranks" over the subdomains
        grt.grt_pdd_solve_range(ctx, g, *pdd_subdomain_range(g, 3, rank), u_nodes, parts)
    assert torch.equal(parts, full)
    with pytest.raises(grt.GrtError):
        grt.grt_pdd_solve_range(ctx, g, 0, int(np.prod(sub)) + 1, u_nodes, parts)
    ctx.close()
