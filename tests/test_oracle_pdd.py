"""Pins of the PDD oracle stages (Sec. 3): not-a-knot spline, shifted-Laplacian solve,
Crank-Nicolson, and the decomposition itself.

  * spline: scipy's CubicSpline with bc_type="not-a-knot" (1-D) and FITPACK's
    interpolating RectBivariateSpline (s = 0, whose knots are the not-a-knot
    ones), and exact reproduction of a polynomial of degree 3 per variable;
  * the DST solve of (I - alpha Lap_h) x = r against a sparse direct solve;
  * Crank-Nicolson: a discrete Dirichlet eigenmode decays by exactly
    ((1 + alpha lam)/(1 - alpha lam))^n; with D = 0 the scheme is a
    second-order ODE integrator (error ratio ~4 when dt halves) against the
    closed forms of u' = u - u^3 and of u' = b2 u^2 / (t + t0);
  * decomposition: fed the global solution's own values on the interfaces,
    the independent subdomain solves reproduce the global solve to round-off;
  * the whole pipeline with exact heat-equation interface data converges to
    the closed-form solution as the grid, the steps and the nodes refine.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy import interpolate

from oracle import pdd


def test_spline_matches_scipy_not_a_knot():
    rng = np.random.default_rng(0)
    for nodes in (np.linspace(-1.0, 2.0, 9), np.sort(rng.uniform(0.0, 5.0, 12)), np.linspace(0.0, 1.0, 4)):
        y = rng.standard_normal(nodes.size)
        span = nodes[-1] - nodes[0]
        tq = np.concatenate([rng.uniform(nodes[0] - 0.1 * span, nodes[-1] + 0.1 * span, 40), nodes])
        W = pdd.spline_matrix(nodes, tq)
        ref = interpolate.CubicSpline(nodes, y, bc_type="not-a-knot")(tq)
        assert np.allclose(W @ y, ref, rtol=1e-12, atol=1e-12 * np.abs(y).max())


def test_spline_2d_matches_fitpack_interpolant():
    rng = np.random.default_rng(1)
    xa, ya = np.linspace(0.0, 4.0, 9), np.linspace(-1.0, 1.0, 6)
    V = rng.standard_normal((9, 6))
    tx, ty = np.sort(rng.uniform(0.0, 4.0, 13)), np.sort(rng.uniform(-1.0, 1.0, 7))
    ours = pdd.spline_tensor(V, [xa, ya], [tx, ty])
    ref = interpolate.RectBivariateSpline(xa, ya, V, kx=3, ky=3, s=0)(tx, ty, grid=True)
    assert np.allclose(ours, ref, rtol=1e-11, atol=1e-11)


def test_tensor_spline_reproduces_cubics():
    rng = np.random.default_rng(2)
    axes = [np.sort(rng.uniform(0.0, 2.0, 7)), np.linspace(-1.0, 1.0, 5), np.linspace(0.0, 1.0, 4)]
    p = lambda x, y, t: (1.0 + x - 2.0 * y + 0.5 * t) ** 3 + x * x * y * t - 3.0 * t ** 3 * y ** 2
    G = np.meshgrid(*axes, indexing="ij")
    tg = [rng.uniform(0.0, 2.0, 6), rng.uniform(-1.0, 1.0, 5), rng.uniform(0.0, 1.0, 3)]
    T = np.meshgrid(*tg, indexing="ij")
    out = pdd.spline_tensor(p(*G), axes, tg)
    assert np.allclose(out, p(*T), rtol=1e-11, atol=1e-10)


@pytest.mark.parametrize("shape", [(17,), (7, 9), (5, 4, 6)])
def test_shifted_solve_against_sparse_direct(shape):
    rng = np.random.default_rng(3)
    h = [0.3, 0.2, 0.45][: len(shape)]
    alpha = 0.07
    r = rng.standard_normal(shape)
    Lap = None
    for a, (m, ha) in enumerate(zip(shape, h)):
        T = sp.diags([np.ones(m - 1), -2.0 * np.ones(m), np.ones(m - 1)], [-1, 0, 1]) / (ha * ha)
        term = sp.identity(1)
        for b, mb in enumerate(shape):
            term = sp.kron(term, T if b == a else sp.identity(mb))
        Lap = term if Lap is None else Lap + term
    A = sp.identity(int(np.prod(shape))) - alpha * Lap
    ref = spla.spsolve(A.tocsc(), r.ravel()).reshape(shape)
    assert np.allclose(pdd.solve_shifted(r, alpha, h), ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_crank_nicolson_discrete_eigenmode(dim):
    L = [2.0, 3.0, 1.5][:dim]
    m = [15, 11, 9][:dim]
    coords = [np.linspace(-La / 2, La / 2, ma + 2) for La, ma in zip(L, m)]
    w = [math.pi / La for La in L]
    pb = dict(dim=dim, D=0.8, f_coef=[0.0], u0=("cos_prod", (0.0, 1.3) + tuple(w)))
    dt, nsteps = 0.013, 25
    zero = lambda n: np.zeros([ma + 2 for ma in m])
    U = pdd.cn_box(pb, coords, zero, dt, nsteps)
    h = [c[1] - c[0] for c in coords]
    lam = sum(-4.0 / (ha * ha) * math.sin(math.pi / (2.0 * (ma + 1))) ** 2 for ha, ma in zip(h, m))
    alpha = 0.5 * dt * pb["D"]
    rho = (1.0 + alpha * lam) / (1.0 - alpha * lam)
    X = np.meshgrid(*[c[1:-1] for c in coords], indexing="ij")
    g0 = 1.3 * np.prod([np.cos(wi * xi) for wi, xi in zip(w, X)], axis=0)
    assert np.allclose(U[tuple(slice(1, -1) for _ in range(dim))], rho ** nsteps * g0, rtol=1e-12, atol=1e-13)


def _ode_error(pb, exact, T, nsteps):
    coords = [np.linspace(0.0, 1.0, 4)]
    ring = lambda n: np.zeros(4)
    U = pdd.cn_box(pb, coords, ring, T / nsteps, nsteps)
    return abs(U[1] - exact)


@pytest.mark.parametrize("case", ["u-u3", "b2/(t+t0) u^2"])
def test_crank_nicolson_reaction_is_second_order(case):
    c0, T = 0.4, 1.2
    if case == "u-u3":
        pb = dict(dim=1, D=0.0, f_coef=[0.0, 1.0, 0.0, -1.0], u0=("const", (c0,)))
        e = math.exp(T)
        exact = c0 * e / math.sqrt(1.0 + c0 * c0 * (e * e - 1.0))
    else:
        b2, t0 = -1.0, 0.1
        pb = dict(dim=1, D=0.0, f_coef=[0.0, 0.0, b2], u0=("const", (c0,)),
                  coef=("gauss_over_t", (0, 0, 0, 0, 0, 0, t0), [2]))
        exact = 1.0 / (1.0 / c0 - b2 * math.log((T + t0) / t0))
    errs = [_ode_error(pb, exact, T, n) for n in (40, 80, 160)]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.4 < r1 < 4.6 and 3.4 < r2 < 4.6, errs


def _grid(dim, sub, cells, nodes, t_nodes, T, nsteps, lo=0.0, hi=None):
    hi = hi if hi is not None else [float(s) for s in sub]
    return dict(dim=dim, lo=[lo] * dim, hi=list(hi), sub=list(sub), cells=[cells] * dim, nodes=[nodes] * dim,
                t_nodes=t_nodes, T=T, nsteps=nsteps)


@pytest.mark.parametrize("dim,sub", [(1, [4]), (2, [3, 2]), (3, [2, 2, 2])])
def test_subdomains_reproduce_the_global_solve(dim, sub):
    g = _grid(dim, sub, 6, 7, 4, 0.6, 12)
    pb = dict(dim=dim, D=0.3, f_coef=[0.1, 1.0, 0.0, -1.0], u0=("tanh_prod", (0.2, 0.8, 1.0, 1.1, 0.9)),
              coef=("gauss", (0.3, 0.2, 0.1, 1.0, 1.0, 1.0), [3]))
    x, t = pdd.points(g)
    # nodal data: a smooth made-up field (the check needs only consistent outer faces)
    u_nodes = 0.3 * np.sin(x.sum(axis=1)) + 0.1 * t
    P = pdd.plane_values(pb, g, u_nodes)
    U_glob, levels = pdd.global_solve(pb, g, plane_data=P, history=True)
    P_exact = pdd.planes_from_levels(g, levels)
    U_pdd = pdd.pdd_solve(pb, g, None, plane_data=P_exact)
    assert np.allclose(U_pdd, U_glob, rtol=0, atol=1e-13 * np.abs(U_glob).max())


def test_points_layout():
    g = _grid(3, [4, 4, 4], 4, 17, 4, 1.0, 8)
    x, t = pdd.points(g)
    assert x.shape == (15 * 17 * 17 * 4, 3) and t.shape == (x.shape[0],)
    assert np.allclose(x[:289, 0], 0.0) and np.allclose(x[289 * 4: 289 * 5, 0], 1.0)
    assert np.allclose(t[:289], 0.25) and np.allclose(t[289: 578], 0.5)
    assert np.allclose(x[:17, 2], np.linspace(0.0, 4.0, 17)) and np.allclose(x[:17, 1], 0.0)


def test_pipeline_with_exact_interface_data_converges_to_heat_solution():
    # f = 0, g Gaussian: the exact solution is the heat-kernel convolution, fed at the nodal points
    def run(cells, nodes, nsteps):
        g = _grid(2, [3, 3], cells, nodes, 4, 0.5, nsteps, lo=-1.5, hi=[1.5, 1.5])
        pb = dict(dim=2, D=0.4, f_coef=[0.0], u0=("gauss", (0.1, 1.0, 0.6, 0.2, -0.1)))
        x, t = pdd.points(g)
        v = 0.36 + 2.0 * 0.4 * t
        exact = lambda X, tt: 0.1 + (0.36 / (0.36 + 0.8 * tt)) * np.exp(
            -((X[..., 0] - 0.2) ** 2 + (X[..., 1] + 0.1) ** 2) / (2.0 * (0.36 + 0.8 * tt)))
        u_nodes = exact(x, t)
        U = pdd.pdd_solve(pb, g, u_nodes)
        c = np.linspace(-1.5, 1.5, 3 * cells + 1)
        X = np.stack(np.meshgrid(c, c, indexing="ij"), axis=-1)
        return np.abs(U - exact(X, 0.5)).max()

    e1, e2 = run(6, 9, 20), run(12, 17, 40)
    assert e1 < 5e-3 and e2 < e1 / 3.0, (e1, e2)
