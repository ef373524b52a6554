"""FP64 CPU oracle of the probabilistic-domain-decomposition stages after the point solve.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU arms may import this module.  It shares no code with the
product library: its own spline, its own finite-difference scheme, its own
initial data and coefficient profiles, written with numpy / scipy.

The PDD algorithm (Sec. 3, text around Fig. sketch_algorithm):
  1. Probabilistic part: the solution at nodal points of the interfaces
     (here: every grid plane that bounds a subdomain, including the outer
     faces of the box, whose values are the probabilistic artificial
     Dirichlet data the text after Example 4 describes).
  2. Interpolation: a tensor product of not-a-knot cubic splines through
     uniformly spaced nodal points on each plane (Sec. 3, "Interpolation"),
     here in the plane's coordinates and in time.
  3. Local solver: each subdomain is solved independently by Crank-Nicolson
     finite differences with the interpolated Dirichlet data (Sec. 3,
     "Local solver"; Example 4 uses Crank-Nicolson).

Readings where the paper is silent (also listed in the design notes):
  * the reaction term is advanced by a linearly implicit Crank-Nicolson:
    the diffusion is averaged over t_n and t_{n+1}, the reaction is taken
    at t_{n+1/2} on the extrapolation u* = (3 u^n - u^{n-1}) / 2 (u* = u^0
    on the first step), which keeps second order without a nonlinear solve;
  * the time direction of the spline uses the exact initial data at t = 0
    plus the probabilistic levels t_j = T j / t_nodes, j = 1..t_nodes, and
    the Dirichlet data at t_0 = 0 are the initial data themselves;
  * a node on several planes (an edge) takes the value of the plane of the
    lowest axis.
The linear system (I - dt/2 D Lap_h) x = r of each step is solved exactly
with the orthonormal type-I discrete sine transform, which diagonalises the
Dirichlet Laplacian of a box; the paper's banded LU gives the same solution.

Grid description (a dict):
  dim, lo[dim], hi[dim], sub[dim] subdomains per axis, cells[dim] finite-
  difference cells per subdomain per axis, nodes[dim] spline nodal points per
  axis on each plane (uniform, both ends included), t_nodes probabilistic
  time levels, T final time, nsteps Crank-Nicolson steps.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import fft


# ---------------------------------------------------------------------------
# problem pieces (own numpy versions: u0, coefficient profiles, f)
# ---------------------------------------------------------------------------
def u0_grid(pb: dict, X: list) -> np.ndarray:
    """Initial data g on a grid given by broadcastable coordinate arrays X[i]."""
    kind, p = pb["u0"]
    p = list(p) + [0.0] * (8 - len(p))
    d = pb["dim"]
    if kind == "const":
        return np.broadcast_to(np.float64(p[0]), np.broadcast_shapes(*[np.shape(x) for x in X])).copy()
    if kind == "gauss":
        r2 = sum((X[i] - p[3 + i]) ** 2 for i in range(d))
        return p[0] + p[1] * np.exp(-r2 / (2.0 * p[2] * p[2]))
    if kind == "cos_prod":
        pr = 1.0
        for i in range(d):
            pr = pr * np.cos(p[2 + i] * X[i])
        return p[0] + p[1] * pr
    if kind == "tanh_prod":
        pr = 1.0
        for i in range(d):
            pr = pr * np.tanh(X[i] - p[2 + i])
        return p[0] + p[1] * pr
    if kind == "logistic":
        return p[0] + p[1] / (1.0 + np.exp(-(X[0] - p[2]) / p[3]))
    if kind == "gauss_axes":
        r = sum(p[2 + i] * (X[i] - p[5 + i]) ** 2 for i in range(d))
        return p[0] + p[1] * np.exp(-r)
    if kind == "quadratic":
        return p[0] + sum(p[1 + i] * X[i] + p[4 + i] * X[i] ** 2 for i in range(d))
    raise ValueError(kind)


def f_grid(pb: dict, X: list, t: float, u: np.ndarray) -> np.ndarray:
    """f(u, x, t) = sum_k c_k(x, t) u^k, c_k = b_k gamma(x, t) for the masked powers (Eq. nonlinear_new)."""
    coef = pb["f_coef"]
    gamma = None
    powers = ()
    if "coef" in pb:
        kind, cp, powers = pb["coef"]
        cp = list(cp) + [0.0] * (8 - len(cp))
        r = sum(cp[i] * (X[i] - cp[3 + i]) ** 2 for i in range(pb["dim"]))
        gamma = np.exp(-r)
        if kind == "gauss_over_t":
            gamma = gamma / (t + cp[6])
    out = np.zeros_like(u)
    for k, b in enumerate(coef):
        if b == 0.0:
            continue
        term = b * u ** k
        if gamma is not None and k in powers:
            term = term * gamma
        out = out + term
    return out


# ---------------------------------------------------------------------------
# not-a-knot cubic spline (Sec. 3, Interpolation)
# ---------------------------------------------------------------------------
def spline_matrix(nodes, targets) -> np.ndarray:
    """W with W @ y = s(targets), s the not-a-knot cubic spline through (nodes, y).

    Textbook construction on the second derivatives M_i = s''(x_i):
      interior rows  h_{i-1} M_{i-1} + 2 (h_{i-1} + h_i) M_i + h_i M_{i+1} = 6 (d_i - d_{i-1}),
                     d_i = (y_{i+1} - y_i) / h_i;
      not-a-knot     s''' continuous at x_1 and x_{n-2}:
                     (M_1 - M_0)/h_0 = (M_2 - M_1)/h_1, likewise at the right end;
    then on [x_i, x_{i+1}], with A = (x_{i+1} - x)/h_i, B = 1 - A,
      s(x) = A y_i + B y_{i+1} + ((A^3 - A) M_i + (B^3 - B) M_{i+1}) h_i^2 / 6,
    extended by the end cubics outside [x_0, x_{n-1}].  Solved for every unit
    data vector at once with a dense LU (numpy.linalg.solve); needs n >= 4.
    """
    x = np.asarray(nodes, float)
    n = x.size
    if n < 4:
        raise ValueError("not-a-knot needs at least 4 nodes")
    h = np.diff(x)
    A = np.zeros((n, n))
    R = np.zeros((n, n))  # right-hand side as a linear map of y
    A[0, 0], A[0, 1], A[0, 2] = h[1], -(h[0] + h[1]), h[0]
    A[n - 1, n - 3], A[n - 1, n - 2], A[n - 1, n - 1] = h[n - 2], -(h[n - 3] + h[n - 2]), h[n - 3]
    for i in range(1, n - 1):
        A[i, i - 1] = h[i - 1]
        A[i, i] = 2.0 * (h[i - 1] + h[i])
        A[i, i + 1] = h[i]
        R[i, i + 1] += 6.0 / h[i]
        R[i, i] -= 6.0 / h[i] + 6.0 / h[i - 1]
        R[i, i - 1] += 6.0 / h[i - 1]
    Mmap = np.linalg.solve(A, R)  # M = Mmap @ y
    tq = np.asarray(targets, float)
    W = np.zeros((tq.size, n))
    for r, xt in enumerate(tq):
        i = int(np.searchsorted(x, xt, side="right")) - 1
        i = min(max(i, 0), n - 2)
        hi = h[i]
        a = (x[i + 1] - xt) / hi
        b = 1.0 - a
        W[r, i] += a
        W[r, i + 1] += b
        W[r] += ((a ** 3 - a) * Mmap[i] + (b ** 3 - b) * Mmap[i + 1]) * hi * hi / 6.0
    return W


def spline_tensor(values: np.ndarray, node_axes: list, target_axes: list) -> np.ndarray:
    """Tensor-product not-a-knot spline of values on the grid node_axes, at the grid target_axes.

    The tensor-product interpolant is obtained by interpolating along one axis
    at a time (it is the unique element of the tensor-product spline space
    through the data, and each 1-D pass is linear); trailing axes of `values`
    beyond len(node_axes) are carried along.
    """
    out = np.asarray(values, float)
    for ax, (nd, tg) in enumerate(zip(node_axes, target_axes)):
        W = spline_matrix(nd, tg)
        out = np.moveaxis(np.tensordot(W, np.moveaxis(out, ax, 0), axes=(1, 0)), 0, ax)
    return out


# ---------------------------------------------------------------------------
# Crank-Nicolson on a box with Dirichlet data (Sec. 3, Local solver)
# ---------------------------------------------------------------------------
def dirichlet_eigs(m: list, h: list) -> np.ndarray:
    """Eigenvalues of the zero-Dirichlet 2nd-order Laplacian on an m[0] x ... interior grid."""
    lam = 0.0
    for a, (ma, ha) in enumerate(zip(m, h)):
        k = np.arange(1, ma + 1, dtype=float)
        la = -4.0 / (ha * ha) * np.sin(np.pi * k / (2.0 * (ma + 1))) ** 2
        shape = [1] * len(m)
        shape[a] = ma
        lam = lam + la.reshape(shape)
    return np.asarray(lam, float)


def solve_shifted(r: np.ndarray, alpha: float, h: list) -> np.ndarray:
    """x with (I - alpha Lap_h) x = r, zero Dirichlet ring, by the orthonormal DST-I."""
    lam = dirichlet_eigs(list(r.shape), h)
    return fft.idstn(fft.dstn(r, type=1, norm="ortho") / (1.0 - alpha * lam), type=1, norm="ortho")


def laplacian_full(U: np.ndarray, h: list) -> np.ndarray:
    """Second-order Laplacian at the interior nodes of a grid that includes its Dirichlet ring."""
    d = U.ndim
    inner = tuple(slice(1, -1) for _ in range(d))
    out = np.zeros(tuple(s - 2 for s in U.shape))
    for a in range(d):
        lo = list(inner)
        hi = list(inner)
        lo[a] = slice(0, -2)
        hi[a] = slice(2, None)
        out += (U[tuple(lo)] - 2.0 * U[inner] + U[tuple(hi)]) / (h[a] * h[a])
    return out


def cn_box(pb: dict, coords: list, ring, dt: float, nsteps: int, history: bool = False):
    """Crank-Nicolson of u_t = D Lap u + f(u, x, t) on a box.

    coords[a]: node coordinates along axis a, ring included (uniform spacing).
    ring(n) -> full array (ring included) whose ring holds the Dirichlet data at t_n
    (its interior is ignored); ring(0)'s interior is not used either: the initial
    interior is g at the nodes.
    Step n -> n+1 (reading: linearly implicit CN, reaction at t_{n+1/2} on
    u* = (3 u^n - u^{n-1})/2, u* = u^0 on the first step):
      (I - dt/2 D Lap_h) u^{n+1} = u^n + dt/2 D Lap_h u^n + dt/2 D (ring part of Lap_h at t_{n+1})
                                   + dt f(u*, x, t_{n+1/2}).
    Returns the full array at t_N (ring from ring(N)), and the list of all levels if history.
    """
    d = len(coords)
    h = [float(c[1] - c[0]) for c in coords]
    X = np.meshgrid(*coords, indexing="ij")
    inner = tuple(slice(1, -1) for _ in range(d))
    Xi = [x[inner] for x in X]
    D = float(pb["D"])
    alpha = 0.5 * dt * D
    U = np.array(ring(0), float)
    U[inner] = u0_grid(pb, Xi)
    prev = U[inner].copy()
    levels = [U.copy()] if history else None
    for n in range(nsteps):
        cur = U[inner].copy()
        ustar = cur if n == 0 else 1.5 * cur - 0.5 * prev
        nxt_ring = np.array(ring(n + 1), float)
        zero_inner = nxt_ring.copy()
        zero_inner[inner] = 0.0
        rhs = cur + alpha * laplacian_full(U, h) + alpha * laplacian_full(zero_inner, h) \
            + dt * f_grid(pb, Xi, (n + 0.5) * dt, ustar)
        new = solve_shifted(rhs, alpha, h)
        prev = cur
        U = nxt_ring
        U[inner] = new
        if history:
            levels.append(U.copy())
    return (U, levels) if history else U


# ---------------------------------------------------------------------------
# the PDD pipeline
# ---------------------------------------------------------------------------
def _axes(g):
    d = g["dim"]
    N = [g["sub"][a] * g["cells"][a] + 1 for a in range(d)]
    coords = [np.linspace(g["lo"][a], g["hi"][a], N[a]) for a in range(d)]
    return N, coords


def planes(g) -> list:
    """(axis, index) of every plane bounding a subdomain, outer faces included, axis-major."""
    return [(a, k) for a in range(g["dim"]) for k in range(g["sub"][a] + 1)]


def plane_nodes(g, a) -> list:
    """Spline nodal coordinates along the in-plane axes (ascending axis order) of an axis-a plane."""
    return [np.linspace(g["lo"][b], g["hi"][b], g["nodes"][b]) for b in range(g["dim"]) if b != a]


def time_levels(g) -> np.ndarray:
    return g["T"] * np.arange(1, g["t_nodes"] + 1) / g["t_nodes"]


def points(g):
    """The probabilistic nodal points (x [n, dim], t [n]) in the order the PDD stage reads them:
    planes axis-major, then time level, then in-plane nodes (row-major, ascending axis)."""
    d = g["dim"]
    xs, ts = [], []
    for a, k in planes(g):
        pa = g["lo"][a] + k * (g["hi"][a] - g["lo"][a]) / g["sub"][a]
        nodes = plane_nodes(g, a)
        grids = np.meshgrid(*nodes, indexing="ij") if nodes else []
        m = int(np.prod([len(v) for v in nodes])) if nodes else 1
        for tj in time_levels(g):
            x = np.empty((m, d))
            x[:, a] = pa
            col = 0
            for b in range(d):
                if b != a:
                    x[:, b] = grids[col].ravel()
                    col += 1
            xs.append(x)
            ts.append(np.full(m, tj))
    return np.concatenate(xs), np.concatenate(ts)


def plane_values(pb: dict, g, u_nodes: np.ndarray) -> dict:
    """Spline every plane to the finite-difference nodes at t_1..t_N: {(a, k): [nsteps+1][in-plane FD nodes]}.
    Level 0 is the initial data at the FD nodes."""
    d = g["dim"]
    N, coords = _axes(g)
    dt = g["T"] / g["nsteps"]
    t_targets = dt * np.arange(1, g["nsteps"] + 1)
    t_nodes = np.concatenate([[0.0], time_levels(g)])
    out = {}
    off = 0
    for a, k in planes(g):
        nodes = plane_nodes(g, a)
        shape = [len(v) for v in nodes]
        m = int(np.prod(shape)) if shape else 1
        V = u_nodes[off: off + m * g["t_nodes"]].reshape([g["t_nodes"]] + shape)
        off += m * g["t_nodes"]
        pa = g["lo"][a] + k * (g["hi"][a] - g["lo"][a]) / g["sub"][a]
        # t = 0 level: the initial data at the nodal points
        Xn = []
        grids = np.meshgrid(*nodes, indexing="ij") if nodes else []
        col = 0
        for b in range(d):
            if b == a:
                Xn.append(np.full(shape if shape else (), pa))
            else:
                Xn.append(grids[col])
                col += 1
        V0 = u0_grid(pb, Xn).reshape([1] + shape)
        V = np.concatenate([V0, V], axis=0)
        fd = [coords[b] for b in range(d) if b != a]
        S = spline_tensor(V, [t_nodes] + nodes, [t_targets] + fd)
        # level 0: exact initial data on the FD nodes of the plane
        Xf = []
        gridf = np.meshgrid(*fd, indexing="ij") if fd else []
        col = 0
        for b in range(d):
            if b == a:
                Xf.append(np.full([len(v) for v in fd] if fd else (), pa))
            else:
                Xf.append(gridf[col])
                col += 1
        L0 = u0_grid(pb, Xf).reshape([1] + [len(v) for v in fd])
        out[(a, k)] = np.concatenate([L0, S], axis=0)
    return out


def _ring_from_planes(g, P: dict, n: int, lo_idx: list, hi_idx: list) -> np.ndarray:
    """Full array over global node ranges [lo_idx[a], hi_idx[a]] with its ring set from the planes at level n
    (a ring node on several planes takes the lowest axis's plane)."""
    d = g["dim"]
    shape = [hi_idx[a] - lo_idx[a] + 1 for a in range(d)]
    U = np.zeros(shape)
    done = np.zeros(shape, bool)
    for a in range(d):
        for side in (0, 1):
            gi = lo_idx[a] if side == 0 else hi_idx[a]
            k = gi // g["cells"][a]
            pv = P[(a, k)][n]  # in-plane FD nodes (global indices of the other axes)
            sl_pv = tuple(slice(lo_idx[b], hi_idx[b] + 1) for b in range(d) if b != a)
            face = [slice(None)] * d
            face[a] = 0 if side == 0 else shape[a] - 1
            face = tuple(face)
            vals = pv[sl_pv] if sl_pv else pv
            U[face] = np.where(done[face], U[face], vals)
            done[face] = True
    return U


def pdd_solve(pb: dict, g, u_nodes: np.ndarray, plane_data: dict | None = None,
              subdomains: tuple | None = None) -> np.ndarray:
    """The PDD solution at t = T on the global FD grid: planes from the spline of u_nodes (or the given
    per-level plane data), subdomain interiors from independent Crank-Nicolson solves -- all of them, or
    only those of the row-major range `subdomains` = (begin, end) (other interiors stay 0)."""
    d = g["dim"]
    N, coords = _axes(g)
    P = plane_data if plane_data is not None else plane_values(pb, g, u_nodes)
    dt = g["T"] / g["nsteps"]
    out = np.zeros(N)
    # plane nodes at T (lowest axis wins: write the highest axis first)
    for a in reversed(range(d)):
        for k in range(g["sub"][a] + 1):
            idx = [slice(None)] * d
            idx[a] = k * g["cells"][a]
            out[tuple(idx)] = P[(a, k)][g["nsteps"]]
    for sid, s in enumerate(np.ndindex(*[g["sub"][a] for a in range(d)])):
        if subdomains is not None and not subdomains[0] <= sid < subdomains[1]:
            continue
        lo_idx = [s[a] * g["cells"][a] for a in range(d)]
        hi_idx = [(s[a] + 1) * g["cells"][a] for a in range(d)]
        sub_coords = [coords[a][lo_idx[a]: hi_idx[a] + 1] for a in range(d)]
        U = cn_box(pb, sub_coords, lambda n: _ring_from_planes(g, P, n, lo_idx, hi_idx), dt, g["nsteps"])
        inner_g = tuple(slice(lo_idx[a] + 1, hi_idx[a]) for a in range(d))
        out[inner_g] = U[tuple(slice(1, -1) for _ in range(d))]
    return out


def global_solve(pb: dict, g, u_nodes: np.ndarray | None = None, plane_data: dict | None = None,
                 history: bool = False):
    """The check: one Crank-Nicolson solve over the whole box, Dirichlet data on the outer faces only
    (the outer planes of the same spline), interfaces solved for."""
    d = g["dim"]
    N, coords = _axes(g)
    P = plane_data if plane_data is not None else plane_values(pb, g, u_nodes)
    dt = g["T"] / g["nsteps"]
    lo_idx = [0] * d
    hi_idx = [N[a] - 1 for a in range(d)]
    return cn_box(pb, coords, lambda n: _ring_from_planes(g, P, n, lo_idx, hi_idx), dt, g["nsteps"],
                  history=history)


def planes_from_levels(g, levels: list) -> dict:
    """Per-level plane data cut out of full-grid solution levels (for the decomposition-exactness check)."""
    d = g["dim"]
    P = {}
    for a, k in planes(g):
        idx = [slice(None)] * d
        idx[a] = k * g["cells"][a]
        P[(a, k)] = np.stack([L[tuple(idx)] for L in levels])
    return P
