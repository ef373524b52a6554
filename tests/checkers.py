"""Independent checkers used to pin the oracle (test-only).

None of this code shares anything with the oracle or the CUDA path.  It holds
mathematics the paper and textbooks fix:

* eps-hierarchy of the ODE that a spatially constant u0 reduces the PDE to:
  exact power-series recursion (Strategy B) and RK4 (Strategy A with a
  potential);
* heat-semigroup closed forms for the initial data families (pure diffusion);
* the first-order (one-split) coefficient as a 1-D time integral;
* a Crank-Nicolson finite-difference solve of 1-D semilinear problems, the
  paper's own check (Sec. 2.4, before Example 1).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, linalg


# ----------------------------------------------------------------------------
# power series helpers
# ----------------------------------------------------------------------------
def series_poly_compose(f_coef, u, nterms):
    """Coefficients of f(u(s)) = sum_k b_k u(s)^k, truncated to nterms."""
    out = np.zeros(nterms)
    pw = np.zeros(nterms)
    pw[0] = 1.0
    for k, b in enumerate(f_coef):
        if k > 0:
            pw = np.convolve(pw, u)[:nterms]
        if b != 0.0:
            out += b * pw
    return out


def ode_taylor(f_coef, c0, nterms):
    """Taylor coefficients phi_n of phi' = f(phi), phi(0) = c0.

    Under Strategy B with constant u0 the order-n coefficient at time t is
    phi_n t^n: the eps-expansion of u' = eps f(u) is phi(eps t).
    """
    phi = np.zeros(nterms)
    phi[0] = c0
    for n in range(nterms - 1):
        fs = series_poly_compose(f_coef, phi[: n + 1], n + 1)
        phi[n + 1] = fs[n] / (n + 1)
    return phi


def ode_taylor_fn(fprime_series, c0, nterms):
    """Taylor coefficients of phi' = F(phi) for an analytic F given as a callable on series."""
    phi = np.zeros(nterms)
    phi[0] = c0
    for n in range(nterms - 1):
        fs = fprime_series(phi[: n + 1].copy(), n + 1)
        phi[n + 1] = fs[n] / (n + 1)
    return phi


def sin_series(u, nterms):
    """sin(u(s)) as a power series (exact sine, for the Pade pins)."""
    u0 = u[0]
    v = u.copy()
    v[0] = 0.0
    # sin(u0 + v) = sin u0 cos v + cos u0 sin v
    cosv = np.zeros(nterms)
    sinv = np.zeros(nterms)
    pw = np.zeros(nterms)
    pw[0] = 1.0
    for k in range(nterms):
        if k > 0:
            pw = np.convolve(pw, v)[:nterms]
        term = pw / math.factorial(k)
        if k % 2 == 0:
            cosv += (-1) ** (k // 2) * term
        else:
            sinv += (-1) ** (k // 2) * term
    return math.sin(u0) * cosv + math.cos(u0) * sinv


def eps_hierarchy_rk4(F_coef, c_pot, c0, t, K, steps=4000):
    """U_n(t) of u' = -c u + eps F(u), u(0) = c0 (the Strategy A series), by RK4."""
    def rhs(U):
        fs = series_poly_compose(F_coef, U, K + 1)
        d = -c_pot * U
        d[1:] += fs[:K]
        return d

    U = np.zeros(K + 1)
    U[0] = c0
    h = t / steps
    for _ in range(steps):
        k1 = rhs(U)
        k2 = rhs(U + 0.5 * h * k1)
        k3 = rhs(U + 0.5 * h * k2)
        k4 = rhs(U + h * k3)
        U = U + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return U


def eps_hierarchy_rk4_t(coef_at, c_pot, c0, t, K, steps=4000):
    """U_n(t) of u' = -c u + eps F(u, t), u(0) = c0, with time-dependent coefficients
    F(u, t) = sum_k coef_at(t)[k] u^k, by RK4 on the order hierarchy."""
    def rhs(U, s):
        fs = series_poly_compose(coef_at(s), U, K + 1)
        d = -c_pot * U
        d[1:] += fs[:K]
        return d

    U = np.zeros(K + 1)
    U[0] = c0
    h = t / steps
    s = 0.0
    for _ in range(steps):
        k1 = rhs(U, s)
        k2 = rhs(U + 0.5 * h * k1, s + 0.5 * h)
        k3 = rhs(U + 0.5 * h * k2, s + 0.5 * h)
        k4 = rhs(U + h * k3, s + h)
        U = U + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        s += h
    return U


def series_of_rational(num, den, nterms):
    """Taylor coefficients of num(e)/den(e) (den[0] != 0)."""
    a = np.zeros(nterms)
    for n in range(nterms):
        s = num[n] if n < len(num) else 0.0
        for j in range(1, min(n, len(den) - 1) + 1):
            s -= den[j] * a[n - j]
        a[n] = s / den[0]
    return a


# ----------------------------------------------------------------------------
# heat semigroup closed forms (variance 2 D tau per coordinate)
# ----------------------------------------------------------------------------
def heat_gauss(x, tau, D, c0, A, s, x0):
    """E[g(x + sqrt(2 D tau) n)] for g = c0 + A exp(-|x - x0|^2/(2 s^2))."""
    x = np.atleast_2d(x)
    d = x.shape[1]
    v = s * s + 2.0 * D * tau
    r2 = ((x - np.asarray(x0)[:d]) ** 2).sum(axis=1)
    return c0 + A * (s * s / v) ** (d / 2.0) * np.exp(-r2 / (2.0 * v))


def heat_cos_prod(x, tau, D, c0, A, w):
    x = np.atleast_2d(x)
    d = x.shape[1]
    pr = np.ones(x.shape[0])
    for i in range(d):
        pr *= np.cos(w[i] * x[:, i]) * math.exp(-w[i] ** 2 * D * tau)
    return c0 + A * pr


def heat_quadrature_1d(fun, x, tau, D, n=120):
    """E[fun(x + sqrt(2 D tau) n)] by Gauss-Hermite quadrature."""
    z, w = np.polynomial.hermite_e.hermegauss(n)
    w = w / math.sqrt(2 * math.pi)
    sig = math.sqrt(2.0 * D * tau)
    return np.array([(w * fun(xx + sig * z)).sum() for xx in np.atleast_1d(x)])


def first_order_gauss_1d(x, t, D, A, s, b, c_pot=0.0):
    """Order-1 coefficient for f = b u^2 (plus a pulled-out potential c), g = A exp(-x^2/(2 s^2)).

    a_1(x,t) = b int_0^t e^{-c s'} e^{-2c(t-s')} P_{s'}[(P_{t-s'} g)^2](x) ds'.
    P_tau g is Gaussian with variance v = s^2 + 2 D tau; its square is Gaussian
    with variance v/2 and amplitude A^2 s^2/v.
    """
    def integrand(sp, xx):
        v = s * s + 2.0 * D * (t - sp)
        amp = A * A * s * s / v
        w = v / 2.0
        vv = w + 2.0 * D * sp
        return math.exp(-c_pot * sp - 2.0 * c_pot * (t - sp)) * amp * math.sqrt(w / vv) * math.exp(-xx * xx / (2 * vv))

    return np.array([b * integrate.quad(integrand, 0.0, t, args=(xx,), epsabs=1e-13, epsrel=1e-11)[0]
                     for xx in np.atleast_1d(x)])


# ----------------------------------------------------------------------------
# Crank-Nicolson for u_t = D u_xx + f(u) on [-Lb, Lb] with Dirichlet data
# ----------------------------------------------------------------------------
def crank_nicolson_1d(f, fprime, u0, D, t_end, Lb, dx, dt, bc):
    """Solve u_t = D u_xx + f(u); bc(t) gives the (equal) Dirichlet value at both ends.

    Nonlinear Crank-Nicolson with Newton iterations on a tridiagonal system.
    Returns (x grid, u(x, t_end)).
    """
    x = np.arange(-Lb, Lb + 0.5 * dx, dx)
    n = x.size
    u = u0(x).astype(np.float64)
    r = D * dt / (dx * dx)
    nsteps = int(round(t_end / dt))
    dt = t_end / nsteps
    r = D * dt / (dx * dx)
    for step in range(nsteps):
        tn1 = (step + 1) * dt
        lap = np.zeros(n)
        lap[1:-1] = u[2:] - 2 * u[1:-1] + u[:-2]
        rhs_old = u + 0.5 * r * lap + 0.5 * dt * f(u)
        v = u.copy()
        v[0] = v[-1] = bc(tn1)
        for _ in range(8):
            lapv = np.zeros(n)
            lapv[1:-1] = v[2:] - 2 * v[1:-1] + v[:-2]
            G = v - 0.5 * r * lapv - 0.5 * dt * f(v) - rhs_old
            G[0] = G[-1] = 0.0
            diag = 1 + r - 0.5 * dt * fprime(v)
            ab = np.zeros((3, n))
            ab[0, 1:] = -0.5 * r
            ab[1, :] = diag
            ab[2, :-1] = -0.5 * r
            ab[1, 0] = ab[1, -1] = 1.0
            ab[0, 1] = 0.0
            ab[2, -2] = 0.0
            dv = linalg.solve_banded((1, 1), ab, -G)
            v = v + dv
            if np.max(np.abs(dv)) < 1e-14:
                break
        u = v
    return x, u
