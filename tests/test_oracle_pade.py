"""Pins of the oracle's [L/M] Pade approximant at eps = 1 (Sec. 2.1 end, Sec. 2.4).

* exactness on a rational function of type [2/2];
* agreement with an independent library Pade (mpmath, 40 digits) on random series;
* the ODE closed forms that the Pade sum must reproduce from exact
  eps-coefficients, including u' = u^2 past its pole (the analytic
  continuation beyond the series' radius) through the degeneracy rule;
* the documented degenerate cases (zero series, geometric series, pole at 1, M = 0).
"""
import math

import mpmath
import numpy as np
import pytest

import oracle
from checkers import ode_taylor, ode_taylor_fn, series_of_rational, sin_series


def _mp_pade_at_one(a, L, M):
    mpmath.mp.dps = 40
    p, q = mpmath.pade([mpmath.mpf(float(v)) for v in a[: L + M + 1]], L, M)
    return float(mpmath.polyval(p[::-1], 1) / mpmath.polyval(q[::-1], 1))


@pytest.mark.parametrize("L,M,degenerate", [(2, 2, False), (3, 2, False), (5, 2, False), (4, 3, True),
                                             (4, 4, True)])
def test_rational_function_is_reproduced(L, M, degenerate):
    # a [2/2] rational: every [L/M] with L >= 2, M >= 2 reproduces it; for M > 2 the
    # Toeplitz system is rank-deficient and the degeneracy rule lowers the type.
    a = series_of_rational([1.0, 2.0, -0.5], [1.0, -0.3, 0.2], 17)
    u, st, lm = oracle.pade(a, L, M)
    assert abs(u - 2.5 / 0.9) < 1e-12
    if degenerate:
        assert st & oracle.STATUS_PADE_SINGULAR and lm[1] < M
    else:
        assert st == 0 and lm == (L, M)


@pytest.mark.parametrize("L,M", [(4, 4), (5, 5), (3, 2), (2, 5), (6, 6), (8, 8), (1, 0), (0, 3)])
def test_matches_library_pade_on_random_series(L, M):
    rng = np.random.default_rng(100 * L + M)
    for _ in range(5):
        a = rng.normal(size=L + M + 1)
        u, st, lm = oracle.pade(a, L, M)
        assert lm == (L, M)
        ref = _mp_pade_at_one(a, L, M)
        assert abs(u - ref) <= 1e-9 * max(1.0, abs(ref)), (u, ref)


def test_scaling_series_by_powers_moves_the_evaluation_point():
    # Pade of a_n s^n at 1 equals the Pade of a_n evaluated at eps = s
    rng = np.random.default_rng(7)
    a = rng.normal(size=11)
    s = 0.37
    u, _, _ = oracle.pade(a * s ** np.arange(11), 5, 5)
    mpmath.mp.dps = 40
    p, q = mpmath.pade([mpmath.mpf(float(v)) for v in a], 5, 5)
    ref = float(mpmath.polyval(p[::-1], s) / mpmath.polyval(q[::-1], s))
    assert abs(u - ref) < 1e-9 * max(1, abs(ref))


@pytest.mark.parametrize("t", [0.5, 1.0, 2.0, 5.0])
def test_quadratic_ode_past_the_pole(t):
    # u' = u^2, u(0) = c0: eps-coefficients c0^{n+1} t^n (a geometric series, degenerate
    # for M >= 2), u = c0/(1 - c0 t) also for t > 1/c0 where the series diverges.
    c0 = 0.8
    a = [c0 ** (n + 1) * t ** n for n in range(9)]
    u, st, lm = oracle.pade(a, 4, 4)
    assert abs(u - c0 / (1 - c0 * t)) < 1e-12 * max(1, abs(c0 / (1 - c0 * t)))
    assert st & oracle.STATUS_PADE_SINGULAR
    assert lm == (1, 1)


def test_cubic_ode_closed_form():
    # u' = u - u^3: u = c0 e^t / sqrt(1 + c0^2 (e^{2t} - 1))
    c0, t = 0.5, 1.0
    phi = ode_taylor([0.0, 1.0, 0.0, -1.0], c0, 13)
    a = phi * t ** np.arange(13)
    exact = c0 * math.exp(t) / math.sqrt(1 + c0 * c0 * (math.exp(2 * t) - 1))
    partial = a[:13].sum()
    u, st, _ = oracle.pade(a, 6, 6)
    assert st == 0
    assert abs(u - exact) < 1e-5
    assert abs(u - exact) < 0.1 * abs(partial - exact)


def test_sine_ode_closed_form():
    # u' = sin u: tan(u/2) = tan(c0/2) e^t
    c0, t = 1.2, 1.0
    phi = ode_taylor_fn(sin_series, c0, 13)
    a = phi * t ** np.arange(13)
    exact = 2 * math.atan(math.tan(c0 / 2) * math.exp(t))
    u, st, _ = oracle.pade(a, 6, 6)
    assert abs(u - exact) < 1e-5
    u5, _, _ = oracle.pade(a, 5, 5)
    assert abs(u5 - exact) < 2e-5


def test_degenerate_cases():
    u, st, lm = oracle.pade(np.zeros(9), 4, 4)
    assert u == 0.0 and lm == (0, 0) and st & oracle.STATUS_PADE_SINGULAR
    u, st, lm = oracle.pade(np.ones(9), 4, 4)        # 1/(1 - eps): pole exactly at eps = 1
    assert st & oracle.STATUS_PADE_POLE_NEAR
    a = np.array([0.3, -0.2, 0.05, 0.01])
    u, st, lm = oracle.pade(a, 3, 0)                   # M = 0: partial sum
    assert abs(u - a.sum()) < 1e-16 and st == 0
    with pytest.raises(ValueError):
        oracle.pade(np.zeros(17), 9, 8)


def test_pade_error_closed_forms(oracle_mod):
    """The per-result error helper on approximants with closed-form derivatives:
    [0/0] u = a0; [1/0] u = a0 + a1; [0/1] u = a0^2 / (a0 - a1)."""
    import numpy as np

    a = np.array([[0.7, 0.3, 0.0], [1.2, -0.4, 0.0]])
    se = np.array([[0.01, 0.02, 0.0], [0.03, 0.005, 0.0]])
    e00 = oracle_mod.pade_error(a, se, 0, 0)
    assert np.allclose(e00, se[:, 0], rtol=1e-9)
    e10 = oracle_mod.pade_error(a, se, 1, 0)
    assert np.allclose(e10, np.hypot(se[:, 0], se[:, 1]), rtol=1e-8)
    e01 = oracle_mod.pade_error(a, se, 0, 1)
    a0, a1 = a[:, 0], a[:, 1]
    d0 = (a0 * a0 - 2.0 * a0 * a1) / (a0 - a1) ** 2
    d1 = a0 * a0 / (a0 - a1) ** 2
    assert np.allclose(e01, np.hypot(d0 * se[:, 0], d1 * se[:, 1]), rtol=1e-6)
