"""Pins of the oracle's time-stepping coefficients (Secs. 3.2.1-3.2.2.4).

Each check comes from outside the oracle: numbers the paper prints
(tests/golden), exactness on polynomials, or the convergence order on ODEs
with known solutions.
"""
import math

import numpy as np
import pytest

import oracle
from conftest import golden

RNG = np.random.default_rng(1909)


def test_ab3_uniform_reduces_to_23_16_5():
    # Eq. 30 at equal steps gives the fixed-step AB3 of Eq. 16.
    w = golden("ab3_uniform_weights_x12")
    for dt in (1.0, 0.37, 2.5e-3):
        beta = oracle.ab3_weights(dt, dt, dt)
        np.testing.assert_allclose(beta, np.array(w) * dt / 12.0, rtol=2e-16 * 8, atol=0)


def test_fd_uniform_reduce_to_textbook_differences():
    # Eqs. 35, 38, 41 at equal steps: backward, central, forward differences.
    for dt in (1.0, 0.01):
        D = oracle.fd_weights(dt, dt)
        np.testing.assert_allclose(D[0], np.array(golden("fd_backward_uniform_x2dt")) / (2 * dt), rtol=1e-15)
        np.testing.assert_allclose(D[1], np.array(golden("fd_central_uniform_x2dt")) / (2 * dt), rtol=1e-15, atol=1e-15 / dt)
        np.testing.assert_allclose(D[2], np.array(golden("fd_forward_uniform_x2dt")) / (2 * dt), rtol=1e-15)


def test_fstar_uniform_reduces_to_2_3_1():
    # Eq. 43 with Eqs. 44-46 at equal steps gives the 2, -3, 1 of Eq. 17.
    for dt in (1.0, 3e-3):
        g = oracle.dstar_weights(dt, dt, dt)
        np.testing.assert_allclose(g, golden("fstar_uniform_weights"), rtol=1e-14, atol=1e-14)


def _times(a, b, c):
    # t_{n+1} = a, t_n = 0, t_{n-1} = -b, t_{n-2} = -b-c
    return a, 0.0, -b, -b - c


def test_ab3_integrates_quadratics_exactly():
    # Eq. 26: the weights integrate the quadratic interpolant, so any quadratic
    # integrand is integrated exactly for any step ratios.
    for _ in range(200):
        a, b, c = RNG.uniform(0.2, 3.0, size=3)
        p = RNG.standard_normal(3)
        t1, t0, tm1, tm2 = _times(a, b, c)
        f = lambda t: p[0] + p[1] * t + p[2] * t * t
        F = lambda t: p[0] * t + p[1] * t * t / 2 + p[2] * t ** 3 / 3
        beta = oracle.ab3_weights(a, b, c)
        approx = beta @ np.array([f(t0), f(tm1), f(tm2)])
        assert abs(approx - (F(t1) - F(t0))) <= 1e-13 * max(1.0, abs(F(t1)))


def test_fd_exact_on_quadratics():
    # Eqs. 35, 38, 41 are derivatives of the 3-point quadratic interpolant.
    for _ in range(200):
        b, c = RNG.uniform(0.1, 4.0, size=2)
        p = RNG.standard_normal(3)
        ts = np.array([0.0, -b, -b - c])
        Y = p[0] + p[1] * ts + p[2] * ts ** 2
        dY = p[1] + 2 * p[2] * ts
        D = oracle.fd_weights(b, c)
        np.testing.assert_allclose(D @ Y, dY, rtol=1e-12, atol=1e-12 * np.abs(p).max() / min(b, c))


def test_fstar_weights_are_quadratic_extrapolation():
    # sum_k beta_k (F*^{n-k})_t: for a quadratic F*, the AB3 integral of its
    # exact derivative is F*(t_{n+1}) - F*(t_n); the weights must reproduce it.
    for _ in range(200):
        a, b, c = RNG.uniform(0.2, 3.0, size=3)
        p = RNG.standard_normal(3)
        t1, t0, tm1, tm2 = _times(a, b, c)
        Y = lambda t: p[0] + p[1] * t + p[2] * t * t
        g = oracle.dstar_weights(a, b, c)
        lhs = g @ np.array([Y(t0), Y(tm1), Y(tm2)])
        assert abs(lhs - (Y(t1) - Y(t0))) <= 1e-12 * max(1.0, abs(Y(t1)))


def test_fstar_weights_closed_form():
    # Closed form of quadratic extrapolation minus e0 with a, b, c the steps.
    for _ in range(100):
        a, b, c = RNG.uniform(0.1, 3.0, size=3)
        g = oracle.dstar_weights(a, b, c)
        g0 = (a * a + 2 * a * b + a * c + b * b + b * c) / (b * (b + c)) - 1.0
        g1 = -a * (a + b + c) / (b * c)
        g2 = a * (a + b) / (c * (b + c))
        np.testing.assert_allclose(g, [g0, g1, g2], rtol=1e-13, atol=1e-13)


def _step_sequence(h, T, seed=5):
    # variable steps dt_i = h * s(t_i) * rho_{i mod 7}, ratios stay in [0.5, 2]
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.75, 1.3, size=7)
    ts = [0.0]
    i = 0
    while ts[-1] < T - 1e-14:
        dt = h * (1.0 + 0.3 * math.sin(3.0 * ts[-1])) * rho[i % 7]
        dt = min(dt, T - ts[-1])
        ts.append(ts[-1] + dt)
        i += 1
    return np.array(ts)


def _ab3_solve(f, x_exact, h, T, euler_start):
    ts = _step_sequence(h, T)
    dts = np.diff(ts)
    X = [x_exact(ts[0])]
    fs = []
    for n in range(len(dts)):
        if n < 2 and not euler_start:
            X.append(x_exact(ts[n + 1]))
            fs.append(f(ts[n], X[n]))
            continue
        fs.append(f(ts[n], X[n]))
        if n < 2:
            X.append(X[n] + dts[n] * fs[n])
        else:
            beta = oracle.ab3_weights(dts[n], dts[n - 1], dts[n - 2])
            X.append(X[n] + beta @ np.array([fs[n], fs[n - 1], fs[n - 2]]))
    return abs(X[-1] - x_exact(ts[-1]))


@pytest.mark.parametrize("problem", ["linear", "forced"])
def test_ab3_third_order_with_exact_start(problem):
    if problem == "linear":
        f = lambda t, x: -1.3 * x
        xe = lambda t: math.exp(-1.3 * t)
    else:
        f = lambda t, x: math.cos(2.0 * t) - 0.5 * x
        # x' + x/2 = cos 2t, x(0) = 1
        xe = lambda t: (0.5 * math.cos(2 * t) + 2 * math.sin(2 * t)) / 4.25 \
            + (1 - 0.5 / 4.25) * math.exp(-0.5 * t)
    hs = [0.08, 0.04, 0.02, 0.01]
    errs = [_ab3_solve(f, xe, h, 2.0, euler_start=False) for h in hs]
    slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert 2.85 <= slope <= 3.15, (slope, errs)


def test_ab3_second_order_with_euler_start():
    # Sec. 3.2.1: two Euler steps start the scheme; their O(h^2) local error
    # makes the global error second order.
    f = lambda t, x: -1.3 * x
    xe = lambda t: math.exp(-1.3 * t)
    hs = [0.04, 0.02, 0.01, 0.005]
    errs = [_ab3_solve(f, xe, h, 2.0, euler_start=True) for h in hs]
    slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert 1.85 <= slope <= 2.15, (slope, errs)


def test_fstar_term_third_order_for_smooth_signal():
    # The dispersive time-derivative term: sum gamma_k Y^{n-k} approximates
    # Y(t_{n+1}) - Y(t_n) with an O(h^3) local error.
    errs = []
    hs = [0.1, 0.05, 0.025, 0.0125]
    for h in hs:
        a, b, c = h, 1.3 * h, 0.8 * h
        t1, t0, tm1, tm2 = _times(a, b, c)
        Y = np.sin
        g = oracle.dstar_weights(a, b, c)
        errs.append(abs(g @ np.array([Y(t0 + 0.3), Y(tm1 + 0.3), Y(tm2 + 0.3)]) - (Y(t1 + 0.3) - Y(t0 + 0.3))))
    slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert 2.8 <= slope <= 3.2, (slope, errs)


def test_thomas_residual():
    for n in (3, 17, 200):
        a = RNG.uniform(-1, 1, n)
        c = RNG.uniform(-1, 1, n)
        a[0] = 0.0
        c[-1] = 0.0
        b = np.abs(a) + np.abs(c) + RNG.uniform(0.5, 2.0, n)
        r = RNG.standard_normal(n)
        x = oracle.thomas(a, b, c, r)
        T = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
        assert np.linalg.norm(T @ x - r) <= 1e-14 * np.linalg.norm(r) * 10
        np.testing.assert_allclose(x, np.linalg.solve(T, r), rtol=1e-12, atol=1e-13)


def test_wavenumber_limits():
    # shallow-water limit k -> omega / sqrt(g d); deep-ish water from the relation
    d, g = 1.0, 9.81
    om = 0.01
    assert abs(oracle.wavenumber(om, d, g, 1 / 15) - om / math.sqrt(g * d)) < 1e-6 * om
    for kd in (0.5, 1.0, 2.0, 3.0):
        k = kd / d
        B = 1 / 15
        om = math.sqrt(g * d * k * k * (1 + B * kd * kd) / (1 + (B + 1 / 3) * kd * kd))
        assert abs(oracle.wavenumber(om, d, g, B) - k) < 1e-12 * k
