"""Pins of the oracle's spatial scheme and whole steps against what the paper
and the mathematics fix: polynomial exactness of the stencils, the tridiagonal
operator of Eqs. 19-21, well-balancing (lake at rest), mass conservation,
the NLSW limit d = 0 against the Stoker and Ritter dam-break solutions, the
Madsen-Sorensen linear dispersion relation, symmetry, the CFL rule of Eq. 22
and the lazy EMA of Eq. 47, dry land and the wave maker.
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
from paper_1909_04153_gb300 import workloads as W

G = 9.81
B15 = 1.0 / 15.0


def _dom(case, **over):
    p = dict(case["params"])
    p.update(over)
    return oracle.OracleDomain(p, case["bed"], case["comps"], case["eta0"], case["P0"], case["Q0"])


def _smooth_bed(nx, ny, dx, seed=3, lo=0.4, hi=1.2):
    rng = np.random.default_rng(seed)
    X, Y = np.meshgrid(np.arange(nx + 1) * dx, np.arange(ny + 1) * dx)
    b = np.zeros_like(X)
    for _ in range(4):
        kx, ky, ph = rng.uniform(0.1, 0.6), rng.uniform(0.1, 0.6), rng.uniform(0, 6.28)
        b += np.cos(kx * X + ph) * np.cos(ky * Y)
    b = (b - b.min()) / (b.max() - b.min())
    return -(lo + (hi - lo) * b)


# ------------------------------------------------------------------ stencils

def test_dispersive_stencils_exact_on_polynomials():
    nx, ny, dx = 24, 20, 0.1
    sx, sy, b0 = 0.03, -0.02, -1.0
    X, Y = np.meshgrid(np.arange(nx + 1) * dx, np.arange(ny + 1) * dx)
    bed = b0 + sx * X + sy * Y
    xc, yc = (np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dx
    Xc, Yc = np.meshgrid(xc, yc)
    c = [0.01, 0.02, -0.015, 0.007, 0.004, -0.003, 0.002, -0.001, 0.0015, 0.0008]
    eta = (c[0] + c[1] * Xc + c[2] * Yc + c[3] * Xc ** 2 + c[4] * Xc * Yc + c[5] * Yc ** 2
           + c[6] * Xc ** 3 + c[7] * Xc ** 2 * Yc + c[8] * Xc * Yc ** 2 + c[9] * Yc ** 3)
    q = [0.05, 0.01, -0.02, 0.03, 0.015, -0.01]
    Qf = q[0] + q[1] * Xc + q[2] * Yc + q[3] * Xc ** 2 + q[4] * Xc * Yc + q[5] * Yc ** 2
    Pf = 0.5 * Qf[::-1, ::-1].copy() + 0.02 * Xc * Yc
    p = W.base_params(nx, ny, dx)
    D = oracle.OracleDomain(p, bed, None, eta, Pf, Qf)
    out = D.dispersive()
    # exact derivatives of the polynomials
    e_x = c[1] + 2 * c[3] * Xc + c[4] * Yc + 3 * c[6] * Xc ** 2 + 2 * c[7] * Xc * Yc + c[8] * Yc ** 2
    e_xx = 2 * c[3] + 6 * c[6] * Xc + 2 * c[7] * Yc
    e_yy = 2 * c[5] + 2 * c[8] * Xc + 6 * c[9] * Yc
    e_xy = c[4] + 2 * c[7] * Xc + 2 * c[8] * Yc
    e_xxx = 6 * c[6] + 0 * Xc
    e_yyy = 6 * c[9] + 0 * Xc
    e_xyy = 2 * c[8] + 0 * Xc
    e_xxy = 2 * c[7] + 0 * Xc
    del e_x
    d = -(b0 + sx * Xc + sy * Yc)
    dx_, dy_ = -sx, -sy
    dispx = B15 * G * d ** 3 * (e_xxx + e_xyy) + B15 * G * d ** 2 * (dx_ * (2 * e_xx + e_yy) + dy_ * e_xy)
    dispy = B15 * G * d ** 3 * (e_yyy + e_xxy) + B15 * G * d ** 2 * (dy_ * (2 * e_yy + e_xx) + dx_ * e_xy)
    Q_x, Q_y, Q_xy = q[1] + 2 * q[3] * Xc + q[4] * Yc, q[2] + q[4] * Xc + 2 * q[5] * Yc, q[4] + 0 * Xc
    Fs = d * dx_ * Q_y / 6 + d * dy_ * Q_x / 6 + (B15 + 1 / 3) * d * d * Q_xy
    s = (slice(2, -2), slice(2, -2))
    for got, ref in ((out["dispx"], dispx), (out["dispy"], dispy), (out["Fs"], Fs)):
        np.testing.assert_allclose(got[s], ref[s], rtol=1e-9, atol=1e-12 * np.abs(ref).max())


def test_flux_consistency_uniform_flow():
    # A spatially uniform wet state on a flat bed: every face flux equals the
    # exact flux, so E = 0 and F = G = 0 in the cells away from the walls, and
    # with friction f, F = -f u |u| (the friction term of Eq. 12).
    nx, ny, dx, h = 12, 10, 0.2, 0.7
    bed = np.full((ny + 1, nx + 1), -h)
    P0 = np.full((ny, nx), 0.21)
    Q0 = np.full((ny, nx), -0.14)
    D = oracle.OracleDomain(W.base_params(nx, ny, dx, friction=0.003), bed, None, None, P0, Q0)
    r = D.rhs()
    s = (slice(3, -3), slice(3, -3))
    eps = dx ** 4
    u = math.sqrt(2) * h * 0.21 / math.sqrt(2 * max(h ** 4, eps))
    v = math.sqrt(2) * h * -0.14 / math.sqrt(2 * max(h ** 4, eps))
    np.testing.assert_allclose(r["E"][s], 0.0, atol=1e-13)
    np.testing.assert_allclose(r["F"][s], -0.003 * u * math.hypot(u, v), rtol=1e-10)
    np.testing.assert_allclose(r["G"][s], -0.003 * v * math.hypot(u, v), rtol=1e-10)


@pytest.mark.parametrize("mode", [0, 1])
def test_line_solve_inverts_eq19_operator(mode):
    # After one Euler step, applying the operator of Eqs. 9-10 / 19-20 to the
    # new P, Q gives the old U*, V* plus dt F, dt G.  The F*, G* terms are zero
    # on the first step, except that cross_mode 1 adds F*(Q^{n+1}) - F*(Q^n)
    # to U*.  The operator is applied forward, independently of the Thomas
    # solve, with wall ghosts supplying the neighbour outside the line.
    case = W.barred_beach(nx=40, ny=36)
    rng = np.random.default_rng(4)
    P0 = 0.05 * rng.standard_normal((36, 40))
    Q0 = 0.03 * rng.standard_normal((36, 40))
    D = oracle.OracleDomain(dict(case["params"], bc=(0, 0, 0, 0), cross_mode=mode), case["bed"],
                            None, None, P0, Q0)
    U0, V0 = D.apply_T()
    r0 = D.rhs()
    dt = 1e-3
    D.step(dt)
    U1, V1 = D.apply_T()
    dFs = D.rhs()["Fs"] - r0["Fs"] if mode == 1 else 0.0
    np.testing.assert_allclose(U1, U0 + dt * r0["F"] + dFs, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(V1, V0 + dt * r0["G"], rtol=1e-12, atol=1e-14)
    assert D.diag_dominant()


def test_d_zero_gives_identity_operator():
    # d = 0 (still water below the bed everywhere): Eqs. 9-10 reduce to U* = P.
    nx, ny, dx = 16, 12, 0.1
    bed = np.zeros((ny + 1, nx + 1))
    P0 = np.random.default_rng(2).standard_normal((ny, nx))
    D = oracle.OracleDomain(W.base_params(nx, ny, dx, w_s=-1.0), bed, None, np.full((ny, nx), 0.5), P0, None)
    U, V = D.apply_T()
    np.testing.assert_array_equal(U, P0)


# ------------------------------------------------------------------ balance and conservation

def test_lake_at_rest_fully_wet_uneven_bed():
    # KP07 is well-balanced and eta = 0, P = Q = 0 zero every dispersive term:
    # the still lake must stay still to round-off over 1000 steps.
    nx, ny, dx = 40, 30, 0.1
    bed = _smooth_bed(nx, ny, dx)
    D = oracle.OracleDomain(W.base_params(nx, ny, dx, cfl=0.125), bed, None, None, None, None)
    D.run(1000)
    assert np.abs(D.get("eta")).max() <= 1e-13
    assert np.abs(D.get("P")).max() <= 1e-13
    assert np.abs(D.get("Q")).max() <= 1e-13
    assert D.info()["clamps"] == 0


def test_mass_conserved_in_walled_basin():
    nx, ny, dx = 48, 32, 0.1
    bed = _smooth_bed(nx, ny, dx, seed=7)
    xc = (np.arange(nx) + 0.5) * dx
    yc = (np.arange(ny) + 0.5) * dx
    X, Y = np.meshgrid(xc, yc)
    eta = 0.08 * np.exp(-((X - 1.5) ** 2 + (Y - 1.2) ** 2) / 0.3)
    D = oracle.OracleDomain(W.base_params(nx, ny, dx, cfl=0.125), bed, None, eta, None, None)
    m0 = D.info()["mass"]
    D.run(400)
    info = D.info()
    assert info["clamps"] == 0
    assert abs(info["mass"] - m0) <= 1e-13 * m0
    assert np.abs(D.get("eta")).max() > 1e-3  # the hump did move


# ------------------------------------------------------------------ NLSW limit (d = 0): dam breaks

def _stoker(x, t, hl, hr):
    cl = math.sqrt(G * hl)

    def fm(hm):
        um = 2.0 * (cl - math.sqrt(G * hm))
        return um - (hm - hr) * math.sqrt(G * (hm + hr) / (2.0 * hm * hr))

    hm = brentq(fm, hr * (1 + 1e-12), hl)
    um = 2.0 * (cl - math.sqrt(G * hm))
    cm = math.sqrt(G * hm)
    s = hm * um / (hm - hr)
    h = np.empty_like(x)
    for i, xi in enumerate(x):
        if xi <= -cl * t:
            h[i] = hl
        elif xi <= (um - cm) * t:
            h[i] = (2.0 * cl - xi / t) ** 2 / (9.0 * G)
        elif xi <= s * t:
            h[i] = hm
        else:
            h[i] = hr
    return h


def _ritter(x, t, hl):
    cl = math.sqrt(G * hl)
    h = np.where(x <= -cl * t, hl, (2.0 * cl - x / t) ** 2 / (9.0 * G))
    return np.where(x >= 2 * cl * t, 0.0, h)


def _dam_break_error(nx, hl, hr, t=1.0, length=20.0):
    dx = length / nx
    ny = 3
    bed = np.zeros((ny + 1, nx + 1))
    xc = (np.arange(nx) + 0.5) * dx - length / 2
    h0 = np.where(xc < 0, hl, hr)
    # w_s below the bed: d = 0, the equations are NLSW (Sec. 2)
    D = oracle.OracleDomain(W.base_params(nx, ny, dx, w_s=-1.0, cfl=0.2), bed, None,
                            np.tile(h0, (ny, 1)), None, None)
    D.advance(t)
    h = D.get("h")
    assert np.all(h >= 0)
    np.testing.assert_array_equal(h[0], h[1])  # y-invariant problem stays y-invariant
    assert np.abs(D.get("Q")).max() == 0.0
    ref = _stoker(xc, t, hl, hr) if hr > 0 else _ritter(xc, t, hl)
    return np.sum(np.abs(h[0] - ref)) * dx


@pytest.mark.parametrize("hr", [0.1, 0.0])
def test_dam_break_matches_stoker_and_ritter(hr):
    e1 = _dam_break_error(200, 1.0, hr)
    e2 = _dam_break_error(400, 1.0, hr)
    assert e2 < (0.03 if hr > 0 else 0.06), (e1, e2)
    assert e2 < e1 / 1.4, (e1, e2)


# ------------------------------------------------------------------ dispersion (Sec. 2, kd < 3)

def _standing_period(kd, Bd, cells=40, depth=1.0, periods=2.0):
    k = kd / depth
    L = 2 * math.pi / k
    nx, ny = cells, 3
    dx = L / nx
    bed = np.full((ny + 1, nx + 1), -depth)
    xc = (np.arange(nx) + 0.5) * dx
    eta = np.tile(1e-3 * np.cos(k * xc), (ny, 1))
    om = math.sqrt(G * depth * k * k * (1 + Bd * kd * kd) / (1 + (Bd + 1 / 3) * kd * kd))
    T = 2 * math.pi / om
    D = oracle.OracleDomain(W.base_params(nx, ny, dx, Bd=Bd, cfl=0.1), bed, None, eta, None, None)
    ts, es = [0.0], [D.get("eta")[0, 0]]
    while ts[-1] < periods * T:
        D.step()
        ts.append(D.info()["t"])
        es.append(D.get("eta")[0, 0])
    ts, es = np.array(ts), np.array(es)
    # upward zero crossings of the wall signal (cos starts at +A)
    idx = np.where((es[:-1] < 0) & (es[1:] >= 0))[0]
    tc = ts[idx] - es[idx] * (ts[idx + 1] - ts[idx]) / (es[idx + 1] - es[idx])
    dn = np.where((es[:-1] > 0) & (es[1:] <= 0))[0]
    td = ts[dn] - es[dn] * (ts[dn + 1] - ts[dn]) / (es[dn + 1] - es[dn])
    return 2.0 * (tc[0] - td[0]) if len(tc) and len(td) else float("nan"), T


@pytest.mark.parametrize("kd", [0.5, 1.0, 2.0, 3.0])
def test_linear_dispersion_madsen_sorensen(kd):
    Tm, T = _standing_period(kd, B15)
    assert abs(Tm - T) / T < 0.01, (Tm, T)


def test_dispersion_depends_on_B():
    # At kd = 3 the B = 1/15 and B = 0 relations differ by ~18% in period;
    # the model must follow the B it is given.
    Tm, T = _standing_period(3.0, 0.0)
    assert abs(Tm - T) / T < 0.01, (Tm, T)
    T15 = _standing_period(3.0, B15)[1]
    assert abs(T15 - T) / T > 0.1


# ------------------------------------------------------------------ symmetry

def test_transpose_symmetry():
    # With both cross terms extrapolated (cross_mode 0, the form printed in
    # Eqs. 17-18) the scheme treats x and y alike: the transposed problem gives
    # the transposed answer.  dx is coarse enough (d/dx <= 1.2) for that form
    # to be stable.
    nx, ny, dx = 40, 28, 1.0
    bed = _smooth_bed(nx, ny, dx, seed=11, lo=0.4, hi=1.2)
    case = W.solitary_basin(nx=nx, ny=ny, dx=dx, x0=10.0, depth=0.8, amp=0.05)
    eta = case["eta0"] * np.linspace(0.5, 1.0, ny)[:, None]
    P0 = case["P0"] * np.linspace(0.5, 1.0, ny)[:, None]
    A = oracle.OracleDomain(W.base_params(nx, ny, dx, cfl=0.125, cross_mode=0), bed, None, eta, P0, None)
    B = oracle.OracleDomain(W.base_params(ny, nx, dx, cfl=0.125, cross_mode=0), bed.T.copy(), None,
                            eta.T.copy(), None, P0.T.copy())
    dts = A.run(120)
    B.run(0, dts=dts)
    assert np.abs(A.get("Q")).max() > 1e-4
    np.testing.assert_allclose(B.get("eta").T, A.get("eta"), atol=1e-14)
    np.testing.assert_allclose(B.get("Q").T, A.get("P"), atol=1e-14)
    np.testing.assert_allclose(B.get("P").T, A.get("Q"), atol=1e-14)


def test_cross_term_forms_stability():
    # Reading of Eqs. 17-18 / 43: explicit quadratic extrapolation of both
    # F* and G* is unstable for diagonal grid modes once d/dx exceeds about
    # 1.5, at any dt (per-step growth > 1).  Solving Q first and taking F* at
    # the new level from Q^{n+1} (cross_mode 1) is stable.
    nx, ny, dx, depth = 40, 30, 0.1, 0.3
    bed = np.full((ny + 1, nx + 1), -depth)
    noise = 1e-10 * np.random.default_rng(0).standard_normal((ny, nx))
    growth = {}
    for mode in (0, 1):
        D = oracle.OracleDomain(W.base_params(nx, ny, dx, cfl=0.05, cross_mode=mode), bed, None, noise, None, None)
        v = []
        for _ in range(150):
            D.step()
            v.append(np.abs(D.get("P")).max())
        growth[mode] = (v[-1] / v[-51]) ** (1 / 50)
    assert growth[0] > 1.05, growth
    assert growth[1] < 1.001, growth


def test_mirror_symmetry():
    nx, ny, dx = 36, 20, 0.1
    bed = _smooth_bed(nx, ny, dx, seed=13)
    xc = (np.arange(nx) + 0.5) * dx
    eta = np.tile(0.05 * np.exp(-(xc - 1.0) ** 2 / 0.2), (ny, 1))
    A = oracle.OracleDomain(W.base_params(nx, ny, dx, cfl=0.125), bed, None, eta, None, None)
    B = oracle.OracleDomain(W.base_params(nx, ny, dx, cfl=0.125), bed[:, ::-1].copy(), None, eta[:, ::-1].copy(), None, None)
    dts = A.run(100)
    B.run(0, dts=dts)
    np.testing.assert_allclose(B.get("eta")[:, ::-1], A.get("eta"), atol=1e-14)
    np.testing.assert_allclose(-B.get("P")[:, ::-1], A.get("P"), atol=1e-14)


# ------------------------------------------------------------------ time step control (Eqs. 22, 47)

def test_cfl_control_without_ema():
    case = W.solitary_basin(nx=64, ny=16)
    D = _dom(case, ema_alpha=1.0)
    for _ in range(30):
        D.step()
        info = D.info()
        assert abs(info["last_dt"] * info["last_rate"] - 0.2) <= 1e-14


def test_lazy_ema_rises_slowly_and_drops_at_once():
    # dt_n may fall to the CFL value at once but only rises by alpha of the gap.
    case = W.planar_beach(nx=96, ny=12, steps=0)
    D = _dom(case, ema_alpha=0.1, dt_init=1e-4)
    prev = None
    rises = 0
    for n in range(300):
        D.step()
        info = D.info()
        dt, dtc = info["last_dt"], D.params["cfl"] / info["last_rate"]
        assert dt <= dtc * (1 + 1e-14)
        if n >= 2 and prev is not None:
            if dtc > prev:
                np.testing.assert_allclose(dt, 0.1 * dtc + 0.9 * prev, rtol=1e-14)
                rises += 1
            else:
                np.testing.assert_allclose(dt, dtc, rtol=1e-14)
        prev = dt
    assert rises > 10


def test_landing_on_t_end():
    case = W.solitary_basin(nx=64, ny=8)
    D = _dom(case)
    D.advance(0.5)
    assert abs(D.info()["t"] - 0.5) <= 1e-15


# ------------------------------------------------------------------ dry land and maker

def test_dry_land_stays_dry_with_eta_zero():
    nx, ny, dx = 60, 8, 0.05
    xk = np.arange(nx + 1) * dx
    bed = np.tile(-0.3 + 0.5 * xk / xk[-1], (ny + 1, 1))  # shoreline at x = 1.8 m
    case = W.solitary_basin(nx=nx, ny=ny, dx=dx, depth=0.3, amp=0.01, x0=0.6)
    bc = 0.25 * (bed[:-1, :-1] + bed[1:, :-1] + bed[:-1, 1:] + bed[1:, 1:])
    eta0 = np.where(bc < 0, case["eta0"], 0.0)
    D = oracle.OracleDomain(W.base_params(nx, ny, dx, cfl=0.125), bed, None, eta0, None, None)
    D.run(200)
    h, eta, d = D.get("h"), D.get("eta"), D.get("d")
    dry = (h == 0) & (d == 0)
    assert dry[:, -5:].all()
    assert np.all(eta[dry] == 0.0)
    assert np.all(h >= 0)


def test_sine_maker_generates_the_model_wavelength():
    # Regular waves from the west side travel east with the wavenumber of the
    # dispersion relation and roughly the requested height.
    depth, T, H = 0.5, 1.2, 0.01
    om = 2 * math.pi / T
    k = brentq(lambda k: G * depth * k * k * (1 + B15 * (k * depth) ** 2) / (1 + (B15 + 1 / 3) * (k * depth) ** 2) - om * om, 1e-6, 100)
    L = 2 * math.pi / k
    nx, ny = 240, 3
    dx = 8 * L / 160
    bed = np.full((ny + 1, nx + 1), -depth)
    prm = W.base_params(nx, ny, dx, bc=(2, 1, 0, 0), sponge_width=(0, 2.5 * L, 0, 0), ramp_time=3 * T)
    D = oracle.OracleDomain(prm, bed, np.array([[H / 2, 1 / T, 0.0, 0.0]]), None, None, None)
    assert abs(D.component_k(0) - k) < 1e-10 * k
    D.advance(14 * T)
    eta = D.get("eta")[1]
    seg = eta[: int(4 * L / dx)]
    xc = (np.arange(len(seg)) + 0.5) * dx
    # least-squares fit of a cos(kx) + b sin(kx) over a range of k
    ks = np.linspace(0.8 * k, 1.2 * k, 801)
    res = []
    for kk in ks:
        A = np.stack([np.cos(kk * xc), np.sin(kk * xc)], 1)
        coef, r, *_ = np.linalg.lstsq(A, seg, rcond=None)
        res.append(np.sum((A @ coef - seg) ** 2))
    k_fit = ks[int(np.argmin(res))]
    assert abs(k_fit - k) / k < 0.02, (k_fit, k)
    amp = 0.5 * (seg.max() - seg.min())
    assert 0.8 * H / 2 < amp < 1.2 * H / 2, amp


def test_oblique_maker_state_closed_form():
    # One linear component travelling at angle theta (A20): eta = r(t) a cos(k (x cos theta +
    # y sin theta) - omega t + phi), P and Q = (omega / k) (cos theta, sin theta) eta, k from
    # the Madsen-Sorensen dispersion relation at the maker's still depth, r = tanh(3 t / ramp).
    # A swapped cos/sin, a dropped sign or a missing ramp fails one of the sampled points.
    depth, T, a, phi, theta, ramp = 0.6, 1.4, 0.004, 0.7, 0.4, 2.0
    om = 2 * math.pi / T
    k = brentq(lambda k: G * depth * k * k * (1 + B15 * (k * depth) ** 2) / (1 + (B15 + 1 / 3) * (k * depth) ** 2) - om * om, 1e-6, 100)
    nx, ny, dx = 40, 30, 0.05
    bed = np.full((ny + 1, nx + 1), -depth)
    prm = W.base_params(nx, ny, dx, bc=(2, 0, 0, 0), ramp_time=ramp)
    D = oracle.OracleDomain(prm, bed, np.array([[a, 1 / T, phi, theta]]), None, None, None)
    assert abs(D.component_k(0) - k) < 1e-10 * k
    c = om / k
    for x, y, t in [(-0.025, 0.3, 0.1), (-0.075, 1.2, 0.9), (-0.025, -0.025, 3.3), (0.4, 0.7, 5.0)]:
        r = math.tanh(3 * t / ramp)
        eta = r * a * math.cos(k * (x * math.cos(theta) + y * math.sin(theta)) - om * t + phi)
        got = D.maker_state(x, y, t)
        np.testing.assert_allclose(got, [eta, c * math.cos(theta) * eta, c * math.sin(theta) * eta],
                                   rtol=1e-12, atol=1e-16)


def test_ghost_corners_follow_the_column_then_row_fill():
    # Reading R6 (Sec. 3.3 is silent on the 2x2 corner blocks): the W/E ghost columns
    # are filled first, then the S/N ghost rows over all columns from the filled
    # columns (Q negated) or, on a maker side, from the maker.  Oblique components
    # make the maker vary along y, so evaluating it at the corner itself would differ.
    nx, ny, dx, t = 20, 16, 0.1, 1.3
    bed = np.full((ny + 1, nx + 1), -0.5)
    comps = np.array([[0.01, 0.8, 0.3, 0.5], [0.006, 1.1, 1.7, -0.4]])
    # maker W, wall S, sponge N: corners take the mirrored maker column
    D = oracle.OracleDomain(W.base_params(nx, ny, dx, bc=(2, 0, 0, 1), sponge_width=(0, 0, 0, 0.5)),
                            bed, comps, None, None, None)
    D.fill_ghosts(t)
    w, P, Q = (D.get_padded(f) for f in ("w", "P", "Q"))
    for gi in (-1, -2):
        for gj, sj in ((-1, 0), (-2, 1), (ny, ny - 1), (ny + 1, ny - 2)):
            c, s = (gj + 2, gi + 2), (sj + 2, gi + 2)
            assert w[c] == w[s] and P[c] == P[s] and Q[c] == -Q[s]
            e, p, q = D.maker_state((gi + 0.5) * dx, (sj + 0.5) * dx, t)
            assert abs(P[s] - p) <= 1e-15 and abs(Q[s] - q) <= 1e-15
        assert abs(Q[(2, gi + 2)]) > 1e-6  # the oblique maker has a y flux to negate
    # maker S, wall W: the S row's corner cells are maker cells at their own position
    D = oracle.OracleDomain(W.base_params(nx, ny, dx, bc=(0, 0, 2, 0)), bed, comps, None, None, None)
    D.fill_ghosts(t)
    P, Q = D.get_padded("P"), D.get_padded("Q")
    for gi in (-1, -2, nx, nx + 1):
        for gj in (-1, -2):
            e, p, q = D.maker_state((gi + 0.5) * dx, (gj + 0.5) * dx, t)
            assert abs(P[gj + 2, gi + 2] - p) <= 1e-15 and abs(Q[gj + 2, gi + 2] - q) <= 1e-15


# ------------------------------------------------------------------ sponge layers (Sec. 3.3, reading A19)

def test_sponge_profile_at_the_wall_middle_and_inner_edge():
    # Reading A19: inside a band of width L the factor rises smoothly from 0 at
    # the outer wall to 1 at the band's inner edge, passes 1/2 half-way, is 1
    # beyond the band, and a corner takes the product of its two sides.  The
    # band widths put a cell centre exactly half-way into each band.
    nx, ny, dx = 40, 30, 0.1
    Lw, Le, Ls, Ln = 0.9, 0.5, 0.7, 1.1   # 2 (k + 1/2) dx: cell k centred at L/2
    bed = np.full((ny + 1, nx + 1), -0.5)
    D = oracle.OracleDomain(W.base_params(nx, ny, dx, bc=(1, 1, 1, 1), sponge_width=(Lw, Le, Ls, Ln)),
                            bed, None, None, None, None)
    g = D.get("sponge")
    assert np.all(g >= 0.0) and np.all(g <= 1.0)
    jm, im = ny // 2, nx // 2
    row, col = g[jm], g[:, im]  # away from the S/N bands, away from the W/E bands
    # half-way into each band
    assert abs(row[4] - 0.5) < 1e-14 and abs(row[nx - 1 - 2] - 0.5) < 1e-14
    assert abs(col[3] - 0.5) < 1e-14 and abs(col[ny - 1 - 5] - 0.5) < 1e-14
    # nearly zero at the wall: the first cell centre sits dx/2 from it, where a
    # profile with zero value and zero slope at the wall is of order (dx/L)^2
    for v, L in ((row[0], Lw), (row[-1], Le), (col[0], Ls), (col[-1], Ln)):
        assert 0.0 < v < (dx / L) ** 2, (v, L)
    # rising from the wall to the inner edge, then exactly 1 outside the bands
    nw, ne = int(round(Lw / dx)), int(round(Le / dx))
    assert np.all(np.diff(row[:nw]) > 0) and np.all(np.diff(row[nx - ne:]) < 0)
    assert np.all(row[nw:nx - ne] == 1.0) and np.all(col[int(round(Ls / dx)):ny - int(round(Ln / dx))] == 1.0)
    # near the inner edge the factor is 1 - O(((L - r)/L)^2): a smooth join
    assert 1.0 - row[nw - 1] < (dx / Lw) ** 2 * 3
    # corners: product of the two sides' factors
    np.testing.assert_allclose(g[0, 0], row[0] * col[0], rtol=1e-14)
    np.testing.assert_allclose(g[-1, -1], row[-1] * col[-1], rtol=1e-14)
    np.testing.assert_allclose(g[3, nx - 3], row[nx - 3] * col[3], rtol=1e-14)


def _channel_eta(nx, east_bc, sponge_len, dx, depth, T, H, t_end, dt):
    ny = 3
    bed = np.full((ny + 1, nx + 1), -depth)
    prm = W.base_params(nx, ny, dx, bc=(2, east_bc, 0, 0), sponge_width=(0, sponge_len, 0, 0),
                        ramp_time=3 * T)
    D = oracle.OracleDomain(prm, bed, np.array([[H / 2, 1 / T, 0.0, 0.0]]), None, None, None)
    D.run(0, dts=[dt] * int(round(t_end / dt)))  # the same fixed steps in every channel
    return D.get("eta")[1]


def test_sponge_absorbs_what_a_wall_reflects():
    # Regular waves from the west run down a 1D channel.  A long channel, whose
    # far end the waves cannot reach and return from in time, gives the
    # incident wave alone.  In a short channel the wave reaches the east end and
    # comes back over the probe zone near the maker: a wall sends back all of
    # it (a standing wave, difference from the incident wave of the order of the
    # wave itself); a sponge band of 1.5 wavelengths must send back little.
    depth, T, H = 0.5, 1.2, 0.01
    om = 2 * math.pi / T
    k = brentq(lambda k: G * depth * k * k * (1 + B15 * (k * depth) ** 2) / (1 + (B15 + 1 / 3) * (k * depth) ** 2) - om * om, 1e-6, 100)
    Lw = 2 * math.pi / k
    dx, dt, t_end = 0.05, 0.004, 24.0
    n_short, n_long = 240, 800                     # 12 m and 40 m
    probe = slice(int(1.0 / dx), int(6.0 / dx))    # 1 m to 6 m from the maker
    ref = _channel_eta(n_long, 0, 0.0, dx, depth, T, H, t_end, dt)[probe]
    wall = _channel_eta(n_short, 0, 0.0, dx, depth, T, H, t_end, dt)[probe]
    sponge = _channel_eta(n_short, 1, 1.5 * Lw, dx, depth, T, H, t_end, dt)[probe]
    nref = np.linalg.norm(ref)
    assert nref > 0.3 * H / 2 * math.sqrt(probe.stop - probe.start)  # the incident wave is there
    r_wall = np.linalg.norm(wall - ref) / nref
    r_sponge = np.linalg.norm(sponge - ref) / nref
    assert r_wall > 0.5, r_wall
    assert r_sponge < 0.02 * r_wall, (r_sponge, r_wall)


# ------------------------------------------------------------------ Euler start (Sec. 3.2.1, reading A12)

@pytest.mark.parametrize("mode", [0, 1])
def test_second_euler_step_adds_the_fstar_difference(mode):
    # The second step is forward Euler too, and it carries the time-derivative
    # terms as the difference of the dispersive fluxes of the last two levels:
    # applying the operator of Eqs. 9-10 / 19-20 to P^2, Q^2 returns
    # U*^1 + dt F^1 + (F*^1 - F*^0) and V*^1 + dt G^1 + (G*^1 - G*^0).  With the
    # sequential cross form (cross_mode 1) the F* difference is the exact one
    # across the step, F*(Q^2) - F*(Q^1).  Dropping the difference on this step,
    # or using the first step's zero, fails the comparison.
    case = W.barred_beach(nx=40, ny=36)
    rng = np.random.default_rng(11)
    P0 = 0.05 * rng.standard_normal((36, 40))
    Q0 = 0.03 * rng.standard_normal((36, 40))
    D = oracle.OracleDomain(dict(case["params"], bc=(0, 0, 0, 0), cross_mode=mode), case["bed"],
                            None, None, P0, Q0)
    r0 = D.rhs()
    dt = 1e-3
    D.step(dt)
    U1, V1 = D.apply_T()
    r1 = D.rhs()
    D.step(dt)
    U2, V2 = D.apply_T()
    beta, gam = D.last_weights()
    assert list(beta) == [dt, 0.0, 0.0]
    dFs = (D.rhs()["Fs"] - r1["Fs"]) if mode == 1 else (r1["Fs"] - r0["Fs"])
    dGs = r1["Gs"] - r0["Gs"]
    assert np.abs(dGs).max() > 1e-3 * np.abs(r1["Gs"]).max() > 0  # the difference is not negligible
    assert np.abs(dFs).max() > 1e-3 * np.abs(r1["Fs"]).max() > 0
    np.testing.assert_allclose(U2, U1 + dt * r1["F"] + dFs, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(V2, V1 + dt * r1["G"] + dGs, rtol=1e-12, atol=1e-14)
