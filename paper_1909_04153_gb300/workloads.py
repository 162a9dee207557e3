"""Seeded synthetic inputs shaped like the paper's experiments (Sec. 5).

This module only builds inputs: bathymetry at cell corners, initial surface
elevation and fluxes, wave-maker component lists and run parameters.  It holds
none of the solver's arithmetic, so the CUDA library and the FP64 oracle can
both be driven from it.  The laboratory datasets of Sec. 5 are not available;
these generators stand in for them with the same kind of geometry and forcing:

* ``solitary_basin`` -- a solitary wave in a walled basin of constant depth
  (the shape of the solitary-wave cases of Secs. 5.1-5.2);
* ``planar_beach`` -- irregular JONSWAP waves running up a 1:20 planar beach
  with wetting and drying (the irregular-wave case of Sec. 5.4);
* ``barred_beach`` -- regular waves over a barred beach cut by three rip
  channels, sponge layers on three sides (the rip-current case of Sec. 5.3);
* ``random_basin`` -- smooth random bathymetry with solitary or JONSWAP
  forcing (for many independent domains);
* ``hamm_rip`` -- a plane beach cut by a rip channel, the analytic bathymetry
  of Eq. 48, irregular JONSWAP waves and quadratic bottom friction (the
  irregular-wave rip case of Sec. 5.4);
* ``conical_island`` -- a solitary wave (H/d = 0.18) running up a conical
  island in the centre of a square basin, with the geometry Sec. 5.1 states
  (the solitary run-up case of Sec. 5.1).

Each returns a dict: ``params`` (nx, ny, dx, dy, bc, ...), ``bed`` ((ny+1, nx+1)
corner elevations, datum = still water level, so ``w_s = 0``), ``comps``
((n, 4): amplitude m, frequency Hz, phase rad, direction rad), ``eta0``,
``P0``, ``Q0`` ((ny, nx) or None) and ``steps`` (the run length of the case).
"""
from __future__ import annotations

import math

import numpy as np

WALL, SPONGE, MAKER = 0, 1, 2
G = 9.81
SEED = 1909


def _grid(nx, ny, dx, dy):
    xc = (np.arange(nx) + 0.5) * dx
    yc = (np.arange(ny) + 0.5) * dy
    xk = np.arange(nx + 1) * dx
    yk = np.arange(ny + 1) * dy
    return xc, yc, xk, yk


def solitary_profile(x, x0, amp, depth):
    """Initial solitary hump eta = A sech^2(kappa (x - x0)), kappa = sqrt(3A/4h^3),
    flux P = c eta with c = sqrt(g (h + A))."""
    kappa = math.sqrt(3.0 * amp / (4.0 * depth ** 3))
    eta = amp / np.cosh(kappa * (x - x0)) ** 2
    c = math.sqrt(G * (depth + amp))
    return eta, c * eta


def jonswap_components(hs, tp, gamma=3.3, n=68, f0=None, df=0.01, seed=SEED, direction=0.0):
    """Discrete JONSWAP spectrum: n components spaced df apart (Sec. 5.4 uses
    68 components, df = 0.01 Hz), amplitudes sqrt(2 S df) scaled so that
    4 sqrt(m0) = Hs, seeded uniform random phases."""
    fp = 1.0 / tp
    if f0 is None:
        f0 = max(df, fp - 0.3)
    f = f0 + df * np.arange(n)
    sigma = np.where(f <= fp, 0.07, 0.09)
    r = np.exp(-((f - fp) ** 2) / (2.0 * sigma ** 2 * fp ** 2))
    S = G ** 2 * (2 * np.pi) ** -4 * f ** -5.0 * np.exp(-1.25 * (fp / f) ** 4) * gamma ** r
    a = np.sqrt(2.0 * S * df)
    m0 = 0.5 * np.sum(a ** 2)
    a *= hs / (4.0 * math.sqrt(m0))
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=n)
    return np.stack([a, f, ph, np.full(n, direction)], axis=1)


def base_params(nx, ny, dx, dy=None, **kw):
    p = dict(nx=int(nx), ny=int(ny), dx=float(dx), dy=float(dx if dy is None else dy),
             g=G, Bd=1.0 / 15.0, cfl=0.2, ema_alpha=0.1, dt_init=0.0, dt_min=1e-9,
             dt_max=0.0, friction=0.0, theta=1.0, eps=0.0, w_s=0.0, ramp_time=0.0, cross_mode=1,
             bc=(WALL, WALL, WALL, WALL), sponge_width=(0.0, 0.0, 0.0, 0.0))
    p.update(kw)
    return p


def solitary_basin(nx=256, ny=64, dx=0.1, depth=1.0, amp=0.1, x0=None, steps=500, **kw):
    """Solitary wave (A/h = 0.1) on constant depth between reflective walls."""
    xc, yc, xk, yk = _grid(nx, ny, dx, dx)
    if x0 is None:
        x0 = 0.5 * nx * dx
    bed = np.full((ny + 1, nx + 1), -depth)
    eta1, p1 = solitary_profile(xc, x0, amp, depth)
    eta0 = np.tile(eta1, (ny, 1))
    P0 = np.tile(p1, (ny, 1))
    return dict(name="solitary_basin", params=base_params(nx, ny, dx, **kw), bed=bed,
                comps=None, eta0=eta0, P0=P0, Q0=None, steps=steps)


def planar_beach(nx=1024, ny=256, length=51.2, depth=0.8, x_toe=15.0, slope=1.0 / 20.0,
                 hs=0.1, tp=2.0, gamma=3.3, n_comp=68, f0=0.20, steps=10000, seed=SEED, **kw):
    """Flat bed of depth 0.8 m, then a 1:20 slope to dry land (shoreline at
    x = 31 m for the full-size case); JONSWAP maker on the west side, walls
    elsewhere."""
    dx = length / nx
    xc, yc, xk, yk = _grid(nx, ny, dx, dx)
    b1 = -depth + np.maximum(xk - x_toe, 0.0) * slope
    bed = np.tile(b1, (ny + 1, 1))
    comps = jonswap_components(hs, tp, gamma, n_comp, f0=f0, seed=seed)
    kw.setdefault("cfl", 0.125)
    prm = base_params(nx, ny, dx, bc=(MAKER, WALL, WALL, WALL), ramp_time=5.0 * tp, **kw)
    return dict(name="planar_beach", params=prm, bed=bed, comps=comps, eta0=None, P0=None,
                Q0=None, steps=steps)


def barred_beach(nx=2048, ny=2048, length=51.2, depth=0.8, shore_x=45.0, slope=1.0 / 30.0,
                 bar_depth=0.3, bar_x=30.0, bar_sigma=1.0, rip_width=2.0, wave_h=0.1,
                 wave_t=1.5, sponge=3.0, steps=20000, **kw):
    """Barred beach with three rip channels (2 m wide) at y = L/4, L/2, 3L/4,
    regular waves from the west, sponge layers on the north, south and east."""
    dx = length / nx
    dy = length / ny
    xc, yc, xk, yk = _grid(nx, ny, dx, dy)
    X, Y = np.meshgrid(xk, yk)
    base = np.minimum(-depth + np.maximum(X - (shore_x - depth / slope), 0.0) * slope, 1.0)
    plain_depth_at_bar = (shore_x - bar_x) * slope
    bump = (plain_depth_at_bar - bar_depth) * np.exp(-(((X - bar_x) / bar_sigma) ** 2))
    cut = np.zeros_like(Y)
    for yr in (0.25 * length, 0.5 * length, 0.75 * length):
        cut = np.maximum(cut, np.exp(-(((Y - yr) / (0.5 * rip_width)) ** 8)))
    bed = base + bump * (1.0 - cut)
    comps = np.array([[0.5 * wave_h, 1.0 / wave_t, 0.0, 0.0]])
    kw.setdefault("cfl", 0.125)
    prm = base_params(nx, ny, dx, dy, bc=(MAKER, SPONGE, SPONGE, SPONGE),
                      sponge_width=(0.0, sponge, sponge, sponge), ramp_time=5.0 * wave_t, **kw)
    return dict(name="barred_beach", params=prm, bed=bed, comps=comps, eta0=None, P0=None,
                Q0=None, steps=steps)


def random_basin(n, dx=0.1, seed=SEED, forcing="solitary", sigma_cells=8.0, dmin=0.2, dmax=2.0,
                 steps=1000, **kw):
    """Square basin of side n with Gaussian-filtered random depth in [dmin, dmax]
    and either a solitary wave (A/h = 0.1) or a JONSWAP maker (Hs = 0.05 m,
    Tp = 2 s) on the west side; walls elsewhere."""
    kw.setdefault("cfl", 0.125)
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((n + 1, n + 1))
    kx = np.fft.fftfreq(n + 1)
    K2 = kx[None, :] ** 2 + kx[:, None] ** 2
    sm = np.real(np.fft.ifft2(np.fft.fft2(noise) * np.exp(-2.0 * (np.pi * sigma_cells) ** 2 * K2)))
    sm = (sm - sm.min()) / max(sm.max() - sm.min(), 1e-30)
    bed = -(dmin + (dmax - dmin) * sm)
    xc, yc, xk, yk = _grid(n, n, dx, dx)
    if forcing == "solitary":
        depth = float(-bed[:, : n // 4].mean())
        eta1, p1 = solitary_profile(xc, 0.25 * n * dx, 0.1 * depth, depth)
        eta0 = np.tile(eta1, (n, 1))
        P0 = np.tile(p1, (n, 1))
        prm = base_params(n, n, dx, **kw)
        return dict(name="random_basin", params=prm, bed=bed, comps=None, eta0=eta0, P0=P0,
                    Q0=None, steps=steps)
    comps = jonswap_components(0.05, 2.0, seed=seed + 1)
    prm = base_params(n, n, dx, bc=(MAKER, WALL, WALL, WALL), ramp_time=10.0, **kw)
    return dict(name="random_basin", params=prm, bed=bed, comps=comps, eta0=None, P0=None,
                Q0=None, steps=steps)


def hamm_rip_bed(x, y):
    """Bottom elevation of Eq. 48 (metres above still water): x onshore from the
    wave maker, y alongshore from the channel centre line."""
    s = 18.0 - x
    return 0.1 - s / 30.0 * (1.0 + 3.0 * np.exp(-s / 3.0) * np.cos(np.pi * y / 30.0) ** 10)


def hamm_rip(nx=1000, ny=1500, length=20.0, width=30.0, hs=0.13, tp=1.6, gamma=3.3, n_comp=68, f0=None,
             friction=0.0025, steps=20000, seed=SEED, **kw):
    """Plane beach with a rip channel (Eq. 48) over x in [0, length], y in
    [-width/2, width/2] (the channel at y = 0; the plane beach's shoreline at
    x = 15 m, about 0.5 m of water at the maker); JONSWAP maker on the west
    side (Hs = 0.13 m, Tp = 1.6 s, 68 components 0.01 Hz apart, seeded
    phases), quadratic friction f = 0.0025, first step 0.003 s, walls
    elsewhere.  The full size has the paper's 0.02 m cells."""
    dx = length / nx
    dy = width / ny
    xk = np.arange(nx + 1) * dx
    yk = np.arange(ny + 1) * dy - 0.5 * width
    X, Y = np.meshgrid(xk, yk)
    bed = hamm_rip_bed(X, Y)
    comps = jonswap_components(hs, tp, gamma, n_comp, f0=f0, seed=seed)
    kw.setdefault("cfl", 0.125)
    kw.setdefault("dt_init", 0.003)
    prm = base_params(nx, ny, dx, dy, bc=(MAKER, WALL, WALL, WALL), ramp_time=5.0 * tp, friction=friction, **kw)
    return dict(name="hamm_rip", params=prm, bed=bed, comps=comps, eta0=None, P0=None, Q0=None, steps=steps)


def conical_island(nx=601, ny=601, length=30.0, depth=0.32, base_radius=3.6, slope=0.25, amp_ratio=0.18,
                   x0=3.5, sponge=2.0, steps=7000, **kw):
    """Solitary wave run-up on a conical island (Sec. 5.1): a length x length
    basin (30 m, 601 x 601 cells at full size) of depth 0.32 m with an island of
    7.2 m base diameter and side slope 1/4 at its centre, here a full cone (its
    top is not given; the peak, 0.58 m above still water, stays dry); a solitary
    wave of H/d = 0.18 centred x0 from the west side travelling east; sponge
    layers west and east, walls north and south, no friction.  The paper runs it
    at CFL 0.145 with a first step of 0.0033 s; the 2D target CFL of this
    solver (0.125) is the default here."""
    dx = length / nx
    dy = length / ny
    xc, yc, xk, yk = _grid(nx, ny, dx, dy)
    X, Y = np.meshgrid(xk, yk)
    r = np.hypot(X - 0.5 * length, Y - 0.5 * length)
    bed = -depth + np.maximum(base_radius - r, 0.0) * slope
    eta1, p1 = solitary_profile(xc, x0, amp_ratio * depth, depth)
    kw.setdefault("cfl", 0.125)
    kw.setdefault("dt_init", 0.0033)
    prm = base_params(nx, ny, dx, dy, bc=(SPONGE, SPONGE, WALL, WALL), sponge_width=(sponge, sponge, 0.0, 0.0),
                      **kw)
    return dict(name="conical_island", params=prm, bed=bed, comps=None, eta0=np.tile(eta1, (ny, 1)),
                P0=np.tile(p1, (ny, 1)), Q0=None, steps=steps)


def batch_sizes(count=64, lo=128, hi=1024, seed=SEED, multiple=32):
    """Side lengths log-uniform in [lo, hi], rounded to a multiple of 32."""
    rng = np.random.default_rng(seed)
    s = np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))
    return [int(max(multiple, round(v / multiple) * multiple)) for v in s]


def batch_cases(count=64, lo=128, hi=1024, seed=SEED, dx=0.1, steps=1000, **kw):
    """Independent square basins for batched runs: sides from batch_sizes, each
    with its own seed, forcing drawn 50/50 (seeded) between a solitary wave and
    a JONSWAP maker."""
    rng = np.random.default_rng(seed + 7)
    sides = batch_sizes(count, lo, hi, seed)
    kinds = rng.integers(0, 2, size=count)
    return [random_basin(n, dx=dx, seed=seed + 100 + q, forcing="solitary" if kinds[q] == 0 else "jonswap",
                         steps=steps, **kw) for q, n in enumerate(sides)]


CASES = {
    "solitary_basin": solitary_basin,
    "planar_beach": planar_beach,
    "barred_beach": barred_beach,
    "hamm_rip": hamm_rip,
    "conical_island": conical_island,
}


def make(name: str, **kw) -> dict:
    return CASES[name](**kw)
