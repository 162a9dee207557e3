"""GPU path (through the C ABI) against the FP64 oracle, element by element.

With the oracle's dt sequence replayed (bsq_step_dt):
  * FP64 GPU within 1e-10 relative L2 of the oracle in eta, P and Q;
  * FP32 with compensated accumulation within 1e-4 relative L2 in eta after
    1000 steps.
Adaptive runs compare the dt traces.  Sizes span several stencil tiles,
several x-line segments and y-line chunks, and ragged tails.
"""
import numpy as np
import pytest

import oracle
from paper_1909_04153_gb300 import bsq
from paper_1909_04153_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
FP64_LINF = 1e-9  # largest cell error, relative to the field's largest magnitude
# a flux field that is zero in exact arithmetic (the transverse flux of a
# 1D run) stays at round-off: 2e-15 against a largest Q of 0.15 in the
# x-invariant column case, where a relative norm says nothing.  A flux field
# below ROUNDOFF_FLUX times the larger flux field's maximum is compared
# absolutely, against that maximum.
ROUNDOFF_FLUX = 1e-12


def flux_scale(o):
    return max(float(np.abs(o.get("P")).max()), float(np.abs(o.get("Q")).max()), 1e-300)
FP32_TOL = 1e-4


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def linf(a, b):
    """Largest cell error relative to the field's largest magnitude: unlike the
    relative L2 norm it is not diluted by the cells a boundary or corner error
    leaves alone."""
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _oracle(case, **over):
    p = dict(case["params"])
    p.update(over)
    return oracle.OracleDomain(p, case["bed"], case["comps"], case["eta0"], case["P0"], case["Q0"])


def _smooth_bed(nx, ny, dx, seed=3, lo=0.3, hi=1.1):
    rng = np.random.default_rng(seed)
    X, Y = np.meshgrid(np.arange(nx + 1) * dx, np.arange(ny + 1) * dx)
    b = np.zeros_like(X)
    for _ in range(4):
        kx, ky, ph = rng.uniform(0.1, 0.6), rng.uniform(0.1, 0.6), rng.uniform(0, 6.28)
        b += np.cos(kx * X + ph) * np.cos(ky * Y)
    b = (b - b.min()) / (b.max() - b.min())
    return -(lo + (hi - lo) * b)


def _hump_case(nx, ny, dx=0.1, seed=3):
    bed = _smooth_bed(nx, ny, dx, seed)
    xc, yc = (np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dx
    X, Y = np.meshgrid(xc, yc)
    eta = 0.06 * np.exp(-((X - 0.3 * nx * dx) ** 2 + (Y - 0.4 * ny * dx) ** 2) / (0.02 * (nx * dx) ** 2))
    return dict(params=W.base_params(nx, ny, dx, cfl=0.125), bed=bed, comps=None, eta0=eta, P0=None, Q0=None)


def _maker_case(nx, ny, bc, seed, dx=0.1):
    # oblique multi-component makers (directions seeded in +-0.7 rad) on the
    # given sides: every side's ghost layers, the corners and the boundary rows
    # of both line directions take maker values
    bed = _smooth_bed(nx, ny, dx, seed, lo=0.4, hi=0.9)
    comps = W.jonswap_components(0.02, 1.2, n=16, seed=seed)
    comps[:, 3] = np.random.default_rng(seed + 1).uniform(-0.7, 0.7, size=len(comps))
    sw = tuple(1.5 if b == W.SPONGE else 0.0 for b in bc)
    prm = W.base_params(nx, ny, dx, bc=bc, sponge_width=sw, ramp_time=2.0, cfl=0.125)
    return dict(params=prm, bed=bed, comps=comps, eta0=None, P0=None, Q0=None)


def _tall_solitary(nx, ny, dx=0.05, depth=0.6, amp=0.06):
    # a solitary wave travelling along y in a column taller than one pass of
    # the y-line chunk scan (more than 256 chunks of 8 rows); the 2D target CFL
    # of reading R2 (round-off across the column seeds the 2D modes that a
    # CFL of 0.2 lets grow)
    yc = (np.arange(ny) + 0.5) * dx
    eta1, q1 = W.solitary_profile(yc, 0.3 * ny * dx, amp, depth)
    bed = np.full((ny + 1, nx + 1), -depth)
    return dict(params=W.base_params(nx, ny, dx, cfl=0.125), bed=bed, comps=None,
                eta0=np.tile(eta1[:, None], (1, nx)), P0=None, Q0=np.tile(q1[:, None], (1, nx)))


CASES = {
    "hump_2d_walls": lambda: _hump_case(77, 45),
    "barred_beach_rips": lambda: W.barred_beach(nx=96, ny=72),
    "planar_beach_jonswap": lambda: W.planar_beach(nx=160, ny=20),
    "solitary_channel": lambda: W.solitary_basin(nx=129, ny=9, dx=0.1),
    "ragged_multi_segment": lambda: _hump_case(301, 37, dx=0.05, seed=5),
    "tall_multi_chunk": lambda: _hump_case(35, 530, dx=0.05, seed=7),
    "tall_multi_segment": lambda: _hump_case(19, 2309, dx=0.05, seed=17),
    "tall_solitary_multi_segment": lambda: _tall_solitary(12, 2309),
    "random_basin_jonswap": lambda: W.random_basin(64, seed=13, forcing="jonswap"),
    "hamm_rip_friction": lambda: W.hamm_rip(nx=100, ny=60),
    "makers_four_sides_oblique": lambda: _maker_case(70, 58, (W.MAKER,) * 4, seed=21),
    "makers_west_east_oblique": lambda: _maker_case(83, 47, (W.MAKER, W.MAKER, W.WALL, W.SPONGE), seed=23),
    "conical_island": lambda: W.conical_island(nx=121, ny=121),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_replay_matches_oracle(name):
    case = CASES[name]()
    steps = 150
    o = _oracle(case)
    dts = o.run(steps)
    with bsq.Domain(case, precision="fp64") as d:
        d.step_dt(dts)
        info = d.info()
        assert info["n"] == steps
        assert abs(info["t"] - o.info()["t"]) <= 1e-12 * o.info()["t"]
        for f in ("eta", "P", "Q"):
            ref, got = o.get(f), d.read(f)
            if f != "eta" and np.abs(ref).max() <= ROUNDOFF_FLUX * flux_scale(o):
                assert np.abs(got).max() <= 1e-11 * flux_scale(o), f
            else:
                assert rel(got, ref) <= FP64_TOL, (f, rel(got, ref))
                assert linf(got, ref) <= FP64_LINF, (f, linf(got, ref))
        assert info["clamps"] == o.info()["clamps"]


def test_fp64_extrapolated_cross_terms_match_oracle():
    # cross_mode 0 (both F*, G* extrapolated as in Eqs. 17-18 / 43) on a grid
    # where that form is stable (d/dx <= 1.1)
    case = _hump_case(64, 48, dx=1.0, seed=11)
    o = _oracle(case, cross_mode=0)
    dts = o.run(200)
    with bsq.Domain(case, precision="fp64", cross_mode=0) as d:
        d.step_dt(dts)
        for f in ("eta", "P", "Q"):
            assert rel(d.read(f), o.get(f)) <= FP64_TOL, f
            assert linf(d.read(f), o.get(f)) <= FP64_LINF, f


def test_fp32_extrapolated_cross_terms_match_oracle():
    # the printed form (cross_mode 0) through the single-precision kernels, on
    # the same stable grid, 1000 steps of the oracle's dt sequence
    case = _hump_case(64, 48, dx=1.0, seed=11)
    o = _oracle(case, cross_mode=0)
    dts = o.run(1000)
    with bsq.Domain(case, precision="fp32", kahan=True, cross_mode=0) as d:
        d.step_dt(dts)
        e = rel(d.read("eta"), o.get("eta"))
        assert e <= FP32_TOL, e
        for f in ("P", "Q"):
            assert rel(d.read(f), o.get(f)) <= 1e-3, f


def test_fp64_adaptive_dt_trace_matches_oracle():
    case = W.barred_beach(nx=80, ny=64)
    o = _oracle(case)
    ref = [o.step() or o.info()["last_dt"] for _ in range(120)]
    with bsq.Domain(case, precision="fp64", graph_steps=7) as d:
        got = []
        for _ in range(120):
            d.advance(max_steps=1)
            got.append(d.info()["last_dt"])
    np.testing.assert_allclose(got, ref, rtol=1e-8)


@pytest.mark.parametrize("prec,tol", [("fp64", FP64_TOL), ("fp32", FP32_TOL)])
def test_fixed_step_mode_matches_oracle_replay(prec, tol):
    # cfl = 0: every step is dt_init (the constant-step AB3 of Eqs. 16-18);
    # the oracle replays the same constant steps, landing on t_end
    case = CASES["hamm_rip_friction"]()
    dt, steps = 0.004, 300
    o = _oracle(case)
    o.run(steps, dts=[dt] * steps)
    with bsq.Domain(case, precision=prec, cfl=0.0, dt_init=dt) as d:
        n = d.advance(t_end=dt * steps)
        info = d.info()
        assert n == steps and abs(info["last_dt"] - dt) <= 1e-15
        assert abs(info["t"] - dt * steps) <= 1e-12
        assert rel(d.read("eta"), o.get("eta")) <= tol


def test_fp64_advance_lands_on_t_end_like_oracle():
    case = W.solitary_basin(nx=64, ny=12)
    o = _oracle(case)
    tr = o.advance(0.37)
    with bsq.Domain(case, precision="fp64", graph_steps=5) as d:
        n = d.advance(0.37)
        info = d.info()
    assert n == len(tr)
    assert abs(info["t"] - 0.37) <= 1e-14
    assert abs(info["last_dt"] - tr[-1]) <= 1e-8 * tr[-1]


@pytest.mark.parametrize("name", ["barred_beach_rips", "hump_2d_walls", "planar_beach_jonswap",
                                  "random_basin_jonswap", "hamm_rip_friction", "makers_four_sides_oblique",
                                  "makers_west_east_oblique", "tall_solitary_multi_segment", "conical_island"])
def test_fp32_kahan_1000_steps_matches_oracle(name):
    case = CASES[name]()
    o = _oracle(case)
    dts = o.run(1000)
    with bsq.Domain(case, precision="fp32", kahan=True) as d:
        d.step_dt(dts)
        e = rel(d.read("eta"), o.get("eta"))
        assert e <= FP32_TOL, e
        # fluxes reported, looser (the oracle itself only pins eta here); a flux
        # that is zero up to round-off in the oracle (Q of y-invariant runs, P
        # of x-invariant ones) is compared absolutely
        for f in ("P", "Q"):
            ref = o.get(f)
            if np.abs(ref).max() <= ROUNDOFF_FLUX * flux_scale(o):
                assert np.abs(d.read(f)).max() <= 1e-5 * flux_scale(o), f
            else:
                assert rel(d.read(f), ref) <= 1e-3, f


def test_fp32_without_kahan_runs():
    case = CASES["hump_2d_walls"]()
    o = _oracle(case)
    dts = o.run(300)
    with bsq.Domain(case, precision="fp32", kahan=False) as d:
        d.step_dt(dts)
        assert rel(d.read("eta"), o.get("eta")) <= 1e-3


# ------------------------------------------------------------------ invariants

def test_gpu_lake_at_rest_fp64_and_fp32():
    nx, ny, dx = 70, 50, 0.1
    case = dict(params=W.base_params(nx, ny, dx, cfl=0.125), bed=_smooth_bed(nx, ny, dx), comps=None,
                eta0=None, P0=None, Q0=None)
    with bsq.Domain(case, precision="fp64") as d:
        d.advance(max_steps=1000)
        assert np.abs(d.read("eta")).max() <= 1e-13
        assert np.abs(d.read("P")).max() <= 1e-13 and np.abs(d.read("Q")).max() <= 1e-13
    with bsq.Domain(case, precision="fp32") as d:
        d.advance(max_steps=1000)
        assert np.abs(d.read("eta")).max() <= 1e-5
        assert np.abs(d.read("P")).max() <= 1e-5


def test_gpu_mass_conservation_fp64():
    case = _hump_case(90, 66, seed=9)
    with bsq.Domain(case, precision="fp64") as d:
        m0 = d.info()["mass"]
        d.advance(max_steps=500)
        info = d.info()
        assert info["clamps"] == 0
        assert abs(info["mass"] - m0) <= 1e-12 * m0


@pytest.mark.parametrize("nx,ny", [(16384, 4), (4, 16384)])
def test_longest_lines_match_oracle(nx, ny):
    # the largest side bsq_create accepts: rows of 16384 cells take the x-solver
    # with 32 elements a thread (registers only), columns of 16384 cells a y-line
    # chunk scan of eight passes
    # The long rows carry a discharge ~1e4 times the cross-line one, so the
    # fluxes are held as one vector field (P, Q): the cross-line flux's own
    # norm would weigh round-off of the large terms 1e4 times over.
    case = _hump_case(nx, ny, dx=0.05, seed=29)
    o = _oracle(case)
    dts = o.run(20)
    with bsq.Domain(case, precision="fp64") as d:
        d.step_dt(dts)
        eta = d.read("eta")
        assert rel(eta, o.get("eta")) <= FP64_TOL
        assert linf(eta, o.get("eta")) <= FP64_LINF
        got = np.stack([d.read("P"), d.read("Q")])
        ref = np.stack([o.get("P"), o.get("Q")])
        assert rel(got, ref) <= FP64_TOL, rel(got, ref)
        assert linf(got, ref) <= FP64_LINF, linf(got, ref)
    with bsq.Domain(case, precision="fp32", kahan=True) as d:
        d.step_dt(dts)
        assert rel(d.read("eta"), o.get("eta")) <= FP32_TOL


def test_tiny_grid_3x3():
    case = _hump_case(3, 3, dx=0.2)
    o = _oracle(case)
    dts = o.run(30)
    with bsq.Domain(case, precision="fp64") as d:
        d.step_dt(dts)
        for f in ("eta", "P", "Q"):
            ref = o.get(f)
            got = d.read(f)
            assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max()), f


def test_checkpoint_restore_is_bitwise():
    case = W.barred_beach(nx=72, ny=40)
    for prec in ("fp32", "fp64"):
        with bsq.Domain(case, precision=prec) as a, bsq.Domain(case, precision=prec) as b:
            a.advance(max_steps=50)
            snap = a.checkpoint()
            a.advance(max_steps=60)
            b.restore(snap)
            b.advance(max_steps=60)
            for f in ("eta", "P", "Q"):
                np.testing.assert_array_equal(a.read(f), b.read(f))
            assert a.info()["t"] == b.info()["t"]


# ------------------------------------------------------------------ failure detection (host-made)

@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_nonfinite_input_is_reported(prec):
    # (double precision selects with integer keys, which carry a NaN on where
    # a floating compare would drop it: the state still ends up flagged)
    case = _hump_case(40, 30)
    P0 = np.zeros((30, 40))
    P0[10, 12] = np.nan
    case["P0"] = P0
    with bsq.Domain(case, precision=prec) as d:
        with pytest.raises(bsq.BsqError) as ei:
            d.advance(max_steps=5)
        assert ei.value.status == bsq.ERR_NONFINITE
        with pytest.raises(bsq.BsqError):  # sticky
            d.advance(max_steps=1)


def test_dt_below_dt_min_is_unstable():
    case = _hump_case(40, 30)
    with bsq.Domain(case, precision="fp64", dt_min=1.0) as d:
        with pytest.raises(bsq.BsqError) as ei:
            d.advance(max_steps=3)
        assert ei.value.status == bsq.ERR_UNSTABLE


def test_bounded_wait_times_out():
    case = W.barred_beach(nx=512, ny=512)
    with bsq.Domain(case, precision="fp64", timeout_s=1e-6) as d:
        with pytest.raises(bsq.BsqError) as ei:
            d.advance(max_steps=2000)
        assert ei.value.status == bsq.ERR_TIMEOUT


@pytest.mark.parametrize("tune", [(0, 0, 2, 0), (0, 0, 2, 0, 16), (0, 0, 8, 0, 4), (0, 0, 8, 0, 8), (0, 0, 0, 0, 4),
                                  (0, 0, 16, 0, 4), (0, 0, 16, 0, 8), (0, 0, 0, 0, 0, 0, 1), (0, 0, 0, 32, 0, 16),
                                  (0, 0, 0, 0, 0, 0, 2), (0, 0, 0, 32, 0, 0, 3), (0, 0, 0, 16),
                                  (0, 0, 0, 24), (0, 0, 0, 48), (0, 0, 0, 24, 0, 16), (0, 0, 0, 64),
                                  (0, 0, 0, 128)])
def test_kernel_variants_match_oracle(tune):
    # every kernel shape (paired or one-column RHS and its rows per warp,
    # warp-per-row, persistent staged or register x-solver and its elements
    # per lane, y-line chunk rows, chunk summaries inside the RHS kernel or by
    # their own kernel) gives the same step to FP64 round-off
    case = CASES["barred_beach_rips"]()
    o = _oracle(case)
    dts = o.run(80)
    with bsq.Domain(case, precision="fp64", tune=tune) as d:
        d.step_dt(dts)
        for f in ("eta", "P", "Q"):
            assert rel(d.read(f), o.get(f)) <= FP64_TOL, (tune, f)
            assert linf(d.read(f), o.get(f)) <= FP64_LINF, (tune, f)
    with bsq.Domain(case, precision="fp32", tune=tune) as d:
        d.step_dt(dts)
        assert rel(d.read("eta"), o.get("eta")) <= FP32_TOL, tune


def test_fp64_fma_rate_is_measured():
    # the FP64 roof of the double-precision path: a positive, finite rate
    # below the FP32 rate's order of magnitude
    r = bsq.fp64_fma_rate()
    assert 0.05 < r < 100.0, r


def test_fp32_maker_with_steps_above_a_25th_of_the_period():
    # fixed steps of 0.19-0.33 rad per step for the maker components: above
    # 1/4 rad the single-precision maker takes sin d and cos d - 1 in FP64
    # instead of their Taylor series; both branches run here
    nx, ny, dx, h = 48, 16, 0.5, 0.4
    bed = np.full((ny + 1, nx + 1), -h)
    comps = W.jonswap_components(0.05, 0.8, n=16, f0=1.0, df=0.05, seed=5)
    comps[:, 3] = np.random.default_rng(6).uniform(-0.5, 0.5, size=16)
    dt = 0.12 * dx / np.sqrt(W.G * h)
    od = 2 * np.pi * comps[:, 1] * dt
    assert (od > 0.25).any() and (od <= 0.25).any()
    prm = W.base_params(nx, ny, dx, bc=(W.MAKER, W.SPONGE, W.WALL, W.WALL), sponge_width=(0, 6.0, 0, 0),
                        ramp_time=2.0, cfl=0.0, dt_init=dt)
    case = dict(params=prm, bed=bed, comps=comps, eta0=None, P0=None, Q0=None)
    steps = 400
    o = _oracle(case)
    o.run(steps, dts=[dt] * steps)
    with bsq.Domain(case, precision="fp32") as d:
        assert d.advance(t_end=dt * steps) == steps
        # FP32 resolves eta to ~1e-7 of the depth; the waves here are ~6e-4 m rms
        assert rel(d.read("eta"), o.get("eta")) <= 1e-3


# ------------------------------------------------------------------ call boundaries

def test_step_slots_are_exact_and_calls_compose():
    # A call enqueues exactly its step slots (whole graphs of graph_steps,
    # then graphs of 1, 2, 4, ... steps): 37 steps in one call, in calls of
    # 16 + 21, in 37 single steps, and through bsq_step_dt with the same step
    # sizes give bitwise the same state, time and step count.
    case = W.barred_beach(nx=96, ny=72)
    with bsq.Domain(case, precision="fp32", graph_steps=16) as a:
        assert a.advance(max_steps=37) == 37
        sa = {f: a.read(f) for f in ("eta", "P", "Q")}
        ia = a.info()
    with bsq.Domain(case, precision="fp32", graph_steps=16) as b:
        assert b.advance(max_steps=16) == 16 and b.advance(max_steps=21) == 21
        for f in ("eta", "P", "Q"):
            np.testing.assert_array_equal(b.read(f), sa[f])
        assert b.info()["t"] == ia["t"] and b.info()["n"] == 37
    dts = []
    with bsq.Domain(case, precision="fp32", graph_steps=16) as c:
        for _ in range(37):
            assert c.advance(max_steps=1) == 1
            dts.append(c.info()["last_dt"])
        for f in ("eta", "P", "Q"):
            np.testing.assert_array_equal(c.read(f), sa[f])
        assert c.info()["t"] == ia["t"]
    with bsq.Domain(case, precision="fp32", graph_steps=16) as e:
        e.step_dt(dts)
        for f in ("eta", "P", "Q"):
            np.testing.assert_array_equal(e.read(f), sa[f])


def test_advance_to_t_end_after_restore_and_batch():
    # the controller state a call starts from is read again whenever other work
    # may have changed it: after a restore, and after a batched advance
    case = W.random_basin(64, seed=31, forcing="jonswap")
    with bsq.Domain(case, precision="fp32") as a, bsq.Domain(case, precision="fp32") as b:
        a.advance(max_steps=10)
        snap = a.checkpoint()
        a.advance(max_steps=30)
        a.restore(snap)
        assert a.info()["n"] == 10
        assert a.advance(max_steps=5) == 5 and a.info()["n"] == 15
        with bsq.Batch([b]) as bt:
            bt.advance(max_steps=12)
        assert b.info()["n"] == 12
        t_end = b.info()["t"] + 0.05
        assert b.advance(t_end=t_end) >= 1
        assert abs(b.info()["t"] - t_end) <= 1e-12 * max(1.0, t_end)
        assert b.advance(max_steps=3) == 3 and b.info()["n"] > 15


def test_read_into_caller_array():
    # bsq_read into a caller-owned array (here page-locked memory, as the end-to-end
    # benchmark passes it) gives the same values as into a new array; a wrong
    # shape or type is refused before any device work
    import torch

    case = W.barred_beach(nx=96, ny=72)
    with bsq.Domain(case, precision="fp32") as d:
        d.advance(max_steps=12)
        out = torch.empty((72, 96), dtype=torch.float64, pin_memory=True).numpy()
        for f in ("eta", "P", "Q", "h", "w"):
            np.testing.assert_array_equal(d.read(f, out=out), d.read(f))
        with pytest.raises(ValueError):
            d.read("eta", out=np.empty((96, 72)))
        with pytest.raises(ValueError):
            d.read("eta", out=np.empty((72, 96), dtype=np.float32))
