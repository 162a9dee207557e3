"""Batched domains (bsq_batch_*): many uneven domains, one launch per stage,
each with its own adaptive dt.

* Each member's result in the mix is bitwise the result of the same domain
  run alone through the batched path (a batch of one), in FP32 and FP64, with
  a common step limit and with per-member t_end.
* In FP64, against the same domain on the single-domain path (other kernel
  shapes, so other rounding order): the same time and 1e-10 relative L2.
* An FP64 member follows the oracle's adaptive dt trace, and its state stays
  within 1e-10 of the oracle's.
* The single-precision grouped kernels that the batched throughput runs (more
  members than one launch group holds) against the FP64 oracle: fixed steps,
  a different step for each member, 1e-4 relative L2 in eta after 1000 steps.
* A failing member (non-finite state) stops alone; the others finish and are
  unchanged by it.
"""
import numpy as np
import pytest

import oracle
from paper_1909_04153_gb300 import bsq
from paper_1909_04153_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _members():
    # uneven shapes, ragged tails, both forcings, walls / makers / sponges
    return [
        W.random_basin(96, seed=11, forcing="solitary"),
        W.random_basin(160, seed=12, forcing="jonswap"),
        W.barred_beach(nx=130, ny=70),
        W.random_basin(64, seed=13, forcing="jonswap"),
        W.solitary_basin(nx=200, ny=9, dx=0.1),
    ]


def _fields(d):
    return {f: d.read(f) for f in ("eta", "P", "Q")}


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _alone(case, prec, **kw):
    """The domain run alone through the batched path (a batch of one)."""
    d = bsq.Domain(case, precision=prec, graph_steps=8)
    with bsq.Batch([d]) as b:
        n = b.advance(**kw)
    return d, int(n[0])


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batch_members_equal_alone_bitwise(prec):
    cases = _members()
    steps = 70
    doms = [bsq.Domain(c, precision=prec, graph_steps=8) for c in cases]
    with bsq.Batch(doms) as b:
        done = b.advance(max_steps=steps)
    assert list(done) == [steps] * len(cases)
    for c, d in zip(cases, doms):
        s, n = _alone(c, prec, max_steps=steps)
        assert n == steps
        i1, i2 = d.info(), s.info()
        assert i1["n"] == i2["n"] and i1["t"] == i2["t"] and i1["clamps"] == i2["clamps"]
        for k in ("eta", "P", "Q"):
            np.testing.assert_array_equal(d.read(k), s.read(k))
        # the single-domain path (other kernel shapes, other rounding order);
        # in FP64 that order is below the parity tolerance.  (In FP32 both
        # paths' kernels are held to the oracle by the kernel-variant tests.)
        if prec == "fp64":
            with bsq.Domain(c, precision=prec) as u:
                u.advance(max_steps=steps)
                assert abs(u.info()["t"] - i1["t"]) <= 1e-12 * i1["t"]
                for k in ("eta", "P", "Q"):
                    ref = u.read(k)
                    if np.linalg.norm(ref) > 0:
                        assert rel(d.read(k), ref) <= 1e-10, k
        s.close()
        d.close()


def test_batch_per_member_t_end():
    cases = _members()[:4]
    t_end = [0.05, 0.11, 0.07, 0.13]
    doms = [bsq.Domain(c, precision="fp32", graph_steps=8) for c in cases]
    with bsq.Batch(doms) as b:
        done = b.advance(t_end=t_end)
    for c, d, te, nd in zip(cases, doms, t_end, done):
        info = d.info()
        assert abs(info["t"] - te) <= 1e-12 * max(1.0, te)
        assert info["n"] == nd
        s, n = _alone(c, "fp32", t_end=[te])
        assert n == nd
        np.testing.assert_array_equal(s.read("eta"), d.read("eta"))
        s.close()
        d.close()


def test_batch_member_follows_oracle_dt_trace():
    case = W.random_basin(72, seed=21, forcing="jonswap")
    other = W.random_basin(40, seed=22, forcing="solitary")
    o = oracle.OracleDomain(case["params"], case["bed"], case["comps"], case["eta0"], case["P0"], case["Q0"])
    ref = []
    for _ in range(60):
        o.step()
        ref.append(o.info()["last_dt"])
    a = bsq.Domain(case, precision="fp64", graph_steps=4)
    z = bsq.Domain(other, precision="fp64", graph_steps=4)
    got = []
    with bsq.Batch([z, a]) as b:
        for _ in range(60):
            b.advance(max_steps=1)
            got.append(a.info()["last_dt"])
    np.testing.assert_allclose(got, ref, rtol=1e-8)
    for f in ("eta", "P", "Q"):
        assert rel(a.read(f), o.get(f)) <= 1e-10, f
    a.close()
    z.close()


def test_failing_member_stops_alone():
    cases = _members()[:3]
    bad = dict(cases[1])
    P0 = np.zeros((bad["params"]["ny"], bad["params"]["nx"]))
    P0[5, 7] = np.nan
    bad["P0"] = P0
    doms = [bsq.Domain(cases[0], precision="fp32", graph_steps=8), bsq.Domain(bad, precision="fp32", graph_steps=8),
            bsq.Domain(cases[2], precision="fp32", graph_steps=8)]
    with bsq.Batch(doms) as b:
        with pytest.raises(bsq.BsqError) as ei:
            b.advance(max_steps=40)
        assert ei.value.status == bsq.ERR_NONFINITE
    assert doms[0].info()["n"] == 40 and doms[2].info()["n"] == 40
    for q in (0, 2):
        s, n = _alone(cases[q], "fp32", max_steps=40)
        np.testing.assert_array_equal(s.read("eta"), doms[q].read("eta"))
        s.close()
    with pytest.raises(bsq.BsqError):  # sticky on the failed member
        doms[1].advance(max_steps=1)
    for d in doms:
        d.close()


def test_batch_rejects_mixed_precision_and_repeats():
    c = W.random_basin(48, seed=3)
    a = bsq.Domain(c, precision="fp32")
    z = bsq.Domain(c, precision="fp64")
    with pytest.raises(bsq.BsqError) as ei:
        bsq.Batch([a, z])
    assert ei.value.status == bsq.ERR_ARG
    with pytest.raises(bsq.BsqError):
        bsq.Batch([a, a])
    a.close()
    z.close()


def test_autotuned_batch_keeps_fp64_parity():
    cases = _members()[:4]
    doms = [bsq.Domain(c, precision="fp64", graph_steps=4) for c in cases]
    with bsq.Batch(doms) as b:
        ch = b.autotune(steps_per_trial=4)
        assert ch["rhs_rows"] in (32, 64) and ch["x_elements"] == 4 and ch["y_rows"] in (8, 16)
        b.advance(max_steps=20)
    for c, d in zip(cases, doms):
        n = d.info()["n"]
        with bsq.Domain(c, precision="fp64") as u:
            u.advance(max_steps=n)
            for k in ("eta", "P", "Q"):
                ref = u.read(k)
                if np.linalg.norm(ref) > 0:
                    assert rel(d.read(k), ref) <= 1e-10, k
        d.close()


def test_autotune_fp32_picks_a_shape():
    doms = [bsq.Domain(c, precision="fp32", graph_steps=4) for c in _members()[:3]]
    with bsq.Batch(doms) as b:
        ch = b.autotune(steps_per_trial=4)
        assert ch["x_elements"] in (4, 8)
        assert list(b.advance(max_steps=8)) == [8, 8, 8]
    for d in doms:
        d.close()


def test_batch_larger_than_one_rhs_group():
    # the single-precision RHS stage launches once per group of 48 members
    # (their descriptors are a kernel parameter); members of the first and of
    # the second group equal their batch-of-one results bitwise
    rng = np.random.default_rng(5)
    sides = [int(32 * rng.integers(1, 4)) for _ in range(53)]
    cases = [W.random_basin(n, seed=100 + k, forcing="solitary" if k % 2 else "jonswap")
             for k, n in enumerate(sides)]
    steps = 24
    doms = [bsq.Domain(c, precision="fp32", graph_steps=8) for c in cases]
    with bsq.Batch(doms) as b:
        done = b.advance(max_steps=steps)
    assert list(done) == [steps] * len(cases)
    for k in (0, 1, 47, 48, 52):
        s, n = _alone(cases[k], "fp32", max_steps=steps)
        assert n == steps
        assert doms[k].info()["t"] == s.info()["t"]
        for f in ("eta", "P", "Q"):
            np.testing.assert_array_equal(doms[k].read(f), s.read(f))
        s.close()
    for d in doms:
        d.close()


def test_batch_reset_keeps_members_independent():
    # bsq_batch_reset swaps members in place (buffers, shapes and graph kept,
    # the graph updated for the new tables): a member carried over keeps
    # stepping as if alone, a new member starts as if alone
    ca, cb, cc = (W.random_basin(96, seed=21, forcing="jonswap"), W.random_basin(64, seed=22),
                  W.barred_beach(nx=130, ny=70))
    da, db, dc = (bsq.Domain(c, precision="fp32", graph_steps=8) for c in (ca, cb, cc))
    with bsq.Batch([da, db]) as b:
        b.advance(max_steps=20)
        b.reset([db, dc])
        done = b.advance(max_steps=20)
        assert list(done) == [20, 20]
        assert b.launches_per_step() >= 5
    sb, n = _alone(cb, "fp32", max_steps=40)
    sc, m = _alone(cc, "fp32", max_steps=20)
    assert (n, m) == (40, 20)
    for f in ("eta", "P", "Q"):
        np.testing.assert_array_equal(db.read(f), sb.read(f))
        np.testing.assert_array_equal(dc.read(f), sc.read(f))
    for d in (da, db, dc, sb, sc):
        d.close()


def test_fp32_grouped_batch_matches_oracle():
    # 53 members: the single-precision RHS and x-line stages launch once per
    # group of 48 members (descriptors as a kernel parameter), so members sit
    # in both launches.  Each member takes fixed steps of its own size (cfl = 0,
    # dt_init: the constant-step AB3 of Eqs. 16-18 after the Euler start), which
    # the oracle replays.  JONSWAP members get a 1 s ramp and 3x the amplitude,
    # so that after 1000 steps their waves stand well above the single-precision
    # resolution of the depth (eta = h - d is formed from values of order d).
    rng = np.random.default_rng(5)
    sides = [int(32 * rng.integers(1, 4)) for _ in range(53)]
    cases = []
    for k, n in enumerate(sides):
        c = W.random_basin(n, seed=300 + k, forcing="solitary" if k % 2 else "jonswap")
        if c["comps"] is not None:
            c["params"]["ramp_time"] = 1.0
            c["comps"] = c["comps"].copy()
            c["comps"][:, 0] *= 3.0
        dt = (0.08 + 0.015 * (k % 3)) * c["params"]["dx"] / np.sqrt(W.G * -c["bed"].min())
        c["params"].update(cfl=0.0, dt_init=float(dt))
        cases.append(c)
    steps = 1000
    doms = [bsq.Domain(c, precision="fp32", kahan=True, graph_steps=16) for c in cases]
    with bsq.Batch(doms) as b:
        assert b.launches_per_step() == 7  # two RHS and two x-line launches
        done = b.advance(max_steps=steps)
    assert list(done) == [steps] * len(cases)
    for k in (0, 1, 47, 48, 52):  # both forcings, both launch groups
        c = cases[k]
        dt = c["params"]["dt_init"]
        assert abs(doms[k].info()["last_dt"] - dt) <= 1e-15
        o = oracle.OracleDomain(c["params"], c["bed"], c["comps"], c["eta0"], c["P0"], c["Q0"])
        o.run(steps, dts=[dt] * steps)
        e = rel(doms[k].read("eta"), o.get("eta"))
        assert e <= 1e-4, (k, e)
        for f in ("P", "Q"):
            assert rel(doms[k].read(f), o.get(f)) <= 1e-3, (k, f)
        assert doms[k].info()["clamps"] == o.info()["clamps"] == 0
    for d in doms:
        d.close()
