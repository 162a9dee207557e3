"""Serving (bsq_server_*): continuous batching of requests of different grid
sizes and end times, admitted by slots and a device-memory budget.

* Requests arriving while others run join between rounds; every result is
  bitwise the result of the same request served alone; FP64 results are
  within 1e-10 of the single-domain path (whose kernels round in another
  order).
* The budget holds a request back until memory is released.
* A failing request finishes alone as failed.
"""
import numpy as np
import pytest

from paper_1909_04153_gb300 import bsq
from paper_1909_04153_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _requests():
    return [
        (W.random_basin(96, seed=31, forcing="solitary"), 0.6),
        (W.random_basin(160, seed=32, forcing="jonswap"), 0.9),
        (W.random_basin(64, seed=33, forcing="jonswap"), 0.4),
        (W.random_basin(128, seed=34, forcing="solitary"), 0.7),
    ]


def _serve_alone(case, t_end):
    with bsq.Server(steps_per_round=16) as s:
        rid = s.submit(case, t_end)
        while s.request(rid)["state"] in (bsq.REQ_PENDING, bsq.REQ_RUNNING):
            s.poll()
        r = s.request(rid)
        assert r["state"] == bsq.REQ_DONE
        return s.read(rid, "eta"), r


def test_results_same_alone_and_in_the_mix():
    reqs = _requests()
    with bsq.Server(steps_per_round=16) as s:
        ids = [s.submit(*reqs[0]), s.submit(*reqs[1])]
        s.poll()
        s.poll()
        ids.append(s.submit(*reqs[2]))  # arrives while the first two run
        s.poll()
        ids.append(s.submit(*reqs[3]))
        out = {}
        for _ in range(100000):
            nr, npd = s.poll()
            for q, rid in enumerate(ids):
                if q not in out and s.request(rid)["state"] == bsq.REQ_DONE:
                    out[q] = (s.read(rid, "eta"), s.request(rid))
                    s.release(rid)
            if len(out) == len(ids):
                break
        assert len(out) == len(ids)
        assert s.bytes_in_use() == 0
    for q, (case, t_end) in enumerate(reqs):
        eta, r = out[q]
        assert abs(r["t"] - t_end) <= 1e-12 * t_end
        alone, ra = _serve_alone(case, t_end)
        assert r["steps"] == ra["steps"]
        np.testing.assert_array_equal(eta, alone)


def test_fp64_requests_match_the_single_domain_path():
    reqs = _requests()[:2]
    with bsq.Server(steps_per_round=16, precision="fp64") as s:
        ids = [s.submit(*reqs[0])]
        s.poll()
        ids.append(s.submit(*reqs[1]))
        while any(s.request(i)["state"] in (bsq.REQ_PENDING, bsq.REQ_RUNNING) for i in ids):
            s.poll()
        for (case, t_end), rid in zip(reqs, ids):
            assert s.request(rid)["state"] == bsq.REQ_DONE
            with bsq.Domain(case, precision="fp64") as d:
                d.advance(t_end)
                for f in ("eta", "P", "Q"):
                    assert rel(s.read(rid, f), d.read(f)) <= 1e-10, f


def test_budget_holds_a_request_back_until_release():
    (a, ta), (b, tb) = _requests()[:2]
    pa, ba, _ = bsq.case_args(a)
    pb, bb, _ = bsq.case_args(b)
    need_a, need_b = bsq.bsq_domain_bytes(pa, ba.n_comp), bsq.bsq_domain_bytes(pb, bb.n_comp)
    with bsq.Server(hbm_budget=max(need_a, need_b) + min(need_a, need_b) - 1, steps_per_round=16) as s:
        ia, ib = s.submit(a, ta), s.submit(b, tb)
        s.poll()
        assert s.request(ia)["state"] == bsq.REQ_RUNNING and s.request(ib)["state"] == bsq.REQ_PENDING
        assert s.bytes_in_use() == need_a
        while s.request(ia)["state"] == bsq.REQ_RUNNING:
            s.poll()
        s.poll()
        assert s.request(ib)["state"] == bsq.REQ_PENDING  # a still holds its memory
        s.release(ia)
        s.poll()
        assert s.request(ib)["state"] in (bsq.REQ_RUNNING, bsq.REQ_DONE)
        while s.request(ib)["state"] == bsq.REQ_RUNNING:
            s.poll()
        assert s.request(ib)["state"] == bsq.REQ_DONE


def test_failing_request_finishes_alone():
    reqs = _requests()[:3]
    bad = dict(reqs[1][0])
    P0 = np.zeros((bad["params"]["ny"], bad["params"]["nx"]))
    P0[3, 4] = np.nan
    bad["P0"] = P0
    with bsq.Server(steps_per_round=16) as s:
        ids = [s.submit(reqs[0][0], reqs[0][1]), s.submit(bad, 0.5), s.submit(reqs[2][0], reqs[2][1])]
        for _ in range(100000):
            s.poll()
            if all(s.request(i)["state"] in (bsq.REQ_DONE, bsq.REQ_FAILED) for i in ids):
                break
        st = [s.request(i) for i in ids]
        assert st[1]["state"] == bsq.REQ_FAILED and st[1]["status"] == bsq.ERR_NONFINITE
        assert st[0]["state"] == bsq.REQ_DONE and st[2]["state"] == bsq.REQ_DONE
        for q in (0, 2):
            alone, _ = _serve_alone(reqs[q][0], reqs[q][1])
            np.testing.assert_array_equal(s.read(ids[q], "eta"), alone)
