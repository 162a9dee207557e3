"""Host logic of the serving layer and of device-memory accounting (no GPU
work: bsq_domain_bytes and bsq_server_create/submit/request/release run on the
host only)."""
import ctypes

import pytest

from paper_1909_04153_gb300 import bsq
from paper_1909_04153_gb300 import workloads as W


def test_domain_bytes_grow_with_size_and_precision():
    small, big = W.random_basin(64, seed=1), W.random_basin(256, seed=1)
    p_small, _, _ = bsq.case_args(small)
    p_big, _, _ = bsq.case_args(big)
    p_big64, _, _ = bsq.case_args(big, precision="fp64")
    n_small, n_big, n_big64 = (bsq.bsq_domain_bytes(p, 0) for p in (p_small, p_big, p_big64))
    assert 0 < n_small < n_big < n_big64
    assert n_big >= 25 * 256 * 256 * 4  # at least the 25 fields of a cell-update
    p_small.nx = 1
    assert bsq.bsq_domain_bytes(p_small, 0) == 0


def test_submit_validation_and_states():
    case = W.random_basin(64, seed=2)
    with bsq.Server(hbm_budget=10 ** 9) as s:
        rid = s.submit(case, 1.0)
        assert rid > 0
        r = s.request(rid)
        assert r["state"] == bsq.REQ_PENDING and r["steps"] == 0
        with pytest.raises(bsq.BsqError) as ei:  # still queued
            s.release(rid)
        assert ei.value.status == bsq.ERR_STATE
        with pytest.raises(bsq.BsqError):
            s.read(rid, "eta")
        with pytest.raises(bsq.BsqError):
            s.request(rid + 100)
        for bad_t in (0.0, -1.0, float("inf"), float("nan")):
            with pytest.raises(bsq.BsqError):
                s.submit(case, bad_t)
        with pytest.raises(bsq.BsqError):  # non-default kernel shapes
            s.submit(dict(case, params=dict(case["params"], tune=(0, 0, 2))), 1.0)
    with bsq.Server(hbm_budget=10 ** 6) as tiny:  # larger than the whole budget
        with pytest.raises(bsq.BsqError) as ei:
            tiny.submit(W.random_basin(512, seed=2), 1.0)
        assert ei.value.status == bsq.ERR_ARG


def test_submit_rejects_other_precision():
    case = W.random_basin(64, seed=3)
    with bsq.Server(precision="fp64") as s:
        p, b, keep = bsq.case_args(case, precision="fp32")
        bed = bsq._f64(case["bed"])
        rid = ctypes.c_longlong()
        st = bsq.lib().bsq_server_submit(s.h, ctypes.byref(p), bsq._ptr(bed), ctypes.byref(b), None, None, None,
                                         1.0, ctypes.byref(rid))
        assert st == bsq.ERR_ARG and rid.value == 0
