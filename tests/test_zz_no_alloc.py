"""The allocation-free volume entry point (bsq_mass_noalloc) against the
regular one (bsq_info's mass), through the C ABI on the GPU.

Callers that cannot call cudaMalloc (an application that owns all device
memory through its own pool, or a stream being captured into a CUDA graph by
another component) use bsq_mass_noalloc with their own buffers; its scratch
is a fixed static device array.  This file is collected last so that a run
stopping at its first failure has already run every other test."""
import numpy as np
import pytest

from paper_1909_04153_gb300 import bsq
from paper_1909_04153_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mass_noalloc_matches_regular_mass_twice(precision):
    import torch

    case = W.barred_beach(nx=96, ny=80)
    p = case["params"]
    tol = 1e-12 if precision == "fp64" else 1e-6
    dt = torch.float64 if precision == "fp64" else torch.float32
    with bsq.Domain(case, precision=precision) as d:
        d.advance(max_steps=40)
        ref = d.info()["mass"]
        w = d.read("w")
        h = d.read("h")
        # bed from the state: h = max(w - b, 0) and w >= b everywhere
        wd = torch.tensor(w, dtype=dt, device="cuda")
        bd = torch.tensor(w - h, dtype=dt, device="cuda")
        out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream()
        prec = bsq.FP64 if precision == "fp64" else bsq.FP32
        for k in range(2):  # two calls in a row share the static scratch
            bsq.bsq_mass_noalloc(prec, wd.data_ptr(), bd.data_ptr(), p["nx"], p["ny"], p["nx"], p["dx"], p["dy"],
                                 out[k:].data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
    assert got[0] == got[1]
    assert abs(got[0] - ref) <= tol * ref, (got, ref)


def test_mass_noalloc_rejects_too_many_rows():
    with pytest.raises(bsq.BsqError) as ei:
        bsq.bsq_mass_noalloc(bsq.FP64, 16, 16, 8, bsq.NOALLOC_MAX_ROWS + 1, 8, 0.1, 0.1, 16)
    assert ei.value.status == bsq.ERR_ARG
