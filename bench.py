"""Throughput of the adaptive-AB3 extended Boussinesq step on GB300.

One bench step = one full time step of the hot path (controller + ghost
cells, KP07 fluxes + dispersive terms + AB3 combine, y-line and x-line
tridiagonal solves, sponge, CFL reduction) over one domain.

Default workload: the barred beach with three rip channels, 2048 x 2048 cells,
FP32 with compensated accumulation (the large single-domain configuration;
its working set, ~0.5 GB, is far larger than the 129 MB L2, so no L2 flush is
needed between steps).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp64]
    python bench.py --impl reference ...   # the FP64 CPU oracle, bounded sample

Under torchrun each rank advances its own replica domain on its own GPU (no
data exchange); ``value`` is the sum over ranks of cell-updates / the slowest
rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1909_04153_gb300 import workloads as W  # noqa: E402

METRIC = "cell-updates/s"
# floating-point operations of one double-precision cell-update (2 per DFMA,
# 1 per DADD or DMUL; smsp__sass_thread_inst_executed_op_{dfma,dadd,dmul}_pred_on)
# and instructions of the FP64 pipe (sm__sass_thread_inst_executed_op_fp64_pred_on),
# counted with ncu on one launch of each kernel of the double-precision step on
# the 2048 x 2048 barred beach: RHS 411.7 flops (337.9 instructions), x-line
# solve 66.2 (52.6), y-line solve 8.3 (5.6), ghost cells 0.1 (summarised under
# profiles/)
FP64_FLOPS_PER_CELL = 486.3
FP64_INSTR_PER_CELL = 396.2
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 rate, beside the rate measured live (bsq_fp64_fma_rate)
# DRAM bytes per launch of the dominant kernel measured by ncu
# (dram__bytes_read.sum + dram__bytes_write.sum), keyed by
# (kernel, precision, nx, ny); the capture is summarised under profiles/
MEASURED_TRAFFIC = {("rhs_combine", "fp32", 2048, 2048): 285.918976e6 + 112.8192e6}
# algorithmic bytes per interior cell of each kernel (values the method needs it
# to read and write once: state, bed, compensation terms, history; the
# right-hand sides dU, dV of the line solves and the stored line factors are
# this design's intermediates and are not counted), per precision; the whole
# step in STEP_VALUES
KERNEL_VALUES = {"fp32": {"rhs_combine": 19, "ysolve": 4, "xsolve": 7},
                 "fp64": {"rhs_combine": 17, "ysolve": 2, "xsolve": 5}}
STEP_VALUES = {"fp32": 25, "fp64": 19}


def case_dims(workload, n):
    """Grid of the workload at size n: barred beach n x n, planar beach
    n x n/4, rip-channel beach n x 3n/2 (1000 x 1500 is the 0.02 m grid),
    conical island n x n (601 x 601 is the grid of Sec. 5.1)."""
    return {"barred_beach": (n, n), "planar_beach": (n, max(4, n // 4)), "hamm_rip": (n, 3 * n // 2),
            "conical_island": (n, n)}[workload]


def make_case(workload, n):
    nx, ny = case_dims(workload, n)
    if workload == "barred_beach":
        return W.barred_beach(nx=nx, ny=ny)
    if workload == "planar_beach":
        return W.planar_beach(nx=nx, ny=ny)
    if workload == "hamm_rip":
        return W.hamm_rip(nx=nx, ny=ny)
    if workload == "conical_island":
        return W.conical_island(nx=nx, ny=ny)
    raise ValueError(workload)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class _Nvml:
    """Read-only NVML queries through ctypes: the SM clock, its maximum and the
    active clock event (throttle) reason bits of one GPU."""

    # clock event reason bits of nvml.h
    REASONS = {0x8: "hw_slowdown", 0x40: "hw_thermal_slowdown", 0x20: "sw_thermal_slowdown",
               0x4: "sw_power_cap", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, cuda_index):
        import ctypes

        self.ct = ctypes
        self.L = ctypes.CDLL("libnvidia-ml.so.1")
        if self.L.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit")
        self.h = ctypes.c_void_p()
        ok = False
        try:
            import torch

            uuid = "GPU-" + str(torch.cuda.get_device_properties(cuda_index).uuid)
            ok = self.L.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.h)) == 0
        except Exception:
            ok = False
        if not ok:
            vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
            idx = cuda_index
            try:
                idx = int(vis.split(",")[cuda_index]) if vis else cuda_index
            except (ValueError, IndexError):
                pass
            if self.L.nvmlDeviceGetHandleByIndex_v2(idx, ctypes.byref(self.h)) != 0:
                raise RuntimeError("nvml handle")
        v = ctypes.c_uint()
        self.max_mhz = float(v.value) if self.L.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(v)) == 0 else 0.0

    def sample(self):
        v = self.ct.c_uint()
        r = self.ct.c_ulonglong()
        if self.L.nvmlDeviceGetClockInfo(self.h, 1, self.ct.byref(v)) != 0:
            return None
        fn = getattr(self.L, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.L.nvmlDeviceGetCurrentClocksThrottleReasons
        bits = r.value if fn(self.h, self.ct.byref(r)) == 0 else 0
        return float(v.value), bits


class Clocks:
    """SM clock and throttle reasons sampled during the timed region: an NVML
    poller thread (about one sample per millisecond, so a region of a few
    milliseconds is covered) and nvidia-smi every 200 ms beside it."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, interval_s=0.001):
        self.index = index
        self.interval_s = interval_s
        self.p = None
        self.nv = None
        self.samples = []
        self.lines = []

    def _poll(self):
        while not self._stop:
            smp = self.nv.sample()
            if smp is not None:
                self.samples.append(smp)
            time.sleep(self.interval_s)

    def __enter__(self):
        import threading

        try:
            self.nv = _Nvml(self.index)
            self._stop = False
            self.th = threading.Thread(target=self._poll, daemon=True)
            self.th.start()
        except Exception:
            self.nv = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.nv is not None:
            self._stop = True
            self.th.join(timeout=2)
        if self.p is not None:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(f) > 5 + k and f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        n_smi = len(sm)
        if self.nv is not None and self.samples:
            mx = max(mx, self.nv.max_mhz)
            for mhz, bits in self.samples:
                sm.append(mhz)
                for b, nm in _Nvml.REASONS.items():
                    if bits & b:
                        reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "nvml_samples": len(sm) - n_smi, "smi_samples": n_smi}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if os.environ.get("BSQ_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def max_over_ranks(v, pg, device=None):
    if pg is None:
        return v
    import torch

    t = torch.tensor([v], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(v, pg, device=None):
    if pg is None:
        return v
    import torch

    t = torch.tensor([v], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


def oracle_rate(case, seconds, max_steps=10 ** 9):
    """Cell-updates/s of the FP64 CPU oracle on one case, for about `seconds`."""
    import oracle

    p = case["params"]
    o = oracle.OracleDomain(p, case["bed"], case["comps"], case["eta0"], case["P0"], case["Q0"])
    o.step()  # warm
    n, t0 = 0, time.perf_counter()
    while n < max_steps:
        rc = o.step()
        if rc:
            raise RuntimeError("oracle step failed %d" % rc)
        n += 1
        if time.perf_counter() - t0 > seconds:
            break
    el = time.perf_counter() - t0
    return p["nx"] * p["ny"] * n / el, n, el


def run_reference(args):
    world, rank, local, pg = dist_setup()
    if rank != 0:
        return 0
    # each step: one oracle time step of a bounded sample of the workload (the
    # same layout on a coarser grid), sized so that warmup + steps take ~2 min
    import oracle

    probe = make_case(args.workload, 128)
    rate, _, _ = oracle_rate(probe, 3.0)
    budget = 120.0
    cells = max(32 * 32, min(args.n * args.n, rate * budget / max(1, args.steps + args.warmup)))
    n = int(max(32, min(args.n, math.sqrt(cells))))
    case = make_case(args.workload, n)
    p = case["params"]
    o = oracle.OracleDomain(p, case["bed"], case["comps"], case["eta0"], case["P0"], case["Q0"])
    for _ in range(args.warmup):
        o.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rc = o.step()
        if rc:
            raise RuntimeError("oracle step failed %d" % rc)
    el = time.perf_counter() - t0
    value = p["nx"] * p["ny"] * args.steps / el
    full = (p["nx"], p["ny"]) == case_dims(args.workload, args.n)
    sample = "%s %dx%d (%s), FP64, one oracle step per bench step, one thread" % (
        args.workload, p["nx"], p["ny"], "the full grid" if full else "same layout, coarser grid")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "%s_%dx%d" % ((args.workload,) + case_dims(args.workload, args.n)),
                   "sample_grid": [p["nx"], p["ny"]]},
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch

    from paper_1909_04153_gb300 import bsq

    world, rank, local, pg = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    case = make_case(args.workload, args.n)
    p = case["params"]
    ncell = p["nx"] * p["ny"]
    prec = args.precision
    fp = "fp32" if prec == "fp32" else "fp64"
    dom = bsq.Domain(case, precision=prec, kahan=(prec == "fp32"), stream=stream.cuda_stream,
                     graph_steps=args.graph_steps, tune=args.tune)
    # warm-up (also builds the CUDA graph)
    dom.advance(max_steps=args.warmup)
    torch.cuda.synchronize(dev)
    if pg is not None:
        pg.barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as ck:
        e0.record(stream)
        n = dom.advance(max_steps=args.steps)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    if n != args.steps:
        raise RuntimeError("took %d of %d steps" % (n, args.steps))
    ms = e0.elapsed_time(e1)
    if pg is not None:
        pg.barrier()
    ms_max = max_over_ranks(ms, pg, dev if pg is not None else None)
    total_cells = sum_over_ranks(float(ncell), pg, dev if pg is not None else None)
    value = total_cells * args.steps / (ms_max * 1e-3)
    clocks = ck.summary()

    # per-kernel durations, live, with CUDA events on the library's stream
    kms = dom.profile_kernels(args.profile_steps)
    top = max(("rhs_combine", "ysolve", "xsolve"), key=lambda k: kms[k])
    esize = 4 if fp == "fp32" else 8
    alg_bytes = KERNEL_VALUES[fp][top] * esize * ncell
    peak, peak_kind = peaks()
    achieved = alg_bytes / (kms[top] * 1e-3) / 1e9
    step_bytes = STEP_VALUES[fp] * esize
    step_achieved = value / world * step_bytes / 1e9
    info = dom.info()
    launches = dom.launches_per_step()
    dom.close()
    traffic = MEASURED_TRAFFIC.get((top, fp, p["nx"], p["ny"]))

    # the FP64 path on the same workload (ALU bound on GB300), short run
    fp64 = None
    if prec == "fp32" and not args.no_fp64:
        d64 = bsq.Domain(case, precision="fp64", stream=stream.cuda_stream, graph_steps=args.graph_steps)
        d64.advance(max_steps=5)
        torch.cuda.synchronize(dev)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        d64.advance(max_steps=args.fp64_steps)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        ms64 = f0.elapsed_time(f1) / args.fp64_steps
        k64 = d64.profile_kernels(3)
        d64.close()
        v64 = ncell / (ms64 * 1e-3)
        fl = FP64_FLOPS_PER_CELL * v64 / 1e12
        fma64 = bsq.fp64_fma_rate()
        # FP64 instructions issue at half the flop rate of fused multiply-adds
        ins = FP64_INSTR_PER_CELL * v64 / 1e12
        fp64 = {"value": v64, "unit": "cell-updates/s", "ms_per_step": ms64, "steps": args.fp64_steps,
                "kernel_ms": k64,
                "roofline": {"bound": "alu", "achieved": fl, "peak": fma64, "unit": "TFLOP/s",
                             "frac": fl / fma64, "peak_kind": "measured (FP64 FMA chains, bsq_fp64_fma_rate)",
                             "nominal_peak": FP64_PEAK_TFLOPS, "flops_per_cell": FP64_FLOPS_PER_CELL,
                             "fp64_instr_per_cell": FP64_INSTR_PER_CELL,
                             "fp64_issue_frac": ins / (fma64 / 2.0)}}

    # end to end through the C ABI with host buffers: create (uploads the
    # bathymetry and initial state from page-locked host arrays), advance, read
    # eta back into a page-locked host array
    def pinned(a):
        if a is None:
            return None
        t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
        t.numpy()[...] = a
        return t
    keep = {k: pinned(case.get(k)) for k in ("bed", "eta0", "P0", "Q0")}
    host_case = dict(case, **{k: (v.numpy() if v is not None else None) for k, v in keep.items()})
    out_t = torch.empty((p["ny"], p["nx"]), dtype=torch.float64, pin_memory=True)
    out = out_t.numpy()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    d2 = bsq.Domain(host_case, precision=prec, kahan=(prec == "fp32"), stream=stream.cuda_stream,
                    graph_steps=args.graph_steps, tune=args.tune)
    d2.advance(max_steps=args.steps)
    eta = d2.read("eta", out=out)
    t_e2e = time.perf_counter() - t0
    d2.close()
    t_e2e = max_over_ranks(t_e2e, pg, dev if pg is not None else None)
    h2d = 8 * ((p["nx"] + 1) * (p["ny"] + 1) + (3 if case["eta0"] is not None else 0) * ncell)
    e2e = {"value": total_cells * args.steps / t_e2e, "unit": "cell-updates/s",
           "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": eta.nbytes / args.steps,
           "includes": "bsq_create from page-locked host arrays + bsq_advance + bsq_read(eta) into a "
                       "page-locked host array"}

    batched = None
    if rank == 0 and prec == "fp32" and not args.no_batched:
        batched = run_batched(args, dev, stream)
    served = None
    if rank == 0 and prec == "fp32" and not args.no_served:
        served = run_served(args, dev, stream)
    fixed_vs_adaptive = None
    if rank == 0 and prec == "fp32" and not args.no_fixed_study:
        fixed_vs_adaptive = run_fixed_vs_adaptive(args, dev, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = run_cpu_baseline(args)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if fp == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": "%s_%dx%d" % (args.workload, p["nx"], p["ny"]), "precision": prec,
                       "kahan": prec == "fp32", "cross_mode": "sequential", "cfl": p["cfl"],
                       "cells": ncell, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "working set %.0f MB > 129 MB L2, no flush" % (
                           bsq_bytes_estimate(ncell, fp) / 1e6)},
            "roofline": {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": traffic, "bytes_per_cell": KERNEL_VALUES[fp][top] * esize},
            "step_roofline": {"bytes_per_cell_update": step_bytes, "achieved": step_achieved,
                              "frac": step_achieved / peak, "peak": peak},
            "kernel_ms": kms,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches * args.steps + 1,
            "launches_per_step": launches,
            "fp64": fp64,
            "batched": batched,
            "served": served,
            "fixed_vs_adaptive": fixed_vs_adaptive,
            "clocks": clocks,
            "sim": {"t": info["t"], "clamps": info["clamps"]},
        }
        print(json.dumps(line))
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()
    return 0


def cpu_model():
    """CPU model name and logical core count of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for l in out.splitlines():
            if l.startswith("Model name:"):
                model = l.split(":", 1)[1].strip()
                break
    except Exception:
        model = None
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for l in f:
                    if l.lower().startswith("model name"):
                        model = l.split(":", 1)[1].strip()
                        break
        except OSError:
            model = None
    import platform

    return model or platform.machine(), os.cpu_count() or 1


def run_cpu_baseline(args, seconds=6.0):
    """The FP64 oracle, as it stands, on the host cores: bounded samples of the
    solitary basin (256 x 64, its full 500 adaptive steps), the planar beach
    (1024 x 256, the first steps of its run) and the benchmark workload at full
    size (its first steps), each on one thread; then the planar-beach sample in
    one independent oracle process per core at once (replicas: the oracle
    itself stays single threaded)."""
    rows = []
    # (name, case, step cap, time cap): the solitary basin runs its 500 steps
    for name, case, cap, tmax in (("solitary_basin_256x64", W.solitary_basin(), 500, 60.0),
                                  ("planar_beach_1024x256", W.planar_beach(), 1000, seconds),
                                  ("%s_%dx%d" % ((args.workload,) + case_dims(args.workload, args.n)),
                                   make_case(args.workload, args.n), 200, seconds)):
        rate, nst, el = oracle_rate(case, tmax, max_steps=cap)
        rows.append({"workload": name, "steps": nst, "seconds": el, "value": rate, "cores": 1})
    model, ncpu = cpu_model()
    procs = [subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-worker", "planar_beach",
                               "--worker-seconds", str(seconds)], stdout=subprocess.PIPE,
                              stderr=subprocess.DEVNULL, text=True) for _ in range(ncpu)]
    total, ok = 0.0, 0
    for pr in procs:
        try:
            out, _ = pr.communicate(timeout=600)
            total += float(json.loads(out.strip().splitlines()[-1])["value"])
            ok += 1
        except Exception:
            pr.kill()
    head = rows[-1]
    return {"value": head["value"], "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
            "sample": "%s, %d FP64 steps in %.1f s, one thread (the full grid; the first steps of the run)" % (
                head["workload"], head["steps"], head["seconds"]),
            "cpu_model": model, "nproc": ncpu, "rows": rows,
            "all_cores": {"value": total, "unit": "cell-updates/s", "cores": ok, "kind": "oracle replicas",
                          "sample": "planar_beach_1024x256, one independent oracle process per core, "
                                    "about %.0f s each" % seconds}}


def oracle_worker(args):
    """One oracle process of the all-cores row (no GPU use)."""
    rate, nst, el = oracle_rate(make_case(args.oracle_worker, 1024), args.worker_seconds)
    print(json.dumps({"value": rate, "steps": nst, "seconds": el}))
    return 0


def run_batched(args, dev, stream):
    """64 independent FP32 basins (sides log-uniform in [128, 1024], multiples
    of 32) advanced as one batch, each with its own adaptive dt; beside it the
    same domains advanced one at a time on the single-domain path, in FP32
    and in FP64."""
    import torch

    from paper_1909_04153_gb300 import bsq

    cases = W.batch_cases(args.batch_domains, 128, 1024)
    cells = [c["params"]["nx"] * c["params"]["ny"] for c in cases]
    total = float(sum(cells))
    doms = [bsq.Domain(c, precision="fp32", stream=stream.cuda_stream, graph_steps=args.graph_steps)
            for c in cases]
    batch = bsq.Batch(doms, stream=stream.cuda_stream)
    tuned = batch.autotune(args.batch_tune_steps) if args.batch_tune_steps > 0 else None
    batch.advance(max_steps=10)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    done = batch.advance(max_steps=args.batch_steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    if not all(int(n) == args.batch_steps for n in done):
        raise RuntimeError("batched run: steps %s" % list(done))
    value = total * args.batch_steps / (ms * 1e-3)
    launches = batch.launches_per_step()
    batch.close()

    def one_at_a_time(ds, steps):
        el = 0.0
        for d in ds:
            d.advance(max_steps=2)
            torch.cuda.synchronize(dev)
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            d.advance(max_steps=steps)
            z.record(stream)
            torch.cuda.synchronize(dev)
            el += a.elapsed_time(z) * 1e-3
        return total * steps / el

    v32 = one_at_a_time(doms, args.batch_solo_steps)
    for d in doms:
        d.close()
    d64 = [bsq.Domain(c, precision="fp64", stream=stream.cuda_stream, graph_steps=args.graph_steps)
           for c in cases]
    v64 = one_at_a_time(d64, args.batch_fp64_steps)
    for d in d64:
        d.close()
    return {
        "workload": "%d random basins, sides log-uniform 128-1024 (multiples of 32), dx 0.1 m, depth 0.2-2 m, "
                    "solitary or JONSWAP maker (seeded 50/50)" % len(cases),
        "domains": len(cases), "cells": int(total), "precision": "fp32", "kahan": True,
        "value": value, "unit": "cell-updates/s", "ms_per_step": ms / args.batch_steps,
        "steps": args.batch_steps, "launches_per_step": launches, "autotuned_shapes": tuned,
        "gpu_launches": launches * args.batch_steps + 1,
        "one_at_a_time_fp32": {"value": v32, "unit": "cell-updates/s", "steps_each": args.batch_solo_steps},
        "one_at_a_time_fp64": {"value": v64, "unit": "cell-updates/s", "steps_each": args.batch_fp64_steps},
        "speedup_vs_fp64_one_at_a_time": value / v64,
        "speedup_vs_fp32_one_at_a_time": value / v32,
    }


def run_served(args, dev, stream):
    """A seeded Poisson stream of FP32 simulation requests (mean 20 per second,
    sides log-uniform in [64, 2048], multiples of 32, simulated durations
    uniform in [5, 60] s times --serve-time-scale, inputs as the batched
    basins), served with continuous batching under a device-memory budget;
    time-to-result is taken from each request's arrival to its result on the
    host."""
    import torch

    from paper_1909_04153_gb300 import bsq

    n = args.serve_requests
    rng = np.random.default_rng(W.SEED + 5)
    gaps = rng.exponential(1.0 / args.serve_rate, size=n)
    arrivals = np.cumsum(gaps) - gaps[0]
    sides = [int(max(32, round(v / 32) * 32)) for v in np.exp(rng.uniform(math.log(64), math.log(2048), size=n))]
    durations = rng.uniform(5.0, 60.0, size=n) * args.serve_time_scale
    kinds = rng.integers(0, 2, size=n)
    cases = [W.random_basin(s, seed=W.SEED + 500 + q, forcing="solitary" if kinds[q] == 0 else "jonswap")
             for q, s in enumerate(sides)]
    budget = int(args.serve_budget_gb * 1e9)
    srv = bsq.Server(hbm_budget=budget, max_slots=args.serve_slots, steps_per_round=args.serve_round,
                     stream=stream.cuda_stream)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    submitted, ids, done_at, steps, failed = 0, {}, {}, {}, 0
    h2d = d2h = 0
    max_running = max_pending = 0
    max_bytes = 0
    held_by_budget = held_by_slots = polls = 0  # polls that ended with requests still queued
    timeline, next_sample, area, last = [], 0.0, 0.0, 0.0
    while len(done_at) < n:
        now = time.perf_counter() - t0
        while submitted < n and arrivals[submitted] <= now:
            rid = srv.submit(cases[submitted], float(durations[submitted]))
            ids[rid] = submitted
            c = cases[submitted]
            h2d += 8 * ((c["params"]["nx"] + 1) * (c["params"]["ny"] + 1)
                        + sum(c[k].size for k in ("eta0", "P0", "Q0") if c.get(k) is not None))
            submitted += 1
        nr, npd = srv.poll()
        polls += 1
        max_running = max(max_running, nr)
        max_pending = max(max_pending, npd)
        used = srv.bytes_in_use()
        max_bytes = max(max_bytes, used)
        if npd > 0:
            if nr < args.serve_slots:
                held_by_budget += 1
            else:
                held_by_slots += 1
        now = time.perf_counter() - t0
        area += npd * (now - last)
        last = now
        if now >= next_sample:
            timeline.append([round(now, 2), nr, npd, round(used / 1e9, 3)])
            next_sample = now + args.serve_sample_s
        for rid, q in list(ids.items()):
            r = srv.request(rid)
            if r["state"] in (bsq.REQ_DONE, bsq.REQ_FAILED):
                if r["state"] == bsq.REQ_DONE:
                    eta = srv.read(rid, "eta")
                    d2h += eta.nbytes
                else:
                    failed += 1
                done_at[q] = time.perf_counter() - t0
                steps[q] = r["steps"]
                srv.release(rid)
                del ids[rid]
        if nr == 0 and npd == 0 and submitted < n:
            time.sleep(max(0.0, arrivals[submitted] - (time.perf_counter() - t0)))
    srv.close()
    lat = np.array([done_at[q] - arrivals[q] for q in range(n)])
    work = float(sum(sides[q] * sides[q] * steps[q] for q in range(n)))
    makespan = max(done_at.values()) - arrivals[0]
    return {
        "workload": "%d requests, Poisson arrivals %.0f/s, sides log-uniform 64-2048 (multiples of 32), "
                    "simulated durations U[5, 60] s x %g, random basins (solitary or JONSWAP maker)" % (
                        n, args.serve_rate, args.serve_time_scale),
        "precision": "fp32", "hbm_budget_bytes": budget, "max_slots": args.serve_slots,
        "steps_per_round": args.serve_round,
        "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
        "mean_s": float(lat.mean()),
        "value": work / makespan, "unit": "cell-updates/s",
        "offered": work / max(arrivals[-1] - arrivals[0], 1e-9),
        "makespan_s": makespan, "cell_updates": work, "failed": failed, "max_running": max_running,
        "max_pending": max_pending, "mean_pending": area / max(last, 1e-9), "max_bytes_in_use": max_bytes,
        "polls": polls, "polls_held_by_budget": held_by_budget, "polls_held_by_slots": held_by_slots,
        "timeline_t_running_pending_gb": timeline,
        "e2e_bytes": {"h2d": h2d, "d2h": d2h},
    }


def run_served_only(args):
    """The served workload alone (one GPU, rank 0): one JSON line with the
    served figures."""
    import torch

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    with Clocks(0, interval_s=0.05) as ck:
        served = run_served(args, dev, stream)
    line = {"metric": "served time-to-result and cell-updates/s", "served": served, "clocks": ck.summary()}
    print(json.dumps(line))
    return 0


def run_fixed_vs_adaptive(args, dev, stream):
    """Adaptive against fixed steps, FP32, on the rip-channel beach of Eq. 48
    (JONSWAP waves, friction; the default) or the conical island of Sec. 5.1
    (solitary run-up): the adaptive run to T gives its mean, smallest and
    largest step; fixed-step runs to the same T (cfl = 0, every step dt_init)
    locate, by bisection, the largest fixed step that stays stable (no
    non-finite state, |eta| below 1 m)."""
    import torch

    from paper_1909_04153_gb300 import bsq

    n = args.fixed_study_n
    T = args.fixed_study_time
    island = args.fixed_study_workload == "conical_island"
    case = W.conical_island(nx=n, ny=n) if island else W.hamm_rip(nx=n, ny=n * 3 // 2)
    p = case["params"]
    ncell = p["nx"] * p["ny"]

    def run(**over):
        """Advance to T; (stable, steps, wall seconds, smallest and largest step
        sampled every 64 steps)."""
        t0 = time.perf_counter()
        steps, lo_dt, hi_dt = 0, float("inf"), 0.0
        try:
            with bsq.Domain(case, precision="fp32", stream=stream.cuda_stream, **over) as d:
                while d.info()["t"] < T - 1e-9:
                    steps += d.advance(t_end=T, max_steps=64)
                    ldt = d.info()["last_dt"]
                    lo_dt, hi_dt = min(lo_dt, ldt), max(hi_dt, ldt)
                eta = d.read("eta")
                ok = bool(np.isfinite(eta).all() and np.abs(eta).max() < 1.0)
        except bsq.BsqError:
            ok = False
        torch.cuda.synchronize(dev)
        return ok, steps, time.perf_counter() - t0, lo_dt, hi_dt

    ok, steps_a, wall_a, lo_dt, hi_dt = run()
    mean_dt = T / steps_a
    lo, hi = 0.25 * mean_dt, 2.0 * mean_dt
    trials = []
    ok_lo = run(cfl=0.0, dt_init=lo)[0]
    ok_hi = run(cfl=0.0, dt_init=hi)[0]
    trials += [(lo, ok_lo), (hi, ok_hi)]
    if ok_lo and not ok_hi:
        for _ in range(6):
            mid = 0.5 * (lo + hi)
            ok_m = run(cfl=0.0, dt_init=mid)[0]
            trials.append((mid, ok_m))
            if ok_m:
                lo = mid
            else:
                hi = mid
    best = lo if ok_lo else None
    ok_f, steps_f, wall_f = run(cfl=0.0, dt_init=best)[:3] if best else (False, 0, 0.0)
    return {
        "workload": ("conical island of Sec. 5.1, %dx%d, dx %.3g m, solitary wave H/d 0.18, FP32, %g s simulated"
                     % (p["nx"], p["ny"], p["dx"], T)) if island else
                    ("rip-channel beach of Eq. 48, %dx%d, dx %.3g m, JONSWAP Hs 0.13 m Tp 1.6 s, friction 0.0025, "
                     "FP32, %g s simulated" % (p["nx"], p["ny"], p["dx"], T)),
        "adaptive": {"steps": steps_a, "mean_dt": mean_dt, "min_dt_sampled": lo_dt, "max_dt_sampled": hi_dt,
                     "cfl": p["cfl"], "wall_s": wall_a, "stable": ok},
        "largest_stable_fixed_dt": best,
        "fixed_to_mean_adaptive": (best / mean_dt) if best else None,
        "fixed": {"steps": steps_f, "wall_s": wall_f, "stable": ok_f},
        "adaptive_speedup_in_steps": (steps_f / steps_a) if best else None,
        "trials": [[float(a), bool(b)] for a, b in sorted(trials)],
        "cells": ncell,
    }


def bsq_bytes_estimate(ncell, fp):
    """Fields a domain holds per cell: FP32 31 (state and Kahan terms 7, history
    15, line-solve right-hand sides 2, bed 1, line factors 6); FP64 39 (state 4,
    the same 24, and 11 static terms of the RHS and the x-solver)."""
    return ncell * (31 if fp == "fp32" else 39) * (4 if fp == "fp32" else 8)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="barred_beach",
                    choices=["barred_beach", "planar_beach", "hamm_rip", "conical_island"])
    ap.add_argument("--n", "--grid", dest="n", type=int, default=2048)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--graph-steps", type=int, default=16)
    ap.add_argument("--profile-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=40)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-fixed-study", action="store_true")
    ap.add_argument("--fixed-study-n", type=int, default=500)
    ap.add_argument("--fixed-study-time", type=float, default=30.0)
    ap.add_argument("--fixed-study-workload", default="hamm_rip", choices=["hamm_rip", "conical_island"])
    ap.add_argument("--serve-requests", type=int, default=48)
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--serve-time-scale", type=float, default=0.1)
    ap.add_argument("--serve-budget-gb", type=float, default=4.0)
    ap.add_argument("--serve-slots", type=int, default=64)
    ap.add_argument("--serve-round", type=int, default=32)
    ap.add_argument("--serve-sample-s", type=float, default=0.25, help="queue timeline sampling interval")
    ap.add_argument("--serve-full", action="store_true",
                    help="the configured served workload: 256 requests, full durations U[5, 60] s, 8 GB budget "
                         "(about two minutes of GPU time); reported alone")
    ap.add_argument("--batch-domains", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=200)
    ap.add_argument("--batch-solo-steps", type=int, default=32)
    ap.add_argument("--batch-tune-steps", type=int, default=16)
    ap.add_argument("--batch-fp64-steps", type=int, default=16)
    ap.add_argument("--tune", type=lambda s: tuple(int(v) for v in s.split(",")), default=None,
                    help="kernel shape knobs (bsq_params.tune), comma separated")
    ap.add_argument("--oracle-worker", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--worker-seconds", type=float, default=6.0, help=argparse.SUPPRESS)
    args = ap.parse_args(argv)
    if args.oracle_worker:
        return oracle_worker(args)
    if args.serve_full:
        args.serve_requests, args.serve_time_scale, args.serve_budget_gb = 256, 1.0, 8.0
        args.serve_sample_s = max(args.serve_sample_s, 1.0)
        return run_served_only(args)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
