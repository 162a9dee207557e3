"""Python binding of the C ABI in ``include/bsq.h`` (ctypes, argument
marshalling only: every step of the solver runs in the CUDA library).

The functions keep the C names (``bsq_create``, ``bsq_advance``, ...).  The
:class:`Domain` wrapper bundles them for the tests and the benchmark.  Loading
fails loudly when the compiled library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NONFINITE, ERR_UNSTABLE, ERR_TIMEOUT, ERR_STATE = range(8)
FP32, FP64 = 0, 1
WALL, SPONGE, MAKER = 0, 1, 2
FIELDS = {"eta": 0, "P": 1, "Q": 2, "h": 3, "w": 4}


class bsq_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double),
        ("g", ctypes.c_double), ("Bd", ctypes.c_double),
        ("cfl", ctypes.c_double), ("ema_alpha", ctypes.c_double),
        ("dt_init", ctypes.c_double), ("dt_min", ctypes.c_double), ("dt_max", ctypes.c_double),
        ("friction", ctypes.c_double), ("theta", ctypes.c_double), ("eps", ctypes.c_double),
        ("w_s", ctypes.c_double), ("ramp_time", ctypes.c_double), ("timeout_s", ctypes.c_double),
        ("precision", ctypes.c_int), ("kahan", ctypes.c_int), ("cross_mode", ctypes.c_int),
        ("graph_steps", ctypes.c_int), ("tune", ctypes.c_int * 8),
    ]


_DP = ctypes.POINTER(ctypes.c_double)


class bsq_boundary(ctypes.Structure):
    _fields_ = [
        ("type", ctypes.c_int * 4), ("sponge_width", ctypes.c_double * 4),
        ("n_comp", ctypes.c_int),
        ("amp", _DP), ("freq", _DP), ("phase", _DP), ("dir", _DP),
    ]


class bsq_server_config(ctypes.Structure):
    _fields_ = [
        ("hbm_budget", ctypes.c_size_t), ("max_slots", ctypes.c_int), ("steps_per_round", ctypes.c_int),
        ("precision", ctypes.c_int), ("kahan", ctypes.c_int), ("cuda_stream", ctypes.c_void_p),
    ]


REQ_PENDING, REQ_RUNNING, REQ_DONE, REQ_FAILED = range(4)


class BsqError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__("%s: %s (status %d)" % (what, bsq_status_string(status), status))


_lib = None


def lib():
    """Load libbsq.so (building it first if the sources are newer)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path) or _build._stale():
            path = _build.build()
        L = ctypes.CDLL(path)
        vp, sz = ctypes.c_void_p, ctypes.c_size_t
        L.bsq_params_default.argtypes = [ctypes.POINTER(bsq_params)]
        L.bsq_create.restype = ctypes.c_int
        L.bsq_create.argtypes = [ctypes.POINTER(bsq_params), _DP, ctypes.POINTER(bsq_boundary), _DP, _DP, _DP,
                                 vp, ctypes.POINTER(vp)]
        L.bsq_advance.restype = ctypes.c_int
        L.bsq_advance.argtypes = [vp, ctypes.c_double, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]
        L.bsq_step_dt.restype = ctypes.c_int
        L.bsq_step_dt.argtypes = [vp, _DP, ctypes.c_longlong]
        L.bsq_read.restype = ctypes.c_int
        L.bsq_read.argtypes = [vp, ctypes.c_int, _DP]
        L.bsq_read_device.restype = ctypes.c_int
        L.bsq_read_device.argtypes = [vp, ctypes.c_int, vp]
        L.bsq_info.restype = ctypes.c_int
        L.bsq_info.argtypes = [vp, _DP, ctypes.POINTER(ctypes.c_longlong), _DP, _DP,
                               ctypes.POINTER(ctypes.c_longlong)]
        L.bsq_checkpoint.restype = ctypes.c_int
        L.bsq_checkpoint.argtypes = [vp, vp, ctypes.POINTER(sz)]
        L.bsq_restore.restype = ctypes.c_int
        L.bsq_restore.argtypes = [vp, vp, sz]
        L.bsq_destroy.argtypes = [vp]
        L.bsq_status_string.restype = ctypes.c_char_p
        L.bsq_status_string.argtypes = [ctypes.c_int]
        L.bsq_device_bytes.restype = sz
        L.bsq_device_bytes.argtypes = [vp]
        L.bsq_profile_kernels.restype = ctypes.c_int
        L.bsq_profile_kernels.argtypes = [vp, ctypes.c_longlong, _DP, ctypes.POINTER(ctypes.c_int)]
        L.bsq_kernel_name.restype = ctypes.c_char_p
        L.bsq_kernel_name.argtypes = [ctypes.c_int]
        L.bsq_launches_per_step.restype = ctypes.c_int
        L.bsq_launches_per_step.argtypes = [vp]
        L.bsq_fp64_fma_rate.restype = ctypes.c_int
        L.bsq_fp64_fma_rate.argtypes = [_DP]
        L.bsq_batch_create.restype = ctypes.c_int
        L.bsq_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp, ctypes.POINTER(vp)]
        L.bsq_batch_advance.restype = ctypes.c_int
        L.bsq_batch_advance.argtypes = [vp, _DP, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]
        L.bsq_batch_reset.restype = ctypes.c_int
        L.bsq_batch_reset.argtypes = [vp, ctypes.POINTER(vp), ctypes.c_int]
        L.bsq_batch_size.restype = ctypes.c_int
        L.bsq_batch_size.argtypes = [vp]
        L.bsq_batch_launches_per_step.restype = ctypes.c_int
        L.bsq_batch_launches_per_step.argtypes = [vp]
        L.bsq_batch_destroy.argtypes = [vp]
        L.bsq_batch_autotune.restype = ctypes.c_int
        L.bsq_batch_autotune.argtypes = [vp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int)]
        L.bsq_clock.restype = ctypes.c_int
        L.bsq_clock.argtypes = [vp, _DP, ctypes.POINTER(ctypes.c_longlong)]
        L.bsq_domain_bytes.restype = sz
        L.bsq_domain_bytes.argtypes = [ctypes.POINTER(bsq_params), ctypes.c_int]
        L.bsq_server_create.restype = ctypes.c_int
        L.bsq_server_create.argtypes = [ctypes.POINTER(bsq_server_config), ctypes.POINTER(vp)]
        L.bsq_server_submit.restype = ctypes.c_int
        L.bsq_server_submit.argtypes = [vp, ctypes.POINTER(bsq_params), _DP, ctypes.POINTER(bsq_boundary), _DP, _DP,
                                        _DP, ctypes.c_double, ctypes.POINTER(ctypes.c_longlong)]
        L.bsq_server_poll.restype = ctypes.c_int
        L.bsq_server_poll.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.bsq_server_request.restype = ctypes.c_int
        L.bsq_server_request.argtypes = [vp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int), _DP,
                                         ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_int)]
        L.bsq_server_read.restype = ctypes.c_int
        L.bsq_server_read.argtypes = [vp, ctypes.c_longlong, ctypes.c_int, _DP]
        L.bsq_server_release.restype = ctypes.c_int
        L.bsq_server_release.argtypes = [vp, ctypes.c_longlong]
        L.bsq_server_bytes_in_use.restype = sz
        L.bsq_server_bytes_in_use.argtypes = [vp]
        L.bsq_server_destroy.argtypes = [vp]
        L.bsq_mass_noalloc.restype = ctypes.c_int
        L.bsq_mass_noalloc.argtypes = [ctypes.c_int, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_longlong,
                                       ctypes.c_double, ctypes.c_double, vp, vp]
        _lib = L
    return _lib


# ---------------------------------------------------------------- C names

def bsq_status_string(s: int) -> str:
    return lib().bsq_status_string(int(s)).decode()


def bsq_params_default() -> bsq_params:
    p = bsq_params()
    lib().bsq_params_default(ctypes.byref(p))
    return p


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_DP)


def bsq_create(params: bsq_params, bed, boundary: bsq_boundary | None = None, eta0=None, P0=None, Q0=None,
               stream: int | None = None):
    h = ctypes.c_void_p()
    bed, eta0, P0, Q0 = (_f64(v) for v in (bed, eta0, P0, Q0))
    st = lib().bsq_create(ctypes.byref(params), _ptr(bed), ctypes.byref(boundary) if boundary else None,
                          _ptr(eta0), _ptr(P0), _ptr(Q0), ctypes.c_void_p(stream or 0), ctypes.byref(h))
    if st != OK:
        raise BsqError(st, "bsq_create")
    return h


def bsq_advance(h, t_end: float, max_steps: int = 0) -> int:
    n = ctypes.c_longlong()
    st = lib().bsq_advance(h, float(t_end), int(max_steps), ctypes.byref(n))
    if st != OK:
        raise BsqError(st, "bsq_advance")
    return n.value


def bsq_step_dt(h, dts) -> None:
    dts = _f64(dts)
    st = lib().bsq_step_dt(h, _ptr(dts), len(dts))
    if st != OK:
        raise BsqError(st, "bsq_step_dt")


def bsq_read(h, field: int, nx: int, ny: int, out=None) -> np.ndarray:
    """Field into ``out`` ((ny, nx) float64, C-contiguous; e.g. a view of
    page-locked memory) or a new array."""
    if out is None:
        out = np.empty((ny, nx), dtype=np.float64)
    elif out.shape != (ny, nx) or out.dtype != np.float64 or not out.flags.c_contiguous:
        raise ValueError("out must be a C-contiguous (ny, nx) float64 array")
    st = lib().bsq_read(h, int(field), _ptr(out))
    if st != OK:
        raise BsqError(st, "bsq_read")
    return out


def bsq_read_device(h, field: int, dev_ptr: int) -> None:
    st = lib().bsq_read_device(h, int(field), ctypes.c_void_p(dev_ptr))
    if st != OK:
        raise BsqError(st, "bsq_read_device")


def bsq_info(h) -> dict:
    t, dt, mass = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    n, cl = ctypes.c_longlong(), ctypes.c_longlong()
    st = lib().bsq_info(h, ctypes.byref(t), ctypes.byref(n), ctypes.byref(dt), ctypes.byref(mass),
                        ctypes.byref(cl))
    if st != OK:
        raise BsqError(st, "bsq_info")
    return dict(t=t.value, n=n.value, last_dt=dt.value, mass=mass.value, clamps=cl.value)


def bsq_checkpoint(h) -> bytes:
    n = ctypes.c_size_t()
    st = lib().bsq_checkpoint(h, None, ctypes.byref(n))
    if st != OK:
        raise BsqError(st, "bsq_checkpoint")
    buf = ctypes.create_string_buffer(n.value)
    st = lib().bsq_checkpoint(h, buf, ctypes.byref(n))
    if st != OK:
        raise BsqError(st, "bsq_checkpoint")
    return buf.raw[: n.value]


def bsq_restore(h, data: bytes) -> None:
    buf = ctypes.create_string_buffer(data, len(data))
    st = lib().bsq_restore(h, buf, len(data))
    if st != OK:
        raise BsqError(st, "bsq_restore")


def bsq_destroy(h) -> None:
    if h:
        lib().bsq_destroy(h)


def bsq_device_bytes(h) -> int:
    return lib().bsq_device_bytes(h)


def bsq_profile_kernels(h, n_steps: int) -> dict:
    ms = (ctypes.c_double * 8)()
    nk = ctypes.c_int()
    st = lib().bsq_profile_kernels(h, int(n_steps), ms, ctypes.byref(nk))
    if st != OK:
        raise BsqError(st, "bsq_profile_kernels")
    return {bsq_kernel_name(k): ms[k] for k in range(nk.value)}


def bsq_kernel_name(k: int) -> str:
    return lib().bsq_kernel_name(int(k)).decode()


def bsq_batch_create(handles, stream: int | None = None):
    arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    h = ctypes.c_void_p()
    st = lib().bsq_batch_create(arr, len(handles), ctypes.c_void_p(stream or 0), ctypes.byref(h))
    if st != OK:
        raise BsqError(st, "bsq_batch_create")
    return h


def bsq_batch_advance(h, n: int, t_end=None, max_steps: int = 0) -> np.ndarray:
    te = None if t_end is None else _f64(np.broadcast_to(np.asarray(t_end, dtype=np.float64), (n,)))
    steps = (ctypes.c_longlong * n)()
    st = lib().bsq_batch_advance(h, _ptr(te), int(max_steps), steps)
    if st != OK:
        raise BsqError(st, "bsq_batch_advance")
    return np.array(steps[:], dtype=np.int64)


def bsq_batch_destroy(h) -> None:
    if h:
        lib().bsq_batch_destroy(h)


NOALLOC_MAX_ROWS = 16384


def bsq_mass_noalloc(precision: int, w_dev: int, b_dev: int, nx: int, ny: int, pitch: int, dx: float, dy: float,
                     mass_dev: int, stream: int | None = None) -> None:
    """Volume of caller-owned device arrays into a caller-owned device double;
    allocates nothing (scratch is a fixed static device array)."""
    st = lib().bsq_mass_noalloc(int(precision), ctypes.c_void_p(w_dev), ctypes.c_void_p(b_dev), int(nx), int(ny),
                                int(pitch), float(dx), float(dy), ctypes.c_void_p(mass_dev),
                                ctypes.c_void_p(stream or 0))
    if st != OK:
        raise BsqError(st, "bsq_mass_noalloc")


# ---------------------------------------------------------------- wrapper

_PKEYS = ("g", "Bd", "cfl", "ema_alpha", "dt_init", "dt_min", "dt_max", "friction", "theta", "eps", "w_s",
          "ramp_time", "timeout_s")


def case_args(case: dict, precision: str = "fp32", kahan: bool = True, **overrides):
    """bsq_params and bsq_boundary of a workload dict (see ``workloads``); the
    third value keeps the component arrays the boundary points to alive."""
    prm = dict(case["params"])
    prm.update(overrides)
    p = bsq_params_default()
    p.nx, p.ny = int(prm["nx"]), int(prm["ny"])
    p.dx, p.dy = float(prm["dx"]), float(prm["dy"])
    for k in _PKEYS:
        if k in prm:
            setattr(p, k, float(prm[k]))
    p.precision = FP64 if precision == "fp64" else FP32
    p.kahan = 1 if kahan else 0
    p.cross_mode = int(prm.get("cross_mode", 1))
    if "graph_steps" in prm:
        p.graph_steps = int(prm["graph_steps"])
    for q, v in enumerate(prm.get("tune", ()) or ()):
        p.tune[q] = int(v)
    b = bsq_boundary()
    bc = prm.get("bc", (WALL, WALL, WALL, WALL))
    sw = prm.get("sponge_width", (0.0, 0.0, 0.0, 0.0))
    for s in range(4):
        b.type[s] = int(bc[s])
        b.sponge_width[s] = float(sw[s])
    comps = case.get("comps")
    keep = None
    if comps is not None and len(comps):
        c = np.ascontiguousarray(np.asarray(comps, dtype=np.float64).T)
        keep = c
        b.n_comp = c.shape[1]
        b.amp, b.freq, b.phase, b.dir = (_ptr(c[k]) for k in range(4))
    return p, b, keep


class Domain:
    """A domain on the GPU built from a workload dict (see ``workloads``):
    ``params`` (nx, ny, dx, dy, bc, sponge_width, ...), ``bed`` corners,
    ``comps`` ((n, 4) amplitude, frequency Hz, phase, direction), ``eta0``,
    ``P0``, ``Q0``.  ``precision`` is "fp32" or "fp64"."""

    def __init__(self, case: dict, precision: str = "fp32", kahan: bool = True, stream: int | None = None,
                 **overrides):
        p, b, self._comps = case_args(case, precision, kahan, **overrides)
        self.nx, self.ny = p.nx, p.ny
        self.precision = precision
        self.params = p
        self.h = bsq_create(p, case["bed"], b, case.get("eta0"), case.get("P0"), case.get("Q0"), stream)

    def close(self):
        if getattr(self, "h", None):
            bsq_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def advance(self, t_end: float = float("inf"), max_steps: int = 0) -> int:
        return bsq_advance(self.h, t_end, max_steps)

    def step_dt(self, dts) -> None:
        bsq_step_dt(self.h, dts)

    def read(self, field: str, out=None) -> np.ndarray:
        return bsq_read(self.h, FIELDS[field], self.nx, self.ny, out)

    def read_device(self, field: str, dev_ptr: int) -> None:
        bsq_read_device(self.h, FIELDS[field], dev_ptr)

    def info(self) -> dict:
        return bsq_info(self.h)

    def checkpoint(self) -> bytes:
        return bsq_checkpoint(self.h)

    def restore(self, data: bytes) -> None:
        bsq_restore(self.h, data)

    def device_bytes(self) -> int:
        return bsq_device_bytes(self.h)

    def profile_kernels(self, n_steps: int) -> dict:
        return bsq_profile_kernels(self.h, n_steps)

    def launches_per_step(self) -> int:
        return lib().bsq_launches_per_step(self.h)


class Batch:
    """Several :class:`Domain` objects advanced together, one launch per stage
    (``bsq_batch_*``).  The domains stay usable on their own between calls and
    must outlive the batch."""

    def __init__(self, domains, stream: int | None = None):
        self.domains = list(domains)
        self.h = bsq_batch_create([d.h for d in self.domains], stream)

    def advance(self, t_end=None, max_steps: int = 0) -> np.ndarray:
        """Per-domain steps taken; t_end is one time for all, a sequence of
        per-domain times, or None (then max_steps > 0)."""
        return bsq_batch_advance(self.h, len(self.domains), t_end, max_steps)

    def reset(self, domains):
        """Replace the members (bsq_batch_reset): buffers, tile shapes and the
        executable graph are kept."""
        domains = list(domains)
        arr = (ctypes.c_void_p * len(domains))(*[d.h.value if isinstance(d.h, ctypes.c_void_p) else d.h
                                                  for d in domains])
        st = lib().bsq_batch_reset(self.h, arr, len(domains))
        if st != OK:
            raise BsqError(st, "bsq_batch_reset")
        self.domains = domains

    def launches_per_step(self) -> int:
        return lib().bsq_batch_launches_per_step(self.h)

    def autotune(self, steps_per_trial: int = 16) -> dict:
        """Pick the fastest tile shapes on this batch (advances every member)."""
        ch = (ctypes.c_int * 3)()
        st = lib().bsq_batch_autotune(self.h, int(steps_per_trial), ch)
        if st != OK:
            raise BsqError(st, "bsq_batch_autotune")
        return dict(rhs_rows=ch[0], x_elements=ch[1], y_rows=ch[2])

    def close(self):
        if getattr(self, "h", None):
            bsq_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def bsq_clock(h) -> tuple:
    t, n = ctypes.c_double(), ctypes.c_longlong()
    st = lib().bsq_clock(h, ctypes.byref(t), ctypes.byref(n))
    return t.value, n.value, st


def fp64_fma_rate() -> float:
    """Measured FP64 FMA rate of the current device, TFLOP/s (bsq_fp64_fma_rate)."""
    v = ctypes.c_double()
    st = lib().bsq_fp64_fma_rate(ctypes.byref(v))
    if st != OK:
        raise BsqError(st, "bsq_fp64_fma_rate")
    return v.value


def bsq_domain_bytes(params: bsq_params, n_comp: int = 0) -> int:
    return lib().bsq_domain_bytes(ctypes.byref(params), int(n_comp))


class Server:
    """Continuous batching of simulation requests (``bsq_server_*``)."""

    def __init__(self, hbm_budget: int = 0, max_slots: int = 64, steps_per_round: int = 32,
                 precision: str = "fp32", kahan: bool = True, stream: int | None = None):
        cfg = bsq_server_config()
        cfg.hbm_budget = int(hbm_budget)
        cfg.max_slots = int(max_slots)
        cfg.steps_per_round = int(steps_per_round)
        cfg.precision = FP64 if precision == "fp64" else FP32
        cfg.kahan = 1 if kahan else 0
        cfg.cuda_stream = stream or 0
        self.precision, self.kahan = precision, kahan
        self._shape = {}
        h = ctypes.c_void_p()
        st = lib().bsq_server_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != OK:
            raise BsqError(st, "bsq_server_create")
        self.h = h

    def submit(self, case: dict, t_end: float) -> int:
        p, b, keep = case_args(case, self.precision, self.kahan)
        arrs = [_f64(case.get(k)) for k in ("bed", "eta0", "P0", "Q0")]
        rid = ctypes.c_longlong()
        st = lib().bsq_server_submit(self.h, ctypes.byref(p), _ptr(arrs[0]), ctypes.byref(b), _ptr(arrs[1]),
                                     _ptr(arrs[2]), _ptr(arrs[3]), float(t_end), ctypes.byref(rid))
        del keep
        if st != OK:
            raise BsqError(st, "bsq_server_submit")
        self._shape[rid.value] = (p.nx, p.ny)
        return rid.value

    def poll(self) -> tuple:
        nr, npd = ctypes.c_int(), ctypes.c_int()
        st = lib().bsq_server_poll(self.h, ctypes.byref(nr), ctypes.byref(npd))
        if st != OK:
            raise BsqError(st, "bsq_server_poll")
        return nr.value, npd.value

    def request(self, rid: int) -> dict:
        state, stat = ctypes.c_int(), ctypes.c_int()
        t, n = ctypes.c_double(), ctypes.c_longlong()
        st = lib().bsq_server_request(self.h, int(rid), ctypes.byref(state), ctypes.byref(t), ctypes.byref(n),
                                      ctypes.byref(stat))
        if st != OK:
            raise BsqError(st, "bsq_server_request")
        return dict(state=state.value, t=t.value, steps=n.value, status=stat.value)

    def read(self, rid: int, field: str) -> np.ndarray:
        nx, ny = self._shape[rid]
        out = np.empty((ny, nx), dtype=np.float64)
        st = lib().bsq_server_read(self.h, int(rid), FIELDS[field], _ptr(out))
        if st != OK:
            raise BsqError(st, "bsq_server_read")
        return out

    def release(self, rid: int) -> None:
        st = lib().bsq_server_release(self.h, int(rid))
        if st != OK:
            raise BsqError(st, "bsq_server_release")
        self._shape.pop(rid, None)

    def bytes_in_use(self) -> int:
        return lib().bsq_server_bytes_in_use(self.h)

    def close(self):
        if getattr(self, "h", None):
            lib().bsq_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
