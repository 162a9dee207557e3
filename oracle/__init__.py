"""FP64 CPU oracle for the adaptive-AB3 extended Boussinesq step (arXiv 1909.04153).

TEST INFRASTRUCTURE ONLY.  This package is the reference the CUDA library is
checked against; it may be loaded by the tests, by the smoke check and by the
CPU-baseline leg of the benchmark, and by nothing else.  It shares no code with
the CUDA path: the numerics live in ``bsq_oracle.c`` (plain C, double
precision, one thread, built with ``-O2 -ffp-contract=off``) and this module
only compiles it and marshals arrays through ctypes.

Every function of the C file cites the equation or section of the paper it
follows; the readings of silent or garbled passages are listed at its top.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bsq_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liborcl.so")
_lock = threading.Lock()
_lib = None

WALL, SPONGE, MAKER = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2 -ffp-contract=off)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-shared", "-fPIC",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double),
        ("g", ctypes.c_double), ("Bd", ctypes.c_double),
        ("cfl", ctypes.c_double), ("ema_alpha", ctypes.c_double),
        ("dt_init", ctypes.c_double), ("dt_min", ctypes.c_double),
        ("dt_max", ctypes.c_double), ("friction", ctypes.c_double),
        ("theta", ctypes.c_double), ("eps", ctypes.c_double),
        ("w_s", ctypes.c_double), ("ramp_time", ctypes.c_double),
        ("cross_mode", ctypes.c_int),
        ("bc", ctypes.c_int * 4), ("sponge_width", ctypes.c_double * 4),
    ]


_D = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_create.restype = ctypes.c_void_p
            L.orc_create.argtypes = [ctypes.POINTER(_Params), _D, ctypes.c_int, _D, _D, _D, _D]
            L.orc_destroy.argtypes = [ctypes.c_void_p]
            L.orc_step.restype = ctypes.c_int
            L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double]
            L.orc_get.restype = ctypes.c_int
            L.orc_get.argtypes = [ctypes.c_void_p, ctypes.c_int, _D]
            L.orc_set_state.argtypes = [ctypes.c_void_p, _D, _D, _D]
            L.orc_get_padded.restype = ctypes.c_int
            L.orc_get_padded.argtypes = [ctypes.c_void_p, ctypes.c_int, _D]
            L.orc_fill_ghosts.argtypes = [ctypes.c_void_p, ctypes.c_double]
            L.orc_info.argtypes = [ctypes.c_void_p, _D, ctypes.POINTER(ctypes.c_longlong), _D, _D, _D,
                                   ctypes.POINTER(ctypes.c_longlong)]
            L.orc_rhs.argtypes = [ctypes.c_void_p, _D, _D, _D, _D, _D, _D]
            L.orc_dispersive.argtypes = [ctypes.c_void_p, _D, _D, _D, _D]
            L.orc_apply_T.argtypes = [ctypes.c_void_p, _D, _D]
            L.orc_last_weights.argtypes = [ctypes.c_void_p, _D, _D]
            L.orc_maker_state.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, _D]
            L.orc_component_k.restype = ctypes.c_double
            L.orc_component_k.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_diag_dominant.restype = ctypes.c_int
            L.orc_diag_dominant.argtypes = [ctypes.c_void_p]
            L.orc_ab3_weights.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, _D]
            L.orc_fd_weights.argtypes = [ctypes.c_double, ctypes.c_double, _D]
            L.orc_dstar_weights.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, _D]
            L.orc_thomas.argtypes = [ctypes.c_int, _D, _D, _D, _D, _D]
            L.orc_wavenumber.restype = ctypes.c_double
            L.orc_wavenumber.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]
            _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_D)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- coefficients

def ab3_weights(a: float, b: float, c: float) -> np.ndarray:
    """Eq. 42 (= Eq. 30) weights of X_t^n, X_t^{n-1}, X_t^{n-2} (dt_n/6 included)."""
    out = np.zeros(3)
    lib().orc_ab3_weights(a, b, c, _ptr(out))
    return out


def fd_weights(b: float, c: float) -> np.ndarray:
    """Eqs. 35/38/41: 3x3, row r = weights giving Y_t at level n-r."""
    out = np.zeros(9)
    lib().orc_fd_weights(b, c, _ptr(out))
    return out.reshape(3, 3)


def dstar_weights(a: float, b: float, c: float) -> np.ndarray:
    """Eq. 43 with Eqs. 44-46: weights of F*^n, F*^{n-1}, F*^{n-2}."""
    out = np.zeros(3)
    lib().orc_dstar_weights(a, b, c, _ptr(out))
    return out


def thomas(a, b, c, r) -> np.ndarray:
    a, b, c, r = (_f64(v) for v in (a, b, c, r))
    x = np.zeros_like(r)
    lib().orc_thomas(len(r), _ptr(a), _ptr(b), _ptr(c), _ptr(r), _ptr(x))
    return x


def wavenumber(omega: float, d: float, g: float = 9.81, Bd: float = 1.0 / 15.0) -> float:
    return lib().orc_wavenumber(omega, d, g, Bd)


# ---------------------------------------------------------------- domain

DEFAULTS = dict(g=9.81, Bd=1.0 / 15.0, cfl=0.2, ema_alpha=0.1, dt_init=0.0, dt_min=1e-9,
                dt_max=0.0, friction=0.0, theta=1.0, eps=0.0, w_s=0.0, ramp_time=0.0, cross_mode=1,
                bc=(WALL, WALL, WALL, WALL), sponge_width=(0.0, 0.0, 0.0, 0.0))


class OracleDomain:
    """One simulation domain in the FP64 oracle.

    ``params``: dict with nx, ny, dx, dy and optional keys of ``DEFAULTS``.
    ``bed``: (ny+1, nx+1) bed elevation at cell corners.
    ``comps``: (ncomp, 4) wave components (amplitude, frequency Hz, phase, direction).
    ``eta0``, ``P0``, ``Q0``: (ny, nx) initial state or None.
    """

    FIELDS = {"eta": 0, "P": 1, "Q": 2, "h": 3, "w": 4, "b": 5, "d": 6, "sponge": 7}

    def __init__(self, params, bed, comps=None, eta0=None, P0=None, Q0=None):
        q = dict(DEFAULTS)
        q.update(params)
        self.nx, self.ny = int(q["nx"]), int(q["ny"])
        p = _Params()
        for k, _ in _Params._fields_:
            if k in ("bc", "sponge_width"):
                continue
            setattr(p, k, q[k])
        for s in range(4):
            p.bc[s] = int(q["bc"][s])
            p.sponge_width[s] = float(q["sponge_width"][s])
        bed = _f64(bed)
        assert bed.shape == (self.ny + 1, self.nx + 1), bed.shape
        comps = _f64(comps) if comps is not None and len(comps) else None
        ncomp = 0 if comps is None else comps.shape[0]
        self._keep = [bed, comps, _f64(eta0), _f64(P0), _f64(Q0)]
        h = lib().orc_create(ctypes.byref(p), _ptr(bed), ncomp, _ptr(comps),
                             *(_ptr(a) for a in self._keep[2:]))
        if not h:
            raise ValueError("oracle: bad parameters")
        self._h = h
        self.params = q

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, dt: float = 0.0, t_end: float = float("inf")) -> int:
        """One step; dt > 0 replays that step size, else the adaptive rule."""
        return lib().orc_step(self._h, float(dt), float(t_end))

    def run(self, n_steps: int, dts=None, t_end: float = float("inf")):
        """Take n steps (or len(dts) replayed steps); returns the dt trace."""
        trace = []
        if dts is not None:
            for dt in dts:
                rc = self.step(float(dt))
                if rc:
                    raise RuntimeError("oracle step failed: %d" % rc)
                trace.append(self.info()["last_dt"])
            return np.array(trace)
        for _ in range(n_steps):
            rc = self.step(0.0, t_end)
            if rc:
                raise RuntimeError("oracle step failed: %d" % rc)
            trace.append(self.info()["last_dt"])
        return np.array(trace)

    def advance(self, t_end: float, max_steps: int = 10 ** 9):
        trace = []
        tol = 1e-12 * max(1.0, abs(t_end))
        while self.info()["t"] < t_end - tol and len(trace) < max_steps:
            rc = self.step(0.0, t_end)
            if rc:
                raise RuntimeError("oracle step failed: %d" % rc)
            trace.append(self.info()["last_dt"])
        return np.array(trace)

    def get(self, field: str) -> np.ndarray:
        out = np.zeros((self.ny, self.nx))
        rc = lib().orc_get(self._h, self.FIELDS[field], _ptr(out))
        if rc:
            raise ValueError(field)
        return out

    def fill_ghosts(self, t: float):
        """Fill the two ghost layers for time t (Sec. 3.3)."""
        lib().orc_fill_ghosts(self._h, float(t))

    def get_padded(self, field: str) -> np.ndarray:
        """w, P or Q with the ghost layers, shape (ny+4, nx+4); cell (i, j) at [j+2, i+2]."""
        out = np.zeros((self.ny + 4, self.nx + 4))
        rc = lib().orc_get_padded(self._h, {"w": 0, "P": 1, "Q": 2}[field], _ptr(out))
        if rc:
            raise ValueError(field)
        return out

    def set_state(self, eta=None, P=None, Q=None):
        a = [_f64(v) for v in (eta, P, Q)]
        self._keep.extend(a)
        lib().orc_set_state(self._h, *(_ptr(v) for v in a))

    def info(self) -> dict:
        t, dt, rate, mass = (ctypes.c_double() for _ in range(4))
        n, cl = ctypes.c_longlong(), ctypes.c_longlong()
        lib().orc_info(self._h, ctypes.byref(t), ctypes.byref(n), ctypes.byref(dt),
                       ctypes.byref(rate), ctypes.byref(mass), ctypes.byref(cl))
        return dict(t=t.value, n=n.value, last_dt=dt.value, last_rate=rate.value,
                    mass=mass.value, clamps=cl.value)

    def rhs(self) -> dict:
        outs = {k: np.zeros((self.ny, self.nx)) for k in ("E", "F", "G", "Fs", "Gs")}
        rate = ctypes.c_double()
        lib().orc_rhs(self._h, *(_ptr(outs[k]) for k in ("E", "F", "G", "Fs", "Gs")), ctypes.byref(rate))
        outs["rate"] = rate.value
        return outs

    def dispersive(self) -> dict:
        outs = {k: np.zeros((self.ny, self.nx)) for k in ("dispx", "dispy", "Fs", "Gs")}
        lib().orc_dispersive(self._h, *(_ptr(outs[k]) for k in ("dispx", "dispy", "Fs", "Gs")))
        return outs

    def apply_T(self):
        U, V = np.zeros((self.ny, self.nx)), np.zeros((self.ny, self.nx))
        lib().orc_apply_T(self._h, _ptr(U), _ptr(V))
        return U, V

    def last_weights(self):
        b, g = np.zeros(3), np.zeros(3)
        lib().orc_last_weights(self._h, _ptr(b), _ptr(g))
        return b, g

    def maker_state(self, x, y, t):
        out = np.zeros(3)
        lib().orc_maker_state(self._h, x, y, t, _ptr(out))
        return out

    def component_k(self, k: int) -> float:
        return lib().orc_component_k(self._h, k)

    def diag_dominant(self) -> bool:
        return bool(lib().orc_diag_dominant(self._h))
