"""ctypes binding of libvlbm.so (the C ABI declared in include/vlbm.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  The functions keep the C names (``vlbm_create``,
``vlbm_init_moments``, ``vlbm_step``, ``vlbm_moments``, ``vlbm_destroy``, ...);
``Solver`` is a small object wrapper over them.  There is no fallback: if the
library is missing this module raises, and without a GPU the calls that need
one raise ``VlbmError`` with code VLBM_ERR_CUDA.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvlbm.so")

VLBM_OK, VLBM_ERR_ARG, VLBM_ERR_UNSUPPORTED, VLBM_ERR_CUDA, VLBM_ERR_NONFINITE, VLBM_ERR_TIMEOUT = 0, -1, -2, -3, -4, -5
VLBM_D2Q9, VLBM_D2Q16 = 3, 4
VLBM_FP64, VLBM_FP32 = 0, 1
NK = 16

_lock = threading.Lock()
_lib = None


class VlbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"vlbm error {code}: {msg}")
        self.code = code


class vlbm_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("weno_eps", ctypes.c_double), ("radius", ctypes.c_double),
                ("polar_filter", ctypes.c_int), ("guard", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("rho_ref", ctypes.c_double), ("tile_rows", ctypes.c_int), ("scheme", ctypes.c_int),
                ("komissarov", ctypes.c_int), ("velocity_set", ctypes.c_int)]


SCHEMES = {"weno5": 0, "u1": 1, "u2": 2, "u3": 3}


class vlbm_diag(ctypes.Structure):
    _fields_ = [("time", ctypes.c_double), ("steps", ctypes.c_longlong), ("mass", ctypes.c_double),
                ("momentum", ctypes.c_double * 3), ("energy", ctypes.c_double), ("pole_flux", ctypes.c_double),
                ("mass0", ctypes.c_double), ("nonfinite", ctypes.c_int)]


_PD = ctypes.POINTER(ctypes.c_double)
_H = ctypes.c_void_p

# name -> (restype, argtypes); mirrors include/vlbm.h
SIGNATURES = {
    "vlbm_default_options": (None, [ctypes.POINTER(vlbm_options)]),
    "vlbm_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   ctypes.POINTER(vlbm_options), ctypes.POINTER(_H)]),
    "vlbm_init_moments": (ctypes.c_int, [_H, _PD, _PD, _PD, _PD]),
    "vlbm_step": (ctypes.c_int, [_H, ctypes.c_int]),
    "vlbm_step_async": (ctypes.c_int, [_H, ctypes.c_int]),
    "vlbm_sync": (ctypes.c_int, [_H]),
    "vlbm_moments": (ctypes.c_int, [_H, _PD, _PD, _PD, _PD]),
    "vlbm_get_populations": (ctypes.c_int, [_H, _PD]),
    "vlbm_set_populations": (ctypes.c_int, [_H, _PD]),
    "vlbm_diagnostics": (ctypes.c_int, [_H, ctypes.POINTER(vlbm_diag)]),
    "vlbm_max_stable_dt": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                          _PD]),
    "vlbm_profile_step": (ctypes.c_int, [_H, ctypes.c_int, _PD, ctypes.POINTER(ctypes.c_int)]),
    "vlbm_set_wait_limit": (ctypes.c_int, [_H, ctypes.c_double]),
    "vlbm_device_bytes": (ctypes.c_size_t, [_H]),
    "vlbm_last_error": (ctypes.c_char_p, [_H]),
    "vlbm_destroy": (None, [_H]),
    "vlbm_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                         _PD, _PD, ctypes.POINTER(vlbm_options), ctypes.POINTER(_H)]),
    "vlbm_batch_init_moments": (ctypes.c_int, [_H, ctypes.c_int, _PD, _PD, _PD, _PD]),
    "vlbm_batch_step": (ctypes.c_int, [_H, ctypes.c_int]),
    "vlbm_batch_step_async": (ctypes.c_int, [_H, ctypes.c_int]),
    "vlbm_batch_sync": (ctypes.c_int, [_H]),
    "vlbm_batch_moments": (ctypes.c_int, [_H, ctypes.c_int, _PD, _PD, _PD, _PD]),
    "vlbm_batch_set_schedule": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int]),
    "vlbm_batch_get_populations": (ctypes.c_int, [_H, ctypes.c_int, _PD]),
    "vlbm_batch_tune": (ctypes.c_int, [_H, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       _PD]),
    "vlbm_batch_profile": (ctypes.c_int, [_H, ctypes.c_int, _PD, ctypes.POINTER(ctypes.c_int)]),
    "vlbm_batch_cells": (ctypes.c_size_t, [_H]),
    "vlbm_batch_last_error": (ctypes.c_char_p, [_H]),
    "vlbm_batch_destroy": (None, [_H]),
    "vlbm_lc_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong, ctypes.POINTER(_H)]),
    "vlbm_lc_num_params": (ctypes.c_int, [_H]),
    "vlbm_lc_get_weights": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_float)]),
    "vlbm_lc_set_weights": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_float)]),
    "vlbm_lc_set_scales": (ctypes.c_int, [_H, _PD, _PD]),
    "vlbm_lc_set_output_form": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_double]),
    "vlbm_lc_predict": (ctypes.c_int, [_H, _PD, _PD]),
    "vlbm_lc_gradients": (ctypes.c_int, [_H, _PD, _PD, _PD, ctypes.POINTER(ctypes.c_float)]),
    "vlbm_lc_train_step": (ctypes.c_int, [_H, _PD, _PD, ctypes.c_float, _PD]),
    "vlbm_lc_apply": (ctypes.c_int, [_H, _H]),
    "vlbm_lc_rollout": (ctypes.c_int, [_H, _H, ctypes.c_int]),
    "vlbm_lc_last_error": (ctypes.c_char_p, [_H]),
    "vlbm_lc_destroy": (None, [_H]),
    "vlbm_diagnostics_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                ctypes.c_void_p, ctypes.c_void_p]),
    "vlbm_noalloc_last_error": (ctypes.c_char_p, []),
}


def load(path: str | None = None):
    """Loads libvlbm.so (built by paper_2504_15574_gb300.build); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} not found: build it with paper_2504_15574_gb300.build.build()")
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(rc, h=None):
    if rc != VLBM_OK:
        msg = load().vlbm_last_error(h)
        raise VlbmError(rc, msg.decode() if msg else "")


def _p(a):
    return None if a is None else a.ctypes.data_as(_PD)


def _host(a, shape):
    if a is None:
        return None
    return np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), shape))


# ---- the C names -----------------------------------------------------------------

def vlbm_default_options() -> vlbm_options:
    o = vlbm_options()
    load().vlbm_default_options(ctypes.byref(o))
    return o


def vlbm_create(n_theta, n_phi, velocity_set, tau, dt, opt: vlbm_options | None = None):
    h = _H()
    rc = load().vlbm_create(int(n_theta), int(n_phi), int(velocity_set), float(tau), float(dt),
                            ctypes.byref(opt) if opt is not None else None, ctypes.byref(h))
    _check(rc, None)
    return h


def vlbm_init_moments(h, rho, u_theta, u_phi, T=None, shape=None):
    _check(load().vlbm_init_moments(h, _p(rho), _p(u_theta), _p(u_phi), _p(T)), h)


def vlbm_step(h, n):
    _check(load().vlbm_step(h, int(n)), h)


def vlbm_step_async(h, n):
    _check(load().vlbm_step_async(h, int(n)), h)


def vlbm_sync(h):
    _check(load().vlbm_sync(h), h)


def vlbm_moments(h, rho, u_theta, u_phi, T=None):
    _check(load().vlbm_moments(h, _p(rho), _p(u_theta), _p(u_phi), _p(T)), h)


def vlbm_get_populations(h, f):
    _check(load().vlbm_get_populations(h, _p(f)), h)


def vlbm_set_populations(h, f):
    _check(load().vlbm_set_populations(h, _p(f)), h)


def vlbm_diagnostics(h) -> dict:
    d = vlbm_diag()
    _check(load().vlbm_diagnostics(h, ctypes.byref(d)), h)
    return {"time": d.time, "steps": d.steps, "mass": d.mass, "px": d.momentum[0], "py": d.momentum[1],
            "pz": d.momentum[2], "energy": d.energy, "pole_flux": d.pole_flux, "mass0": d.mass0,
            "nonfinite": d.nonfinite}


def vlbm_set_wait_limit(h, seconds):
    _check(load().vlbm_set_wait_limit(h, float(seconds)), h)


def vlbm_max_stable_dt(n_theta, n_phi, tau, polar_filter=False, velocity_set=VLBM_D2Q16) -> float:
    out = ctypes.c_double()
    rc = load().vlbm_max_stable_dt(int(n_theta), int(n_phi), int(velocity_set), float(tau), int(bool(polar_filter)),
                                   ctypes.byref(out))
    _check(rc, None)
    return out.value


def vlbm_profile_step(h, n):
    """(stage kernel ms [3], polar filter ms [3], kernels per step)"""
    ms = (ctypes.c_double * 6)()
    launches = ctypes.c_int()
    _check(load().vlbm_profile_step(h, int(n), ms, ctypes.byref(launches)), h)
    return list(ms[:3]), list(ms[3:]), launches.value


def vlbm_device_bytes(h) -> int:
    return int(load().vlbm_device_bytes(h))


def vlbm_last_error(h=None) -> str:
    m = load().vlbm_last_error(h)
    return m.decode() if m else ""


def vlbm_destroy(h):
    load().vlbm_destroy(h)


# ---- object wrapper --------------------------------------------------------------

class Solver:
    """One vLBM solver on the GPU: ``Solver(n_theta, n_phi, tau, dt, precision="fp64"|"fp32")``."""

    def __init__(self, n_theta, n_phi, tau, dt, precision="fp64", eps=1e-6, R=1.0, polar_filter=False,
                 guard=True, stream=None, rho_ref=0.0, tile_rows=0, scheme="weno5", komissarov=False,
                 velocity_set="d2q16"):
        o = vlbm_default_options()
        o.scheme = SCHEMES[scheme]
        o.komissarov = int(bool(komissarov))
        o.precision = VLBM_FP32 if precision in ("fp32", VLBM_FP32) else VLBM_FP64
        o.weno_eps = float(eps)
        o.radius = float(R)
        o.polar_filter = int(bool(polar_filter))
        o.guard = int(bool(guard))
        o.stream = stream
        o.rho_ref = float(rho_ref)
        o.tile_rows = int(tile_rows)
        self.n_theta, self.n_phi = int(n_theta), int(n_phi)
        self.tau, self.dt = float(tau), float(dt)
        self.precision = "fp32" if o.precision == VLBM_FP32 else "fp64"
        vs = {"d2q16": VLBM_D2Q16, "d2q9": VLBM_D2Q9}[velocity_set]
        self.nk = vs * vs
        self.h = vlbm_create(n_theta, n_phi, vs, tau, dt, o)

    @property
    def shape(self):
        return (self.n_theta, self.n_phi)

    def init_moments(self, rho, u_theta, u_phi, T=None):
        s = self.shape
        rho, ut, up, T = _host(rho, s), _host(u_theta, s), _host(u_phi, s), _host(T, s)
        vlbm_init_moments(self.h, rho, ut, up, T)

    def step(self, n=1):
        vlbm_step(self.h, n)

    def step_async(self, n=1):
        vlbm_step_async(self.h, n)

    def sync(self):
        vlbm_sync(self.h)

    def moments(self, with_T=False):
        s = self.shape
        rho, ut, up = np.empty(s), np.empty(s), np.empty(s)
        T = np.empty(s) if with_T else None
        vlbm_moments(self.h, rho, ut, up, T)
        return (rho, ut, up, T) if with_T else (rho, ut, up)

    def get_populations(self):
        f = np.empty((self.nk,) + self.shape)
        vlbm_get_populations(self.h, f)
        return f

    def set_populations(self, f):
        vlbm_set_populations(self.h, _host(f, (self.nk,) + self.shape))

    def diagnostics(self):
        return vlbm_diagnostics(self.h)

    def profile_step(self, n=1):
        return vlbm_profile_step(self.h, n)

    def device_bytes(self):
        return vlbm_device_bytes(self.h)

    def close(self):
        if getattr(self, "h", None):
            vlbm_destroy(self.h)
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


# ---- batched ensembles -----------------------------------------------------------

def _bcheck(rc, b=None):
    if rc != VLBM_OK:
        msg = load().vlbm_batch_last_error(b)
        raise VlbmError(rc, msg.decode() if msg else "")


class Batch:
    """Many FP32 runs of uneven grids advanced together (vlbm_batch_*).

    grids: list of (n_theta, n_phi); tau, dt: scalars or per-run sequences."""

    def __init__(self, grids, tau, dt, eps=1e-6, R=1.0, polar_filter=False, guard=True, stream=None,
                 scheme="weno5", komissarov=False, velocity_set="d2q16"):
        lib = load()
        n = len(grids)
        self.grids = [(int(a), int(b)) for a, b in grids]
        nt = (ctypes.c_int * n)(*[g[0] for g in self.grids])
        np_ = (ctypes.c_int * n)(*[g[1] for g in self.grids])
        taus = np.ascontiguousarray(np.broadcast_to(np.asarray(tau, dtype=np.float64), (n,)))
        dts = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (n,)))
        o = vlbm_default_options()
        o.precision = VLBM_FP32
        o.weno_eps = float(eps)
        o.radius = float(R)
        o.polar_filter = int(bool(polar_filter))
        o.guard = int(bool(guard))
        o.stream = stream
        o.scheme = SCHEMES[scheme]
        o.komissarov = int(bool(komissarov))
        o.velocity_set = VLBM_D2Q9 if velocity_set == "d2q9" else VLBM_D2Q16
        self.q = 3 if velocity_set == "d2q9" else 4
        self.b = _H()
        _bcheck(lib.vlbm_batch_create(n, nt, np_, _p(taus), _p(dts), ctypes.byref(o), ctypes.byref(self.b)))

    def __len__(self):
        return len(self.grids)

    def init_moments(self, run, rho, u_theta, u_phi, T=None):
        s = self.grids[run]
        _bcheck(load().vlbm_batch_init_moments(self.b, int(run), _p(_host(rho, s)), _p(_host(u_theta, s)),
                                               _p(_host(u_phi, s)), _p(_host(T, s))), self.b)

    def step(self, n=1):
        _bcheck(load().vlbm_batch_step(self.b, int(n)), self.b)

    def step_async(self, n=1):
        _bcheck(load().vlbm_batch_step_async(self.b, int(n)), self.b)

    def sync(self):
        _bcheck(load().vlbm_batch_sync(self.b), self.b)

    def moments(self, run, with_T=False):
        s = self.grids[run]
        rho, ut, up = np.empty(s), np.empty(s), np.empty(s)
        T = np.empty(s) if with_T else None
        _bcheck(load().vlbm_batch_moments(self.b, int(run), _p(rho), _p(ut), _p(up), _p(T)), self.b)
        return (rho, ut, up, T) if with_T else (rho, ut, up)

    def get_populations(self, run):
        f = np.empty((self.q * self.q,) + self.grids[run])
        _bcheck(load().vlbm_batch_get_populations(self.b, int(run), _p(f)), self.b)
        return f

    def set_schedule(self, tile_rows, ctas_per_sm=0):
        _bcheck(load().vlbm_batch_set_schedule(self.b, int(tile_rows), int(ctas_per_sm)), self.b)

    def tune(self, cache_path=None):
        ty, c, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        path = cache_path.encode() if cache_path else None
        _bcheck(load().vlbm_batch_tune(self.b, path, ctypes.byref(ty), ctypes.byref(c), ctypes.byref(ms)), self.b)
        return {"tile_rows": ty.value, "ctas_per_sm": c.value, "ms_per_step": ms.value}

    def profile(self, n=1):
        ms, l = ctypes.c_double(), ctypes.c_int()
        _bcheck(load().vlbm_batch_profile(self.b, int(n), ctypes.byref(ms), ctypes.byref(l)), self.b)
        return ms.value, l.value

    def cells(self):
        return int(load().vlbm_batch_cells(self.b))

    def close(self):
        if getattr(self, "b", None):
            load().vlbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- learned correction ----------------------------------------------------------

class LearnedCorrection:
    """The coarse-grid correction network (vlbm_lc_*)."""

    # scales of the 14 data channels: rho-1, u^theta, u^phi, T-1, then the ten differences
    DEFAULT_IN_SCALE = (1e-3, 1e-2, 1e-2, 1e-3) + (1e-6,) * 2 + (1e-5,) * 8

    FORMS = {"direct": 0, "stream": 1, "vorticity": 2}

    def __init__(self, n_theta, n_phi, seed=1, in_scale=DEFAULT_IN_SCALE, out_scale=(1e-5, 1e-4, 1e-4),
                 form="direct", R=1.0):
        self.shape = (int(n_theta), int(n_phi))
        self.h = _H()
        rc = load().vlbm_lc_create(self.shape[0], self.shape[1], int(seed), ctypes.byref(self.h))
        if rc:
            raise VlbmError(rc, "vlbm_lc_create failed")
        self.set_scales(in_scale, out_scale)
        self.set_output_form(form, R)

    def set_output_form(self, form, R=1.0):
        """"direct": outputs (drho, du^theta, du^phi); "stream": output 0 is a stream function
        whose centred curl on a sphere of radius R is the velocity correction (drho = 0);
        "vorticity": output 0 is a vorticity correction, the stream function the solution of the
        finite-volume Poisson equation for it."""
        self._chk(load().vlbm_lc_set_output_form(self.h, self.FORMS[form], float(R)))
        self.form, self.R = form, float(R)

    def _chk(self, rc):
        if rc != VLBM_OK:
            m = load().vlbm_lc_last_error(self.h)
            raise VlbmError(rc, m.decode() if m else "")

    def set_scales(self, in_scale, out_scale):
        self.in_scale = np.asarray(in_scale, dtype=np.float64)
        self.out_scale = np.asarray(out_scale, dtype=np.float64)
        if self.in_scale.shape != (14,) or self.out_scale.shape != (3,):
            raise ValueError("in_scale takes 14 values, out_scale 3")
        self._chk(load().vlbm_lc_set_scales(self.h, _p(self.in_scale), _p(self.out_scale)))

    def num_params(self):
        return int(load().vlbm_lc_num_params(self.h))

    def get_weights(self):
        w = np.empty(self.num_params(), dtype=np.float32)
        self._chk(load().vlbm_lc_get_weights(self.h, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return w

    def set_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        self._chk(load().vlbm_lc_set_weights(self.h, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def predict(self, x):
        x = _host(x, (4,) + self.shape)
        out = np.empty((3,) + self.shape)
        self._chk(load().vlbm_lc_predict(self.h, _p(x), _p(out)))
        return out

    def gradients(self, x, t):
        x, t = _host(x, (4,) + self.shape), _host(t, (3,) + self.shape)
        loss = ctypes.c_double()
        g = np.empty(self.num_params(), dtype=np.float32)
        self._chk(load().vlbm_lc_gradients(self.h, _p(x), _p(t), ctypes.byref(loss),
                                           g.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return loss.value, g

    def train_step(self, x, t, lr):
        x, t = _host(x, (4,) + self.shape), _host(t, (3,) + self.shape)
        loss = ctypes.c_double()
        self._chk(load().vlbm_lc_train_step(self.h, _p(x), _p(t), float(lr), ctypes.byref(loss)))
        return loss.value

    def apply(self, solver):
        self._chk(load().vlbm_lc_apply(self.h, solver.h))

    def rollout(self, solver, steps):
        """`steps` corrected coarse steps (step, then correction) as device graph launches."""
        self._chk(load().vlbm_lc_rollout(self.h, solver.h, int(steps)))

    def close(self):
        if getattr(self, "h", None):
            load().vlbm_lc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def vlbm_diagnostics_noalloc(f_dev_ptr, n_theta, n_phi, radius, out_dev_ptr, stream=None):
    """Diagnostics of a caller-owned D2Q16 device array with no allocation in the library
    (for callers that cannot call cudaMalloc where they need the numbers: their own memory
    pool or budget, latency-bound loops).  Takes raw device addresses; enqueues on `stream`
    and returns without waiting.  out[5] counts the cells holding a NaN or Inf population."""
    rc = load().vlbm_diagnostics_noalloc(ctypes.c_void_p(f_dev_ptr), int(n_theta), int(n_phi), float(radius),
                                         ctypes.c_void_p(out_dev_ptr), stream)
    if rc != VLBM_OK:
        m = load().vlbm_noalloc_last_error()
        raise VlbmError(rc, m.decode() if m else "")
