"""Plain FP64 CPU oracle of the vielbein lattice Boltzmann method on the sphere.

TEST INFRASTRUCTURE ONLY: the CUDA library is checked against this code.  Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference leg may import it; the product path never does.

The numerics live in ``vlbm_oracle.c`` (plain C, FP64, no FMA contraction);
this module compiles it with gcc and wraps it with ctypes.  Every routine
follows arXiv 2504.15574 Sec. 3 (see the header of ``vlbm_oracle.c`` for the
equation each step follows and the readings taken where the paper is silent).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vlbm_oracle.c")
_LIB = os.path.join(_HERE, "libvlbm_oracle.so")
_lock = threading.Lock()
_lib = None

NK = 16


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libvlbm_oracle.so`` with gcc."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC",
           "-std=c11", "-D_GNU_SOURCE", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        D = ctypes.c_double
        P = ctypes.POINTER(ctypes.c_double)
        lib.vo_create.restype = ctypes.c_void_p
        lib.vo_create.argtypes = [ctypes.c_int, ctypes.c_int, D, D, D, D, ctypes.c_int]
        lib.vo_create_q.restype = ctypes.c_void_p
        lib.vo_create_q.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, D, D, D, D, ctypes.c_int]
        lib.vo_quadrature_q.argtypes = [ctypes.c_int, P, P]
        lib.vo_kernels_q.argtypes = [ctypes.c_int, P, P]
        lib.vo_equilibrium_q.argtypes = [ctypes.c_int, D, D, D, D, P]
        lib.vo_destroy.argtypes = [ctypes.c_void_p]
        lib.vo_set_scheme.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
        lib.vo_quadrature.argtypes = [P, P]
        lib.vo_kernels.argtypes = [P, P]
        lib.vo_weno5.restype = D
        lib.vo_weno5.argtypes = [D, D, D, D, D, D]
        lib.vo_equilibrium.argtypes = [D, D, D, D, P]
        lib.vo_init_moments.argtypes = [ctypes.c_void_p, P, P, P, P]
        lib.vo_set_populations.argtypes = [ctypes.c_void_p, P]
        lib.vo_get_populations.argtypes = [ctypes.c_void_p, P]
        lib.vo_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.vo_moments.argtypes = [ctypes.c_void_p, P, P, P, P]
        lib.vo_operator.restype = D
        lib.vo_operator.argtypes = [ctypes.c_void_p, P, P, P, P]
        lib.vo_diagnostics.argtypes = [ctypes.c_void_p, P]
        lib.vo_geometry.argtypes = [ctypes.c_void_p, P, P, ctypes.POINTER(ctypes.c_int)]
        _lib = lib
        return lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = np.ascontiguousarray(np.broadcast_to(a, shape), dtype=np.float64)
    return a


def quadrature(q=4):
    """Velocities (ascending roots of H_Q) and 1-D weights, Eq. (GH_weights); Q = 4 or 3."""
    lib = _load()
    v = np.zeros(q)
    w = np.zeros(q)
    lib.vo_quadrature_q(int(q), _ptr(v), _ptr(w))
    return v, w


def kernels(q=4):
    """K^H and Ktilde^H of Eqs. (KH), (KtildeH) as Q x Q arrays."""
    lib = _load()
    K = np.zeros(q * q)
    Kt = np.zeros(q * q)
    lib.vo_kernels_q(int(q), _ptr(K), _ptr(Kt))
    return K.reshape(q, q), Kt.reshape(q, q)


def weno5(a, b, c, d, e, eps=1e-6):
    """WENO-5 reconstruction at c+1/2 from upwind-ordered values."""
    return _load().vo_weno5(float(a), float(b), float(c), float(d), float(e), float(eps))


def equilibrium(n, ut, up, T=1.0, q=4):
    """Populations of the Hermite equilibrium of order Q (T = 1: Eq. feq_Q=4, or Eq. feq_Q=3)."""
    out = np.zeros(q * q)
    _load().vo_equilibrium_q(int(q), float(n), float(ut), float(up), float(T), _ptr(out))
    return out


class Oracle:
    """FP64 CPU vLBM on an n_theta x n_phi grid (mirror of the C ABI)."""

    SCHEMES = {"weno5": 0, "u1": 1, "u2": 2, "u3": 3}

    def __init__(self, n_theta, n_phi, tau, dt, eps=1e-6, R=1.0, polar_filter=False, scheme="weno5",
                 komissarov=False, q=4):
        lib = _load()
        self._lib = lib
        self.q, self.nk = int(q), int(q) * int(q)
        self.n_theta, self.n_phi = int(n_theta), int(n_phi)
        self.tau, self.dt, self.eps, self.R = float(tau), float(dt), float(eps), float(R)
        h = lib.vo_create_q(self.q, self.n_theta, self.n_phi, self.tau, self.dt, self.eps, self.R,
                            1 if polar_filter else 0)
        if not h:
            raise ValueError("oracle: invalid arguments")
        self._h = ctypes.c_void_p(h)
        if lib.vo_set_scheme(self._h, self.SCHEMES[scheme], 1 if komissarov else 0) != 0:
            raise ValueError("oracle: unknown scheme")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.vo_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (self.n_theta, self.n_phi)

    def init_moments(self, rho, u_theta, u_phi, T=None):
        s = self.shape
        rho, ut, up = _f64(rho, s), _f64(u_theta, s), _f64(u_phi, s)
        T = _f64(T, s)
        rc = self._lib.vo_init_moments(self._h, _ptr(rho), _ptr(ut), _ptr(up), _ptr(T))
        if rc:
            raise RuntimeError("oracle init_moments failed")

    def set_populations(self, f):
        f = _f64(f, (self.nk,) + self.shape)
        if self._lib.vo_set_populations(self._h, _ptr(f)):
            raise RuntimeError("oracle set_populations failed")

    def get_populations(self):
        f = np.zeros((self.nk,) + self.shape)
        self._lib.vo_get_populations(self._h, _ptr(f))
        return f

    def step(self, n=1):
        if self._lib.vo_step(self._h, int(n)):
            raise RuntimeError("oracle step failed")

    def moments(self, with_T=False):
        s = self.shape
        rho, ut, up = np.zeros(s), np.zeros(s), np.zeros(s)
        T = np.zeros(s) if with_T else None
        self._lib.vo_moments(self._h, _ptr(rho), _ptr(ut), _ptr(up), _ptr(T))
        return (rho, ut, up, T) if with_T else (rho, ut, up)

    def operator(self, g):
        """L[g] plus interface fluxes (Ft: [Q^2, nt+1, np], Fp: [Q^2, nt, np+1]) and
        the pole mass-flux rate."""
        g = _f64(g, (self.nk,) + self.shape)
        nt, np_ = self.shape
        L = np.zeros((self.nk, nt, np_))
        Ft = np.zeros((self.nk, nt + 1, np_))
        Fp = np.zeros((self.nk, nt, np_ + 1))
        m = self._lib.vo_operator(self._h, _ptr(g), _ptr(L), _ptr(Ft), _ptr(Fp))
        return L, Ft, Fp, m

    def diagnostics(self):
        out = np.zeros(10)
        self._lib.vo_diagnostics(self._h, _ptr(out))
        keys = ["mass", "px", "py", "pz", "energy", "pole_budget", "mass0", "t", "steps", "nonfinite"]
        return dict(zip(keys, out.tolist()))

    def geometry(self):
        nt = self.n_theta
        s, c = np.zeros(nt), np.zeros(nt)
        b = np.zeros(nt, dtype=np.int32)
        self._lib.vo_geometry(self._h, _ptr(s), _ptr(c), b.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return s, c, b
