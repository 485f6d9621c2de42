"""Seeded synthetic initial conditions for the vLBM workloads.

This module only produces moment fields (rho, u^theta-hat, u^phi-hat, T) on the
cell-centred grid of arXiv 2504.15574 Sec. 3.4, Eq. (discrete_coord_sphere).  It
holds none of the method's arithmetic (no equilibrium, no fluxes), so both the
CUDA library's tests and the CPU oracle's tests may draw their inputs from it.

Random numbers come from splitmix64 (Steele, Lea & Flood 2014), implemented here
from its published definition so that every field is reproducible from a seed.
"""
from __future__ import annotations

import math

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """splitmix64: state += 0x9E3779B97F4A7C15, then the two xor-shift-multiply rounds."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def integer(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi]."""
        return lo + int(self.uniform() * (hi - lo + 1)) if hi > lo else lo

    def normal_array(self, shape) -> np.ndarray:
        """Standard normals by Box-Muller (for noise fixtures)."""
        n = int(np.prod(shape))
        out = np.empty(n)
        for i in range(0, n, 2):
            u1 = max(self.uniform(), 1e-300)
            u2 = self.uniform()
            r = math.sqrt(-2.0 * math.log(u1))
            out[i] = r * math.cos(2 * math.pi * u2)
            if i + 1 < n:
                out[i + 1] = r * math.sin(2 * math.pi * u2)
        return out.reshape(shape)


def cell_centres(n_theta: int, n_phi: int):
    """theta_s = pi (s - 1/2) / N_theta, phi_q = 2 pi (q - 1/2) / N_phi (s, q 1-based)."""
    th = (np.arange(n_theta) + 0.5) * (math.pi / n_theta)
    ph = (np.arange(n_phi) + 0.5) * (2.0 * math.pi / n_phi)
    return th, ph


def _grid(n_theta, n_phi):
    th, ph = cell_centres(n_theta, n_phi)
    return np.meshgrid(th, ph, indexing="ij")


def shear_p21(n_theta: int, n_phi: int, amplitude: float = 1e-3):
    """rho = 1, u^theta = 0, u^phi = A P_2^1(cos theta) = -3 A sin cos (Condon-Shortley phase)."""
    TH, _ = _grid(n_theta, n_phi)
    rho = np.ones_like(TH)
    return rho, np.zeros_like(TH), amplitude * (-3.0 * np.sin(TH) * np.cos(TH)), None


def sound_parabola(n_theta: int, n_phi: int = 1, U0: float = 1e-5):
    """Axisymmetric sound-wave start: u^theta = U0 (pi - theta) theta, rho = 1."""
    TH, _ = _grid(n_theta, n_phi)
    return np.ones_like(TH), U0 * (math.pi - TH) * TH, np.zeros_like(TH), None


def rotated_frame(n_theta: int, n_phi: int, alpha: float):
    """Geometry of a grid rotated by alpha about the y axis (App. C, Eqs. transf, transf_inv).

    For every cell (theta', phi') of the n_theta x n_phi grid, the coordinates (theta, phi)
    of the same point in the original frame, and the 2 x 2 matrix M (shape [2, 2, nt, np])
    that maps original-frame vielbein components (u^theta, u^phi) at that point to the
    grid's components (u^theta', u^phi'): the Cartesian rotation x' = R_2(alpha) x applied
    to u^theta e_theta + u^phi e_phi, projected on e_theta', e_phi'."""
    TH, PH = _grid(n_theta, n_phi)
    ca, sa = math.cos(alpha), math.sin(alpha)
    # the cell's position in the grid's (primed) Cartesian frame, then x = R_2(alpha)^T x'
    xp, yp, zp = np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)
    x = ca * xp - sa * zp
    y = yp
    z = sa * xp + ca * zp
    th = np.arccos(np.clip(z, -1.0, 1.0))
    ph = np.mod(np.arctan2(y, x), 2 * math.pi)

    def rot(v):   # x' = R_2(alpha) x
        return np.stack([ca * v[0] + sa * v[2], v[1], -sa * v[0] + ca * v[2]])

    e_th = rot(np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)]))
    e_ph = rot(np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)]))
    ep_th = np.stack([np.cos(TH) * np.cos(PH), np.cos(TH) * np.sin(PH), -np.sin(TH)])
    ep_ph = np.stack([-np.sin(PH), np.cos(PH), np.zeros_like(PH)])
    M = np.array([[(ep_th * e_th).sum(0), (ep_th * e_ph).sum(0)],
                  [(ep_ph * e_th).sum(0), (ep_ph * e_ph).sum(0)]])
    return th, ph, M


def sound_parabola_rotated(n_theta: int, n_phi: int, U0: float = 1e-5, alpha: float = -math.pi / 2):
    """The axisymmetric sound-wave start of sound_parabola about an axis tilted by alpha:
    on the grid rotated by alpha (App. C), u = U0 (pi - theta) theta e_theta of the
    original frame, rho = 1."""
    th, _, M = rotated_frame(n_theta, n_phi, alpha)
    ut0 = U0 * (math.pi - th) * th
    return np.ones_like(th), M[0, 0] * ut0, M[1, 0] * ut0, None


def shear_uniform(n_theta: int, n_phi: int = 1, V0: float = 1e-5):
    """Axisymmetric shear-wave start: u^phi = V0, rho = 1."""
    TH, _ = _grid(n_theta, n_phi)
    return np.ones_like(TH), np.zeros_like(TH), V0 * np.ones_like(TH), None


def schmidt_legendre(ell: int, m: int, x):
    """Schmidt semi-normalised associated Legendre function (no Condon-Shortley phase)."""
    x = np.asarray(x, dtype=np.float64)
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    pmm = np.ones_like(x)
    for i in range(1, m + 1):
        pmm = pmm * (2 * i - 1) * s
    if ell == m:
        p = pmm
    else:
        pm1 = x * (2 * m + 1) * pmm
        if ell == m + 1:
            p = pm1
        else:
            a, b = pmm, pm1
            for l in range(m + 2, ell + 1):
                a, b = b, ((2 * l - 1) * x * b - (l + m - 1) * a) / (l - m)
            p = b
    norm = math.sqrt((2.0 if m > 0 else 1.0) * math.factorial(ell - m) / math.factorial(ell + m))
    return norm * p


def _legendre_phases(ell: int):
    rng = SplitMix64(0x2504155740 + ell)
    return [rng.uniform(0.0, 2.0 * math.pi) for _ in range(ell + 1)]


def legendre_field(n_theta: int, n_phi: int, ell: int):
    """sum_{m=0}^{ell} Pbar_ell^m(cos theta) cos(m phi + alpha_m) / (ell + 1), alpha seeded."""
    TH, PH = _grid(n_theta, n_phi)
    al = _legendre_phases(ell)
    out = np.zeros_like(TH)
    for m in range(ell + 1):
        out += schmidt_legendre(ell, m, np.cos(TH)) * np.cos(m * PH + al[m])
    return out / (ell + 1)


def sound_legendre(n_theta: int, n_phi: int, ell: int, amplitude: float = 1e-3):
    """rho = 1 + A * legendre_field, u = 0 (sound set of degree ell)."""
    d = legendre_field(n_theta, n_phi, ell)
    return 1.0 + amplitude * d, np.zeros_like(d), np.zeros_like(d), None


def shear_legendre(n_theta: int, n_phi: int, ell: int, amplitude: float = 1e-3):
    """Stream function psi = A * legendre_field; u^theta = -(1/sin) d_phi psi, u^phi = d_theta psi."""
    TH, PH = _grid(n_theta, n_phi)
    al = _legendre_phases(ell)
    ut = np.zeros_like(TH)
    up = np.zeros_like(TH)
    x = np.cos(TH)
    h = 1e-6
    for m in range(ell + 1):
        P = schmidt_legendre(ell, m, x)
        # d/dtheta by a centred difference of the (smooth, closed-form) Legendre function
        dP = (schmidt_legendre(ell, m, np.cos(TH + h)) - schmidt_legendre(ell, m, np.cos(TH - h))) / (2 * h)
        ut += -(1.0 / np.sin(TH)) * P * (-m * np.sin(m * PH + al[m]))
        up += dP * np.cos(m * PH + al[m])
    ut *= amplitude / (ell + 1)
    up *= amplitude / (ell + 1)
    return np.ones_like(TH), ut, up, None


def shock_cap(n_theta: int, n_phi: int, cap: float = 0.2, rho_in: float = 4.0, T_in: float = 1.5):
    """Polar cap theta < cap at (rho_in, T_in), rho = 1, T = 1 elsewhere, u = 0."""
    TH, _ = _grid(n_theta, n_phi)
    inside = TH < cap
    rho = np.where(inside, rho_in, 1.0)
    T = np.where(inside, T_in, 1.0)
    z = np.zeros_like(TH)
    return rho, z, z.copy(), T


def riemann_cap(n_theta: int, n_phi: int = 1, rho1: float = 1.0, rho2: float = 0.125,
                theta_disc: float = math.pi / 10):
    """Sod-like start: rho1 for theta < theta_disc, rho2 beyond, fluid at rest."""
    TH, _ = _grid(n_theta, n_phi)
    rho = np.where(TH < theta_disc, rho1, rho2)
    z = np.zeros_like(TH)
    return rho, z, z.copy(), None


def riemann_cap_rotated(n_theta: int, n_phi: int, alpha: float = -math.pi / 2, rho1: float = 1.0,
                        rho2: float = 0.125, theta_disc: float = math.pi / 10):
    """The riemann_cap start about an axis tilted by alpha (App. C, Fig. riemann_2D): on the
    grid rotated by alpha, rho1 where the original-frame polar angle is below theta_disc,
    rho2 beyond, fluid at rest."""
    th, _, _ = rotated_frame(n_theta, n_phi, alpha)
    rho = np.where(th < theta_disc, rho1, rho2)
    z = np.zeros_like(th)
    return rho, z, z.copy(), None


def gaussian_vortices(n_theta: int, n_phi: int, run: int, umax: float = 0.05):
    """2-8 Gaussian vortices psi_i = A_i exp(-d_i^2 / (2 r_i^2)) at random centres.

    d_i is the great-circle angle to centre i, r_i ~ U[0.1, 0.3], peak speed
    U_i ~ U[0.02, 0.05] (A_i = +-U_i r_i e^{1/2}); the summed field is rescaled
    so that max |u| <= umax.  rho = 1.  Seed: splitmix64(0x4C42 + run).
    """
    rng = SplitMix64(0x4C42 + run)
    count = rng.integer(2, 8)
    TH, PH = _grid(n_theta, n_phi)
    st, ct = np.sin(TH), np.cos(TH)
    ut = np.zeros_like(TH)
    up = np.zeros_like(TH)
    for _ in range(count):
        ctc = rng.uniform(-1.0, 1.0)
        stc = math.sqrt(max(0.0, 1.0 - ctc * ctc))
        phc = rng.uniform(0.0, 2.0 * math.pi)
        r = rng.uniform(0.1, 0.3)
        U = rng.uniform(0.02, 0.05)
        sign = 1.0 if rng.uniform() < 0.5 else -1.0
        A = sign * U * r * math.exp(0.5)
        dph = PH - phc
        cosd = np.clip(ct * ctc + st * stc * np.cos(dph), -1.0, 1.0)
        d = np.arccos(cosd)
        sind = np.sin(d)
        ratio = np.where(d > 1e-12, d / np.where(sind > 0, sind, 1.0), 1.0)
        e = A * np.exp(-d * d / (2 * r * r)) * ratio / (r * r)
        ut += e * stc * np.sin(dph)
        up += e * (ct * stc * np.cos(dph) - st * ctc)
    speed = np.sqrt(ut * ut + up * up).max()
    if speed > umax:
        ut *= umax / speed
        up *= umax / speed
    return np.ones_like(TH), ut, up, None
