"""Closed-form axisymmetric solutions of arXiv 2504.15574 App. B, used as pins.

Everything here is written from App. B: the Jacobi-polynomial series
(Eq. Jacobi_series), the normalised acoustic modes F^e_n (Eq. sound_Fen) with
lambda^2_{e;n} = 2n(2n-1) (Eq. sound_lambda_aux) and damping/frequency
(Eq. sound_damping_coeffs with nu = nu_v), and the shear modes G^e_n
(Eq. shear_Gen) with kappa^e_n = 2n(2n+3) nu / R^2 (Eq. shear_kappaen).
Projections follow Eqs. (sound_uncos) and (shear_veon).  Transport
coefficients: Q = 4 BGK gives eta = zeta = tau p (App. A.4), so nu = nu_v = tau
and c_s^2 = T0 = 1 in lattice units with R = 1.
"""
import math

import numpy as np


def jacobi(n, alpha, beta, x):
    """P_n^{(alpha,beta)}(x) from the explicit series, Eq. (Jacobi_series)."""
    x = np.asarray(x, dtype=np.float64)
    pre = math.gamma(alpha + n + 1) / (math.factorial(n) * math.gamma(alpha + beta + n + 1)) \
        if (alpha + beta + n + 1) > 0 or float(alpha + beta + n + 1).is_integer() is False else None
    total = np.zeros_like(x)
    for m in range(n + 1):
        # Gamma(alpha+beta+n+m+1) / Gamma(alpha+m+1); handle alpha = -1 poles by the
        # ratio of the two factorial-like products (the m = 0 term vanishes then).
        num = _gamma_ratio(alpha + beta + n + m + 1, alpha + m + 1)
        total += math.comb(n, m) * num * ((x - 1.0) / 2.0) ** m
    return _gamma_ratio(alpha + n + 1, None) / math.factorial(n) * total / _gamma_or_inf(alpha + beta + n + 1)


def _gamma_or_inf(z):
    if z <= 0 and float(z).is_integer():
        return math.inf
    return math.gamma(z)


def _gamma_ratio(a, b):
    """Gamma(a) / Gamma(b) with Gamma at non-positive integers treated as a pole
    (a pole in the denominator gives 0); b None means Gamma(a)."""
    ga = _gamma_or_inf(a)
    if b is None:
        return ga
    gb = _gamma_or_inf(b)
    if math.isinf(gb):
        return 0.0
    return ga / gb


def sound_F_even(n, th):
    """F^e_n(theta) = (-1)^n sqrt(n(4n-1)/(2n-1)) P_n^{(-1,-1/2)}(cos 2 theta).

    The series prefactor Gamma(alpha+n+1)/Gamma(alpha+beta+n+1) is finite for
    alpha = -1, n >= 1; evaluated with the factorial form of the series."""
    alpha, beta = -1.0, -0.5
    x = np.cos(2.0 * np.asarray(th, dtype=np.float64))
    total = np.zeros_like(x)
    for m in range(n + 1):
        if alpha + m + 1 <= 0:
            continue  # 1/Gamma(0) = 0
        total += math.comb(n, m) * math.gamma(alpha + beta + n + m + 1) / math.gamma(alpha + m + 1) \
            * ((x - 1.0) / 2.0) ** m
    P = math.gamma(alpha + n + 1) / (math.factorial(n) * math.gamma(alpha + beta + n + 1)) * total
    return (-1) ** n * math.sqrt(n * (4 * n - 1) / (2 * n - 1)) * P


def shear_G_even(n, th):
    """G^e_n(theta) = sqrt((2n+1)(4n+3)/(4(n+1))) P_n^{(1,-1/2)}(cos 2 theta)."""
    alpha, beta = 1.0, -0.5
    x = np.cos(2.0 * np.asarray(th, dtype=np.float64))
    total = np.zeros_like(x)
    for m in range(n + 1):
        total += math.comb(n, m) * math.gamma(alpha + beta + n + m + 1) / math.gamma(alpha + m + 1) \
            * ((x - 1.0) / 2.0) ** m
    P = math.gamma(alpha + n + 1) / (math.factorial(n) * math.gamma(alpha + beta + n + 1)) * total
    return math.sqrt((2 * n + 1) * (4 * n + 3) / (4 * (n + 1))) * P


def sound_rates(n, tau, R=1.0, cs2=1.0):
    """(gamma, omega) of even sound mode n with nu = nu_v = tau."""
    lam2 = 2 * n * (2 * n - 1)
    nu = tau
    gamma = nu / R**2 * (lam2 - 1)
    omega = math.sqrt(lam2 * cs2 / R**2 - gamma**2)
    return gamma, omega


def sound_amplitude(n, t, frak_u, tau):
    """U^e_n(t) = frak_u e^{-gamma t} (cos omega t - gamma/omega sin omega t), Eq. (sound_amplitudes)."""
    g, w = sound_rates(n, tau)
    return frak_u * math.exp(-g * t) * (math.cos(w * t) - g / w * math.sin(w * t))


def shear_kappa(n, tau, R=1.0):
    return tau / R**2 * 2 * n * (2 * n + 3)


def project_sound(ut_profile, th, n):
    """U_n = int_0^pi dtheta u^theta F^e_n (Eq. sound_uncos), midpoint rule on the cell centres."""
    dth = math.pi / len(th)
    return float(np.sum(ut_profile * sound_F_even(n, th)) * dth)


def project_shear(up_profile, th, n):
    """V_n = int_0^pi dtheta sin^2 u^phi G^e_n (Eq. shear_veon), midpoint rule."""
    dth = math.pi / len(th)
    return float(np.sum(np.sin(th) ** 2 * up_profile * shear_G_even(n, th)) * dth)


def load_golden(path, **names):
    """Evaluates 'name = expr' lines of a golden fixture with math functions in scope."""
    env = {"sqrt": math.sqrt, "pi": math.pi, "cos": np.cos, "sin": np.sin}
    env.update(names)
    out = {}
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, e = line.split("=", 1)
            out[k.strip()] = eval(e, {"__builtins__": {}}, env)
    return out
