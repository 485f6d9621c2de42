"""Helpers shared by the GPU parity tests: error metrics (reading R17 of the
design notes) and a GPU availability check."""
import math

import numpy as np
import pytest


def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def require_gpu():
    if not gpu_available():
        pytest.skip("needs a CUDA GPU")


def errors(gpu, ora):
    """Relative max errors of (rho, u_theta, u_phi) against the oracle:
    err_rho = max|d rho| / max|rho|, err_drho = max|d rho| / max|rho - mean rho|,
    err_u = max|d u| / max|u| with |.| the vielbein vector magnitude."""
    rg, utg, upg = gpu[:3]
    ro, uto, upo = ora[:3]
    d_r = np.abs(rg - ro).max()
    e = {"rho": d_r / np.abs(ro).max()}
    dev = np.abs(ro - ro.mean()).max()
    e["drho"] = d_r / dev if dev > 0 else 0.0
    du = np.sqrt((utg - uto) ** 2 + (upg - upo) ** 2).max()
    um = np.sqrt(uto**2 + upo**2).max()
    e["u"] = du / um if um > 0 else du
    return e


def literal_dt(nt):
    """dt = 0.25 dtheta / max|xi| (v_max = sqrt(3 + sqrt 6))."""
    return 0.25 * (math.pi / nt) / math.sqrt(3 + math.sqrt(6))


def clamped_dt(nt, np_, tau):
    dth = math.pi / nt
    lim = dth if np_ == 1 else min(dth, math.sin(dth / 2) * 2 * math.pi / np_)
    return min(0.25 * lim / math.sqrt(3 + math.sqrt(6)), tau)
