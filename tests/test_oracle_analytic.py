"""Whole-method pins of the oracle against the paper's closed-form solutions.

- shear P_2^1 mode on the 32 x 64 grid (odd shear mode n = 0, kappa^o_0 = 4 nu,
  Eq. shear_kappaon with nu = tau, App. A.4): the amplitude decays as
  exp(-4 tau t) after the initial kinetic transient of length ~tau;
- axisymmetric shear wave u^phi_0 = V0 (Sec. 4.2, App. B.2): mode amplitudes
  V^e_n(t) = v^e_n exp(-kappa^e_n t) with the printed v^e_n and the undamped n = 0;
- axisymmetric sound wave u^theta_0 = U0 (pi - theta) theta (Sec. 4.1, App. B.1):
  U^e_n(t) of Eq. (sound_amplitudes) with the printed initial amplitudes.
"""
import math
import os

import numpy as np
import pytest

import analytic as A
import oracle
from conftest import GOLDEN
from paper_2504_15574_gb300 import inputs


def test_printed_mode_functions_match_jacobi_definition():
    th = np.linspace(0.05, 3.0, 9)
    g = A.load_golden(os.path.join(GOLDEN, "axisymmetric_modes.txt"), th=th)
    for n in (1, 2, 3):
        assert np.allclose(A.sound_F_even(n, th), g[f"F{n}"], rtol=1e-13, atol=1e-14)
    for n in (0, 2, 3):
        assert np.allclose(A.shear_G_even(n, th), g[f"G{n}"], rtol=1e-13, atol=1e-14)
    # The printed G^e_1 carries sqrt(21/32) where the normalisation of Eq. (shear_Gen)
    # (and the printed amplitude v^e_1) give sqrt(21/128): a factor 2 typo.
    assert np.allclose(A.shear_G_even(1, th), g["G1"] / 2, rtol=1e-13, atol=1e-14)


def test_printed_initial_amplitudes_match_projections():
    nt = 40000
    th = (np.arange(nt) + 0.5) * math.pi / nt
    g = A.load_golden(os.path.join(GOLDEN, "axisymmetric_modes.txt"), th=th)
    for n in (1, 2, 3):
        assert A.project_sound((math.pi - th) * th, th, n) == pytest.approx(g[f"u{n}"], rel=1e-9)
    for n in (0, 1, 2, 3):
        assert A.project_shear(np.ones(nt), th, n) == pytest.approx(g[f"v{n}"], rel=1e-9)


def _p21_amplitude(o, th):
    _, _, up = o.moments()
    basis = -3e-3 * np.sin(th) * np.cos(th)
    w = np.sin(th)
    return float((up[:, 0] * basis * w).sum() / (basis * basis * w).sum()), up


def test_p21_shear_mode_decays_at_four_tau():
    nt, np_, tau = 32, 64, 0.02
    dt = 0.25 * (math.pi / nt) / math.sqrt(3 + math.sqrt(6))    # 1.0515e-2, the literal rule
    o = oracle.Oracle(nt, np_, tau=tau, dt=dt)
    o.init_moments(*inputs.shear_p21(nt, np_)[:3])
    th, _ = inputs.cell_centres(nt, np_)
    o.step(100)
    a1, _ = _p21_amplitude(o, th)
    o.step(400)
    a2, up = _p21_amplitude(o, th)
    rate = math.log(a1 / a2) / (400 * dt)
    assert rate == pytest.approx(4 * tau, rel=5e-3)
    # literal dt stays stable here because the run is exactly axisymmetric
    assert np.array_equal(up, np.broadcast_to(up[:, :1], up.shape))


@pytest.fixture(scope="module")
def shear_runs():
    out = {}
    for nt in (64, 128):
        o = oracle.Oracle(nt, 1, tau=1e-3, dt=1e-4)
        o.init_moments(*inputs.shear_uniform(nt, 1, 1e-5)[:3])
        o.step(5000)
        out[nt] = (o.moments()[2][:, 0], o.diagnostics()["t"])
    return out


def test_shear_wave_amplitudes(shear_runs):
    errs = {}
    for nt, (up, t) in shear_runs.items():
        th, _ = inputs.cell_centres(nt, 1)
        errs[nt] = []
        for n in range(4):
            v0 = A.project_shear(np.ones(20000), (np.arange(20000) + 0.5) * math.pi / 20000, n)
            theory = v0 * math.exp(-A.shear_kappa(n, 1e-3) * t)
            errs[nt].append(abs(A.project_shear(up, th, n) / 1e-5 - theory))
    assert max(errs[128]) < 1e-4, errs
    # converges with resolution
    assert all(e128 < e64 / 3 for e64, e128 in zip(errs[64], errs[128])), errs


def test_sound_wave_amplitudes():
    nt, tau, dt, U0 = 128, 2e-3, 1e-4, 1e-5
    o = oracle.Oracle(nt, 1, tau=tau, dt=dt)
    rho, ut, up, _ = inputs.sound_parabola(nt, 1, U0)
    o.init_moments(rho, ut, up)
    th, _ = inputs.cell_centres(nt, 1)
    frak = [A.project_sound(ut[:, 0], th, n) / U0 for n in (1, 2, 3)]
    for _ in range(2):
        o.step(2500)
        t = o.diagnostics()["t"]
        ut_sim = o.moments()[1][:, 0]
        for n in (1, 2, 3):
            sim = A.project_sound(ut_sim, th, n) / U0
            theory = A.sound_amplitude(n, t, frak[n - 1], tau)
            assert abs(sim - theory) < 5e-5, (n, t, sim, theory)
