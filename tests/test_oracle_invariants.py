"""Pins of the oracle's operator and stepper by invariants the paper fixes.

- collision and force conserve mass per cell (App. A.3 identities), and the
  force supplies exactly the geometric momentum sources of the Navier-Stokes
  equations on the sphere (Eqs. NSE_sph: +cot(theta)/R Pi^{phi phi} for the theta
  momentum, -cot(theta)/R Pi^{theta phi} for the phi momentum);
- the global mass changes only through the pole fluxes (reading R6);
- rotation about the polar axis by whole cells commutes with a step, bitwise;
- axisymmetric data stays axisymmetric, bitwise;
- the equatorial mirror commutes with a step;
- the rest state is a steady state up to the WENO truncation error (5th order);
- the time stepper is the Shu-Osher SSP-RK3 of Sec. 3.7.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2504_15574_gb300 import inputs


def _noisy_state(nt, np_, seed=3, amp=0.02):
    """Near-equilibrium populations with random, unsymmetric perturbations."""
    rho, ut, up, _ = inputs.gaussian_vortices(nt, np_, run=seed)
    o = oracle.Oracle(nt, np_, tau=0.05, dt=1e-3)
    o.init_moments(rho, ut, up)
    f = o.get_populations()
    rng = inputs.SplitMix64(seed)
    noise = rng.normal_array(f.shape)
    return f * (1.0 + amp * noise)


def _V():
    v, _ = oracle.quadrature()
    return np.repeat(v, 4), np.tile(v, 4)


def test_mass_and_momentum_sources_per_cell():
    nt, np_ = 8, 6
    o = oracle.Oracle(nt, np_, tau=0.05, dt=1e-3)
    g = _noisy_state(nt, np_)
    L, Ft, Fp, _ = o.operator(g)
    va, vb = _V()
    s, c, _ = o.geometry()
    dth, dph = math.pi / nt, 2 * math.pi / np_
    R = 1.0
    divt = -(Ft[:, 1:, :] - Ft[:, :-1, :]) / (R * s[None, :, None] * dth)
    divp = -(Fp[:, :, 1:] - Fp[:, :, :-1]) / (R * s[None, :, None] * dph)
    adv = divt + divp
    scale = np.abs(L).max()
    # mass: collision and force add nothing
    assert np.abs(L.sum(0) - adv.sum(0)).max() < 1e-13 * scale
    # theta momentum: BGK adds nothing, -force adds +cot/R * Pi^{phi phi}
    cot = (c / s)[:, None]
    Pi_pp = np.einsum("k,kij->ij", vb * vb, g)
    Pi_tp = np.einsum("k,kij->ij", va * vb, g)
    lhs_t = np.einsum("k,kij->ij", va, L - adv)
    assert np.abs(lhs_t - cot / R * Pi_pp).max() < 1e-12 * scale
    lhs_p = np.einsum("k,kij->ij", vb, L - adv)
    assert np.abs(lhs_p + cot / R * Pi_tp).max() < 1e-12 * scale


def test_mass_budget_closes_through_pole_fluxes():
    nt, np_ = 12, 8
    o = oracle.Oracle(nt, np_, tau=0.05, dt=2e-4)
    o.set_populations(_noisy_state(nt, np_, seed=7))
    o.step(15)
    d = o.diagnostics()
    assert abs(d["pole_budget"]) > 1e-9          # the pole flux is not zero (reading R5)
    assert abs((d["mass"] - d["mass0"]) - d["pole_budget"]) < 1e-13 * d["mass0"]


def test_pole_flux_budget_shrinks_with_resolution():
    """The mass leak through the poles is a truncation error: it converges to 0."""
    leaks = []
    for nt in (16, 32, 64):
        np_ = 2 * nt
        rho, ut, up, _ = inputs.sound_legendre(nt, np_, ell=2, amplitude=1e-2)
        o = oracle.Oracle(nt, np_, tau=0.02, dt=1e-5)
        o.init_moments(rho, ut, up)
        L, Ft, Fp, m = o.operator(o.get_populations())
        leaks.append(abs(m))
    assert leaks[1] < leaks[0] / 4 and leaks[2] < leaks[1] / 4, leaks


def test_phi_rotation_commutes_bitwise():
    nt, np_, r = 10, 12, 5
    f = _noisy_state(nt, np_, seed=11)
    a = oracle.Oracle(nt, np_, tau=0.05, dt=5e-4)
    b = oracle.Oracle(nt, np_, tau=0.05, dt=5e-4)
    a.set_populations(f)
    b.set_populations(np.roll(f, r, axis=2))
    a.step(3)
    b.step(3)
    assert np.array_equal(np.roll(a.get_populations(), r, axis=2), b.get_populations())


def test_axisymmetric_state_stays_axisymmetric_bitwise():
    nt, np_ = 16, 8
    rho, ut, up, _ = inputs.shear_p21(nt, np_)
    o = oracle.Oracle(nt, np_, tau=0.02, dt=1e-3)
    o.init_moments(rho + 0.01 * np.cos(np.linspace(0, 3, nt))[:, None], ut, up)
    o.step(5)
    f = o.get_populations()
    assert np.array_equal(f, np.broadcast_to(f[:, :, :1], f.shape))


def test_equatorial_mirror_commutes():
    """theta -> pi - theta with v_theta -> -v_theta (population a -> 3 - a)."""
    nt, np_ = 10, 6
    f = _noisy_state(nt, np_, seed=13)
    perm = np.array([4 * (3 - (k // 4)) + k % 4 for k in range(16)])
    mirror = lambda x: x[perm][:, ::-1, :]
    a = oracle.Oracle(nt, np_, tau=0.05, dt=5e-4)
    b = oracle.Oracle(nt, np_, tau=0.05, dt=5e-4)
    a.set_populations(f)
    b.set_populations(mirror(f))
    a.step(3)
    b.step(3)
    assert np.abs(mirror(a.get_populations()) - b.get_populations()).max() < 1e-14


def test_rest_state_tendency_is_weno_truncation():
    """rho = 1, u = 0: advection of sin(theta) w and the force cancel up to the
    5th-order truncation error of the theta flux difference."""
    errs = []
    for nt in (16, 32, 64):
        o = oracle.Oracle(nt, 2, tau=0.02, dt=1e-5)
        one = np.ones((nt, 2))
        o.init_moments(one, 0 * one, 0 * one)
        L, _, _, _ = o.operator(o.get_populations())
        errs.append(np.abs(L).max())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[0] < 1e-3 and min(orders) > 3.5, (errs, orders)


def test_step_is_shu_osher_rk3():
    """One oracle step equals the three stages of Sec. 3.7 composed from the
    oracle's own operator L."""
    nt, np_ = 8, 4
    dt = 3e-4
    f = _noisy_state(nt, np_, seed=17)
    o = oracle.Oracle(nt, np_, tau=0.05, dt=dt)
    L = lambda g: o.operator(g)[0]
    f1 = f + dt * L(f)
    f2 = 0.75 * f + 0.25 * f1 + 0.25 * dt * L(f1)
    f3 = f / 3.0 + 2.0 / 3.0 * f2 + 2.0 / 3.0 * dt * L(f2)
    o.set_populations(f)
    o.step(1)
    assert np.abs(o.get_populations() - f3).max() < 1e-15 * np.abs(f).max()


def test_rk3_amplification_on_bgk_relaxation():
    """On a uniform-in-phi, no-flow state with a non-equilibrium part that only
    relaxes (populations symmetric so that advection is negligible on a short
    step), the decay of f - f^eq over one step follows the RK3 polynomial
    1 + z + z^2/2 + z^3/6, z = -dt/tau, up to the small advective part."""
    nt, np_ = 32, 2
    tau = 1e-3
    dt = 5e-4
    o = oracle.Oracle(nt, np_, tau=tau, dt=dt)
    one = np.ones((nt, np_))
    o.init_moments(one, 0 * one, 0 * one)
    feq = o.get_populations()
    # add a non-equilibrium part that carries no mass or momentum
    va, vb = _V()
    pert = (va * va - vb * vb)[:, None, None] * feq * 1e-3
    o.set_populations(feq + pert)
    o.step(1)
    z = -dt / tau
    amp = 1 + z + z * z / 2 + z**3 / 6
    got = o.get_populations() - feq
    mid = slice(nt // 4, 3 * nt // 4)
    live = np.abs(va * va - vb * vb) > 1.0
    ratio = got[live][:, mid] / pert[live][:, mid]
    assert np.abs(ratio - amp).max() < 3e-3  # RK2 would be off by 2e-2, Euler by 0.1
