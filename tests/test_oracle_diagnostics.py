"""Pins of the oracle's moment read-back, diagnostics and (project-defined,
not in the paper) polar ring filter."""
import math

import numpy as np
import pytest

import oracle
from paper_2504_15574_gb300 import inputs


def test_moments_return_initial_fields_including_temperature():
    nt, np_ = 12, 8
    rho, ut, up, _ = inputs.gaussian_vortices(nt, np_, run=4, umax=0.2)
    T = 1.0 + 0.3 * np.cos(np.arange(nt))[:, None] * np.ones((1, np_))
    o = oracle.Oracle(nt, np_, tau=0.01, dt=1e-4)
    o.init_moments(rho, ut, up, T)
    r2, ut2, up2, T2 = o.moments(with_T=True)
    assert np.allclose(r2, rho, rtol=1e-14)
    assert np.allclose(ut2, ut, atol=1e-15)
    assert np.allclose(up2, up, atol=1e-15)
    assert np.allclose(T2, T, rtol=1e-13)


def test_diagnostics_closed_forms():
    """Rest state: mass 4 pi R^2, energy sum f|v|^2/2 = n (u^2 + 2T)/2 -> 4 pi.
    Tangential projection of a constant Cartesian velocity U: P = (8 pi / 3) U."""
    nt, np_ = 64, 128
    o = oracle.Oracle(nt, np_, tau=0.01, dt=1e-4)
    TH, PH = np.meshgrid(*inputs.cell_centres(nt, np_), indexing="ij")
    U = np.array([0.01, -0.02, 0.03])
    e_th = np.stack([np.cos(TH) * np.cos(PH), np.cos(TH) * np.sin(PH), -np.sin(TH)])
    e_ph = np.stack([-np.sin(PH), np.cos(PH), 0 * PH])
    ut = np.einsum("a,aij->ij", U, e_th)
    up = np.einsum("a,aij->ij", U, e_ph)
    o.init_moments(np.ones_like(TH), ut, up)
    d = o.diagnostics()
    # midpoint sum of sin over the cell centres: sum_i sin(theta_i) = 1 / sin(dth / 2)
    dth = math.pi / nt
    assert d["mass"] == pytest.approx(2 * math.pi * dth / math.sin(dth / 2), rel=1e-13)
    assert d["mass"] == pytest.approx(4 * math.pi, rel=2e-4)
    assert np.allclose([d["px"], d["py"], d["pz"]], 8 * math.pi / 3 * U, rtol=1e-3)
    u2 = ut**2 + up**2
    E = (np.sin(TH) * (u2 + 2.0) / 2).sum() * (math.pi / nt) * (2 * math.pi / np_)
    assert d["energy"] == pytest.approx(E, rel=1e-13)
    assert d["nonfinite"] == 0.0


def test_polar_filter_conserves_ring_mass_and_commutes_with_block_shifts():
    nt, np_ = 16, 64
    o = oracle.Oracle(nt, np_, tau=0.02, dt=1e-4, polar_filter=True)
    _, _, blocks = o.geometry()
    assert blocks[0] > 1 and blocks[nt // 2] == 1 and blocks[0] == blocks[-1]
    rho, ut, up, _ = inputs.gaussian_vortices(nt, np_, run=9)
    o.init_moments(rho, ut, up)
    f0 = o.get_populations()
    o.step(1)
    f1 = o.get_populations()
    # after the step every filtered ring is constant over aligned blocks
    for i in range(nt):
        b = blocks[i]
        if b > 1:
            blk = f1[:, i, :].reshape(16, np_ // b, b)
            assert np.array_equal(blk, np.broadcast_to(blk[:, :, :1], blk.shape))
    d = o.diagnostics()
    assert abs((d["mass"] - d["mass0"]) - d["pole_budget"]) < 1e-13 * d["mass0"]
    # shifting by a multiple of the largest block commutes bitwise
    r = int(blocks.max())
    p = oracle.Oracle(nt, np_, tau=0.02, dt=1e-4, polar_filter=True)
    p.set_populations(np.roll(f0, r, axis=2))
    p.step(1)
    assert np.array_equal(np.roll(f1, r, axis=2), p.get_populations())
