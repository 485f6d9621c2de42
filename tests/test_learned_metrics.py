"""Pins of the learned-coarse judging helpers (host-side numpy): block
downsampling and the discrete vorticity against closed forms."""
import math

import numpy as np
import pytest

from paper_2504_15574_gb300 import inputs
from paper_2504_15574_gb300.learned import downsample, rel_l2, vorticity


def _rotation(H, W, axis, omega=0.02):
    """Solid-body rotation about a Cartesian axis: u = omega (axis x r), tangential."""
    TH, PH = np.meshgrid(*inputs.cell_centres(H, W), indexing="ij")
    r = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)])
    u = omega * np.cross(np.asarray(axis, dtype=float)[:, None, None], r, axis=0)
    e_th = np.stack([np.cos(TH) * np.cos(PH), np.cos(TH) * np.sin(PH), -np.sin(TH)])
    e_ph = np.stack([-np.sin(PH), np.cos(PH), 0 * PH])
    return (u * e_th).sum(0), (u * e_ph).sum(0), r


def test_vorticity_of_solid_body_rotation_is_twice_the_normal_component():
    """omega_r = 2 Omega . r for u = Omega x r (any axis, so the pole ghosts matter)."""
    H, W = 64, 128
    for axis in ([0, 0, 1], [1, 0, 0], [0.3, -0.5, 0.8]):
        ut, up, r = _rotation(H, W, axis)
        expect = 2 * 0.02 * np.einsum("a,ahw->hw", np.asarray(axis, float), r)
        assert rel_l2(vorticity(ut, up), expect) < 2e-3


def test_downsample_preserves_uniform_and_rotating_states():
    Hf, Wf = 32, 64
    one = np.ones((Hf, Wf))
    rc, uc, vc, Tc = downsample(2 * one, 0 * one, 0 * one, 1.5 * one)
    assert np.allclose(rc, 2) and np.allclose(uc, 0) and np.allclose(Tc, 1.5)
    ut, up, _ = _rotation(Hf, Wf, [1, 0, 0])
    _, uc, vc, _ = downsample(one, ut, up, one)
    ut_c, up_c, _ = _rotation(Hf // 4, Wf // 4, [1, 0, 0])
    # block means of a linear Cartesian field equal the centre value up to the block curvature
    assert rel_l2(uc, ut_c) < 0.05 and rel_l2(vc, up_c) < 0.05
    # mass is the area-weighted block mean
    th = (np.arange(Hf) + 0.5) * math.pi / Hf
    rho = 1 + 0.1 * np.cos(th)[:, None] * one
    rc, _, _, _ = downsample(rho, 0 * one, 0 * one, one)
    wf = np.sin(th)[:, None] * one
    wc = wf.reshape(Hf // 4, 4, Wf // 4, 4).sum(axis=(1, 3))
    assert (rc * wc).sum() == pytest.approx((rho * wf).sum(), rel=1e-13)


def test_population_downsampling_keeps_mass_and_density():
    from paper_2504_15574_gb300.learned import downsample_populations
    rng = np.random.default_rng(3)
    Hf, Wf = 16, 32
    f = 0.05 + 0.01 * rng.random((16, Hf, Wf))
    fc = downsample_populations(f)
    rho_f, rho_c = f.sum(0), fc.sum(0)
    rc, _, _, _ = downsample(rho_f, 0 * rho_f, 0 * rho_f, 1 + 0 * rho_f)
    assert np.allclose(rho_c, rc, rtol=1e-14)
