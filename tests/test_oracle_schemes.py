"""Pins of the oracle's lower-order fluxes and of the Komissarov theta flux
(arXiv 2504.15574 Sec. 3.5, Eqs. fluxes_U1-3, Komissarov_scheme, Komissarov_sin_cos;
Sec. 4.1, Fig. sound_convergence).

- the axisymmetric sound wave of Sec. 4.1 converges at the order of each upwind
  scheme (U1 first, U2 second, U3 third order), against its closed-form amplitudes;
- with the Komissarov flux the order is at most two whatever the reconstruction
  (the interface sines cap it, as the paper states) but the scheme still converges;
- the Komissarov form conserves the mass with the exact cell areas
  R^2 dphi (cos theta_{s-1/2} - cos theta_{s+1/2}) to round-off: no flux crosses a pole;
- rotation about the polar axis and the equatorial mirror commute with a step for
  every scheme.
"""
import math

import numpy as np
import pytest

import analytic as A
import oracle
from paper_2504_15574_gb300 import inputs

TAU, DT, U0, STEPS = 2e-3, 1e-4, 1e-5, 2500
GRIDS = (16, 32, 64)


def _sound_errors(scheme, komissarov):
    """|amplitude - closed form| of the sound modes n = 1, 2, 3 at t = 0.25 per grid."""
    out = []
    for nt in GRIDS:
        o = oracle.Oracle(nt, 1, tau=TAU, dt=DT, scheme=scheme, komissarov=komissarov)
        rho, ut, up, _ = inputs.sound_parabola(nt, 1, U0)
        o.init_moments(rho, ut, up)
        th, _ = inputs.cell_centres(nt, 1)
        o.step(STEPS)
        t = o.diagnostics()["t"]
        u = o.moments()[1][:, 0]
        e = []
        for n in (1, 2, 3):
            frak = A.project_sound((math.pi - th) * th, th, n)
            e.append(abs(A.project_sound(u, th, n) / U0 - A.sound_amplitude(n, t, frak, TAU)))
        out.append(e)
        o.close()
    return np.array(out)


def _orders(errs, mode):
    return np.log2(errs[:-1, mode - 1] / errs[1:, mode - 1])


@pytest.mark.parametrize("scheme,mode,lo,hi", [("u1", 2, 0.8, 1.3), ("u2", 1, 1.7, 2.5), ("u3", 2, 2.5, 3.5)])
def test_upwind_schemes_converge_at_their_order(scheme, mode, lo, hi):
    orders = _orders(_sound_errors(scheme, False), mode)
    assert np.all((orders > lo) & (orders < hi)), orders


@pytest.mark.parametrize("scheme", ["u3", "weno5"])
def test_komissarov_flux_is_at_most_second_order(scheme):
    e = _sound_errors(scheme, True)
    orders = _orders(e, 1)
    assert np.all((orders > 1.0) & (orders < 2.3)), orders
    # the plain form of the same reconstruction is more accurate on the finest grid
    assert e[-1, 0] > 2 * _sound_errors(scheme, False)[-1, 0]


@pytest.mark.parametrize("scheme", ["u1", "u2", "u3", "weno5"])
def test_komissarov_conserves_mass_with_exact_cell_areas(scheme):
    nt, np_ = 12, 16
    rho, ut, up, _ = inputs.gaussian_vortices(nt, np_, run=4, umax=0.1)
    o = oracle.Oracle(nt, np_, tau=0.02, dt=2e-4, scheme=scheme, komissarov=True)
    o.init_moments(rho, ut, up)
    i = np.arange(nt + 1)
    cf = np.cos(i * math.pi / nt)
    area = (cf[:-1] - cf[1:])[:, None] * (2 * math.pi / np_)

    def mass():
        return float((o.moments()[0] * area).sum())

    m0 = mass()
    o.step(20)
    assert abs(mass() - m0) < 1e-13 * m0
    # no flux crosses a pole: the mass budget of the run has nothing to add
    assert o.diagnostics()["pole_budget"] == 0.0


@pytest.mark.parametrize("scheme,komissarov", [("u1", False), ("u3", False), ("u2", True), ("weno5", True)])
def test_phi_rotation_and_mirror_commute_for_every_scheme(scheme, komissarov):
    nt, np_, r = 10, 12, 5
    rho, ut, up, _ = inputs.gaussian_vortices(nt, np_, run=9)
    base = oracle.Oracle(nt, np_, tau=0.05, dt=5e-4)
    base.init_moments(rho, ut, up)
    f = base.get_populations() * (1.0 + 0.02 * inputs.SplitMix64(9).normal_array((16, nt, np_)))
    perm = np.array([4 * (3 - (k // 4)) + k % 4 for k in range(16)])
    mirror = lambda x: x[perm][:, ::-1, :]
    runs = {}
    for name, g in (("a", f), ("rot", np.roll(f, r, axis=2)), ("mir", mirror(f))):
        o = oracle.Oracle(nt, np_, tau=0.05, dt=5e-4, scheme=scheme, komissarov=komissarov)
        o.set_populations(g)
        o.step(3)
        runs[name] = o.get_populations()
    assert np.array_equal(np.roll(runs["a"], r, axis=2), runs["rot"])
    assert np.abs(mirror(runs["a"]) - runs["mir"]).max() < 1e-14
