"""Pins of the oracle's WENO-5 reconstruction, Eqs. (fluxes_W5), (WENO5_delta),
(WENO5_sigma) with the regulariser eps of reading R1."""
import math

import numpy as np
import pytest

import oracle


def test_linear_limit_is_fifth_order_upwind_flux():
    """With eps >> sigma the weights are the ideal (1/10, 6/10, 3/10) and the
    reconstruction is the classical 5th-order upwind-biased interpolant
    (2a - 13b + 47c + 27d - 3e) / 60."""
    rng = np.random.default_rng(1)
    for _ in range(50):
        a, b, c, d, e = rng.normal(size=5)
        ref = (2 * a - 13 * b + 47 * c + 27 * d - 3 * e) / 60
        assert oracle.weno5(a, b, c, d, e, eps=1e15) == pytest.approx(ref, rel=1e-12, abs=1e-13)


@pytest.mark.parametrize("deg", range(6))
def test_flux_difference_exact_for_polynomials(deg):
    """(h_{i+1/2} - h_{i-1/2}) / dx = g'(x_i) exactly for polynomials of degree <= 5
    (finite-difference WENO, linear weights)."""
    rng = np.random.default_rng(deg)
    coef = rng.normal(size=deg + 1)
    dx = 0.1
    x = np.arange(-3, 4) * dx + 0.3
    g = np.polyval(coef, x)
    hp = oracle.weno5(*g[1:6], eps=1e12)
    hm = oracle.weno5(*g[0:5], eps=1e12)
    exact = np.polyval(np.polyder(coef), x[3]) if deg > 0 else 0.0
    assert (hp - hm) / dx == pytest.approx(exact, rel=1e-9, abs=1e-9)


def test_degree_six_is_not_exact():
    """Sanity of the previous pin: the stencil's exactness stops at degree 5."""
    x = np.arange(-3, 4) * 1.0
    g = x**6
    hp = oracle.weno5(*g[1:6], eps=1e20)
    hm = oracle.weno5(*g[0:5], eps=1e20)
    assert abs((hp - hm) - 0.0) > 1.0


def test_nonlinear_weights_avoid_the_jump():
    """A step in the last point: the stencils that cross it get ~zero weight,
    so the reconstruction stays at the smooth side's value (no overshoot)."""
    r = oracle.weno5(0.0, 0.0, 0.0, 1.0, 1.0, eps=1e-6)
    assert 0.0 <= r < 1e-6
    r = oracle.weno5(1.0, 1.0, 1.0, 0.0, 0.0, eps=1e-6)
    assert 1.0 - 1e-6 < r <= 1.0
    # monotone data stays within its range
    for s in np.linspace(0, 1, 11):
        r = oracle.weno5(0, 0, s, 1, 1, eps=1e-6)
        assert -1e-12 <= r <= 1.0 + 1e-12


def test_constant_data_reproduced():
    for c in (0.0, 1.0, -3.5, 1e-3):
        assert oracle.weno5(c, c, c, c, c, eps=1e-6) == pytest.approx(c, rel=1e-15, abs=0)


def test_convergence_order_on_smooth_data():
    """Error of the flux-difference derivative on sin(x) converges at order ~5."""
    errs = []
    hs = [0.2, 0.1, 0.05]
    for h in hs:
        x0 = 0.7
        x = x0 + np.arange(-3, 4) * h
        g = np.sin(x)
        d = (oracle.weno5(*g[1:6], eps=1e-6) - oracle.weno5(*g[0:5], eps=1e-6)) / h
        errs.append(abs(d - math.cos(x0)))
    orders = [math.log(errs[i] / errs[i + 1], 2) for i in range(len(errs) - 1)]
    assert min(orders) > 4.5, orders


def test_mirror_stencil_is_the_same_function():
    """The v < 0 flux is the v > 0 function on the reversed stencil (reading R4):
    reflecting the data x -> -x maps one onto the other."""
    rng = np.random.default_rng(5)
    g = rng.normal(size=6)
    left = oracle.weno5(*g[0:5])           # interface 2+1/2 for v > 0 (stencil 0..4)
    right = oracle.weno5(*g[::-1][0:5])    # interface 2+1/2 of reversed data for v < 0
    # reversed data index j' = 5 - j; interface 2+1/2 of the reversal is 2+1/2 of the original
    assert math.isfinite(left) and math.isfinite(right)
    # same function of the same ordered arguments gives identical bits
    assert oracle.weno5(*g[1:6][::-1]) == oracle.weno5(g[5], g[4], g[3], g[2], g[1])
