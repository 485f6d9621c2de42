"""Isotropy pin of the oracle (arXiv 2504.15574 App. C): the axisymmetric sound wave of
Sec. 4.1 run on a grid rotated by alpha = -pi/2 about the y axis (Eqs. transf,
transf_inv; the wave's axis then lies in the grid's equatorial plane, crossing its
pole rows and its phi seam) agrees with the same wave on the unrotated axisymmetric
grid, and the difference converges at the order of WENO-5 as the paper reports
(Fig. isotropy_test)."""
import math

import numpy as np
import pytest

import oracle
from paper_2504_15574_gb300 import inputs

TAU, DT, U0, STEPS = 2e-3, 1e-4, 1e-5, 2000
ALPHA = -math.pi / 2


def test_rotation_geometry():
    # alpha = 0 is the identity; the rotation maps the original pole onto the grid's equator
    th, ph, M = inputs.rotated_frame(8, 16, 0.0)
    T, P = inputs.cell_centres(8, 16)
    assert np.abs(th - T[:, None]).max() < 1e-14
    assert np.abs(M - np.eye(2)[:, :, None, None]).max() < 1e-14
    th, ph, M = inputs.rotated_frame(16, 16, ALPHA)
    T, P = inputs.cell_centres(16, 16)
    # the component map is a rotation in every cell
    assert np.abs(np.einsum("ji...,jk...->ik...", M, M) - np.eye(2)[:, :, None, None]).max() < 1e-14
    # original north pole (z = 1) sits at theta' = pi/2, phi' = pi of the rotated grid
    i, j = np.unravel_index(np.argmin(th), th.shape)
    assert abs(T[i] - math.pi / 2) < math.pi / 16 and abs(P[j] - math.pi) < 2 * math.pi / 16
    # the rotated start equals the plain one for alpha = 0
    a = inputs.sound_parabola_rotated(8, 16, U0, 0.0)
    b = inputs.sound_parabola(8, 16, U0)
    assert np.allclose(a[1], b[1], rtol=1e-12, atol=0) and np.abs(a[2]).max() < 1e-20


@pytest.fixture(scope="module")
def reference():
    """The wave on the unrotated grid: axisymmetric (n_phi = 1), 512 rows."""
    nt = 512
    o = oracle.Oracle(nt, 1, tau=TAU, dt=DT)
    o.init_moments(*inputs.sound_parabola(nt, 1, U0)[:3])
    o.step(STEPS)
    th, _ = inputs.cell_centres(nt, 1)
    return th, o.moments()[1][:, 0]


def _rotated_error(n, reference):
    th_r, u_r = reference
    o = oracle.Oracle(n, n, tau=TAU, dt=DT)
    o.init_moments(*inputs.sound_parabola_rotated(n, n, U0, ALPHA)[:3])
    o.step(STEPS)
    _, ut, up = o.moments()
    th, _, M = inputs.rotated_frame(n, n, ALPHA)
    # back to the original frame's components (M is orthogonal)
    u_th = M[0, 0] * ut + M[1, 0] * up
    u_ph = M[0, 1] * ut + M[1, 1] * up
    ref = np.interp(th, th_r, u_r)
    T, _ = inputs.cell_centres(n, n)
    w = np.sin(T)[:, None] * np.ones((1, n))
    return math.sqrt((w * ((u_th - ref) ** 2 + u_ph ** 2)).sum() / (w * ref ** 2).sum())


def test_rotated_sound_wave_matches_the_axisymmetric_run_at_fifth_order(reference):
    e = np.array([_rotated_error(n, reference) for n in (16, 32, 64)])
    orders = np.log2(e[:-1] / e[1:])
    # measured: 1.5e-1, 2.4e-3, 4.9e-5 (orders 6.0, 5.6)
    assert e[-1] < 2e-4, e
    assert np.all(orders > 4.5), (e, orders)


# ---- the shock tube on the rotated grid (App. C, Fig. riemann_2D) -----------------------
# The spherical Sod problem of Sec. 4.3 (Eq. riemann_ic: rho 1 / 0.125 at theta = pi/10, at
# rest) about an axis in the grid's equatorial plane.  The paper compares a 1024 x 1024
# rotated run with the 1024 x 1 axisymmetric one and reports agreement without a figure of
# merit; here, at tau = 0.02 (the shock is then resolved, so the comparison converges) and
# t = 1 (the shock has crossed the original equator, where the rotated grid has its poles),
# the rotated runs on 32^2 and 64^2 grids are compared with a 512-row axisymmetric run.
TAU_RIEMANN, T_RIEMANN = 0.02, 1.0
VMAX = math.sqrt(3 + math.sqrt(6))


@pytest.fixture(scope="module")
def shock_reference():
    nt = 512
    dt = 0.25 * (math.pi / nt) / VMAX
    o = oracle.Oracle(nt, 1, tau=TAU_RIEMANN, dt=dt)
    o.init_moments(*inputs.riemann_cap(nt, 1)[:3])
    o.step(int(round(T_RIEMANN / dt)))
    r, u, _ = o.moments()
    th, _ = inputs.cell_centres(nt, 1)
    return th, r[:, 0], u[:, 0]


def _rotated_shock_errors(n, ref):
    """Area-weighted L1 differences of rho, u^theta and |u^phi| (original frame) between the
    rotated n x n run and the axisymmetric reference, relative to the reference's rho - rho2
    and u^theta."""
    th_r, r_r, u_r = ref
    dth = math.pi / n
    dt = 0.25 * min(dth, math.sin(dth / 2) * 2 * math.pi / n) / VMAX
    steps = int(round(T_RIEMANN / dt))
    o = oracle.Oracle(n, n, tau=TAU_RIEMANN, dt=T_RIEMANN / steps)
    o.init_moments(*inputs.riemann_cap_rotated(n, n, ALPHA)[:3])
    o.step(steps)
    r, ut, up = o.moments()
    th, _, M = inputs.rotated_frame(n, n, ALPHA)
    u_th = M[0, 0] * ut + M[1, 0] * up
    u_ph = M[0, 1] * ut + M[1, 1] * up
    rr, uu = np.interp(th, th_r, r_r), np.interp(th, th_r, u_r)
    T, _ = inputs.cell_centres(n, n)
    w = np.sin(T)[:, None] * np.ones((1, n))
    return np.array([(w * np.abs(r - rr)).sum() / (w * np.abs(rr - 0.125)).sum(),
                     (w * np.abs(u_th - uu)).sum() / (w * np.abs(uu)).sum(),
                     (w * np.abs(u_ph)).sum() / (w * np.abs(uu)).sum()])


def test_rotated_shock_tube_converges_to_the_axisymmetric_run(shock_reference):
    e32 = _rotated_shock_errors(32, shock_reference)
    e64 = _rotated_shock_errors(64, shock_reference)
    # measured: rho, u^theta, u^phi 1.37e-1, 1.31e-1, 3.4e-2 (32^2) and 4.1e-2, 4.1e-2, 1.2e-2 (64^2);
    # a phi flux with a wrong metric factor gives 0.34, 0.23, 0.14 at 64^2 and stops converging
    assert np.all(e64 < np.array([0.06, 0.06, 0.02])), (e32, e64)
    assert np.all(e32 / e64 > 2.4), (e32, e64)
