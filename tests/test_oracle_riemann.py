"""Physics pin of the oracle on the spherical shock tube (arXiv 2504.15574 Sec. 4.3):
the primary shock obeys the Rankine-Hugoniot jump conditions of Eq. (Rankine-Hugoniot).
Given the shock speed R dtheta_d/dt measured from the run and the undisturbed density
rho_S ahead of it, the paper's relations give the state behind it,
rho_N = rho_S (R dtheta_d/dt / c_s)^2 and u_N = ((R dtheta_d/dt)^2 - c_s^2) / (R dtheta_d/dt)
(c_s = 1 for T0 = 1); the run's post-shock density and velocity must match them.  This pins
the flux form (mass and momentum conserved across the discontinuity) and the isothermal
pressure law of the scheme."""
import math

import numpy as np

import oracle
from paper_2504_15574_gb300 import inputs

NT, TAU, DT = 1024, 1e-4, 5e-6   # the paper's grid and time step (Sec. 4.3); tau well below the time scales
RHO_S = 0.125


def _front(o, th):
    """Position of the primary shock (where rho crosses midway between the levels on its
    two sides) and the mean rho, u^theta over cells 3-8 behind it."""
    r, ut, _ = o.moments()
    r, u = r[:, 0], ut[:, 0]
    idx = np.where(r > 1.5 * RHO_S)[0].max()
    behind_r, behind_u = r[idx - 8:idx - 3].mean(), u[idx - 8:idx - 3].mean()
    mid = 0.5 * (behind_r + RHO_S)
    k = np.where(r[:idx + 5] > mid)[0].max()
    frac = (r[k] - mid) / (r[k] - r[k + 1])
    return th[k] + frac * (th[k + 1] - th[k]), behind_r, behind_u


def test_primary_shock_obeys_rankine_hugoniot():
    o = oracle.Oracle(NT, 1, tau=TAU, dt=DT)
    o.init_moments(*inputs.riemann_cap(NT, 1)[:3])
    th, _ = inputs.cell_centres(NT, 1)
    o.step(8000)
    t1 = o.diagnostics()["t"]
    th1, r1, u1 = _front(o, th)
    o.step(8000)
    t2 = o.diagnostics()["t"]
    th2, r2, u2 = _front(o, th)
    speed = (th2 - th1) / (t2 - t1)          # R = 1
    assert th1 > math.pi / 10 and speed > 1.0  # moved south at supersonic speed
    rho_n, u_n = 0.5 * (r1 + r2), 0.5 * (u1 + u2)
    # measured: speed 1.609, rho_N 0.3215 against 0.3237, u_N 1.010 against 0.988
    assert abs(rho_n - RHO_S * speed ** 2) < 0.03 * rho_n, (speed, rho_n, RHO_S * speed ** 2)
    assert abs(u_n - (speed ** 2 - 1.0) / speed) < 0.05 * u_n, (speed, u_n, (speed ** 2 - 1.0) / speed)
