"""Writes tests/golden/oracle_horizons.npz: long-horizon results of the FP64 CPU oracle, the
expected values of tests/test_gpu_horizons.py.  Calls only oracle/ (and the seeded input
generators); nothing here comes from the CUDA path.

Cases (SSP-RK3, Sec. 3.7; WENO-5, Eqs. fluxes_W5 - WENO5_sigma; pole boundary, Eq. bcs_theta):
- "sound_l2", "shear_l3": the degree-l sound and shear sets of the 256 x 512 workload
  (rho = 1 + 1e-3 sum_m Pbar_l^m cos(m phi + alpha_m) / (l + 1), and its stream-function twin),
  D2Q16, tau = 0.02, dt = 0.25 min(dtheta, sin(dtheta / 2) dphi) / v_max (no polar filter),
  10^4 steps.  Stored: rho, u_theta, u_phi on the rows ROWS at every 4th column, and the
  oracle's diagnostics (mass, momentum, energy, pole budget).
- "shock_cap": the 1024 x 2048 shock cap (rho = 4, T = 1.5 for theta < 0.2), tau = 1e-3,
  dt = 0.25 dtheta / v_max with the polar ring filter, 100 steps.  The state is axisymmetric (the
  oracle keeps it independent of phi bit for bit), so column 0 of rho, u_theta, u_phi holds every
  column, plus the diagnostics.

Run: python tests/golden/make_oracle_horizons.py   (about 4 minutes on 16 cores)
"""
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2504_15574_gb300 import inputs  # noqa: E402

VMAX = math.sqrt(3 + math.sqrt(6))
NT2, NP2, STEPS2, TAU2 = 256, 512, 10000, 0.02
# rows kept of the 256 x 512 cases: both polar caps' first rows and a spread over the sphere
ROWS = np.array(sorted(set(list(range(0, 6)) + list(range(250, 256)) + list(range(8, 250, 12)) + [127, 128])))
COLS = np.arange(0, NP2, 4)
NT3, NP3, STEPS3, TAU3 = 1024, 2048, 100, 1e-3


def clamped_dt(nt, np_, tau):
    dth = math.pi / nt
    return min(0.25 * min(dth, math.sin(dth / 2) * 2 * math.pi / np_) / VMAX, tau)


def diag_vector(o):
    d = o.diagnostics()
    return np.array([d["mass"], d["px"], d["py"], d["pz"], d["energy"], d["pole_budget"], d["mass0"]])


def main(out=os.path.join(HERE, "oracle_horizons.npz")):
    res = {"rows": ROWS, "cols": COLS}
    for name, ic in (("sound_l2", inputs.sound_legendre(NT2, NP2, 2)), ("shear_l3", inputs.shear_legendre(NT2, NP2, 3))):
        t0 = time.time()
        o = oracle.Oracle(NT2, NP2, tau=TAU2, dt=clamped_dt(NT2, NP2, TAU2))
        o.init_moments(*ic)
        o.step(STEPS2)
        r, ut, up = o.moments()
        res[name + "_moments"] = np.stack([r, ut, up])[:, ROWS][:, :, COLS]
        res[name + "_diag"] = diag_vector(o)
        print(name, f"{time.time() - t0:.0f} s", flush=True)
    t0 = time.time()
    o = oracle.Oracle(NT3, NP3, tau=TAU3, dt=0.25 * (math.pi / NT3) / VMAX, polar_filter=True)
    o.init_moments(*inputs.shock_cap(NT3, NP3))
    o.step(STEPS3)
    r, ut, up = o.moments()
    for a in (r, ut, up):
        assert np.array_equal(a, np.broadcast_to(a[:, :1], a.shape)), "shock cap lost its axisymmetry"
    res["shock_cap_moments"] = np.stack([r[:, 0], ut[:, 0], up[:, 0]])
    res["shock_cap_diag"] = diag_vector(o)
    print("shock_cap", f"{time.time() - t0:.0f} s", flush=True)
    np.savez_compressed(out, **res)
    print("wrote", out, os.path.getsize(out), "bytes")


if __name__ == "__main__":
    main(*sys.argv[1:])
