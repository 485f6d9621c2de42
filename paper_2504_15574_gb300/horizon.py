"""The 1024 x 2048 axisymmetric shock cap over its full horizon of 2 x 10^4 RK3 steps on the FP32
path (arXiv 2504.15574 Sec. 3.7 stepping, WENO-5 of Eqs. fluxes_W5 - WENO5_sigma, pole boundary
Eq. bcs_theta; polar ring filter on, dt = 0.25 dtheta / v_max, tau = 1e-3; cap theta < 0.2 at
rho = 4, T = 1.5, rho = 1, T = 1 elsewhere, u = 0).

Every `--every` steps it records, from the library's FP64 reductions of the FP32 state
(vlbm_diagnostics): the mass, its change against the accumulated pole mass-flux budget
(mass - mass0 - pole_flux, reading R6: the only mass the method may lose crosses the pole faces),
the energy sum f |v|^2 / 2 (reported; the isothermal BGK target does not conserve it), the
non-finite guard, and from the moments whether rho and u^theta are still the same in every column
bit for bit (the start and the method are axisymmetric) with the largest |u^phi|.  Prints a
markdown table and one JSON line with the device time of the steps.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import inputs, vlbm


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--every", type=int, default=1000)
    ap.add_argument("--n-theta", type=int, default=1024)
    ap.add_argument("--n-phi", type=int, default=2048)
    a = ap.parse_args(argv)
    import torch

    nt, np_ = a.n_theta, a.n_phi
    dt = 0.25 * (math.pi / nt) / math.sqrt(3 + math.sqrt(6))
    stream = torch.cuda.Stream()
    s = vlbm.Solver(nt, np_, 1e-3, dt, precision="fp32", polar_filter=True, stream=stream.cuda_stream)
    s.init_moments(*inputs.shock_cap(nt, np_))
    d0 = s.diagnostics()
    rows = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dev_ms = 0.0
    t_wall = time.perf_counter()
    done = 0
    while done < a.steps:
        n = min(a.every, a.steps - done)
        ev0.record(stream)
        s.step(n)
        ev1.record(stream)
        torch.cuda.synchronize()
        dev_ms += ev0.elapsed_time(ev1)
        done += n
        d = s.diagnostics()
        r, ut, up = s.moments()
        axis = bool(np.array_equal(r, np.broadcast_to(r[:, :1], r.shape)) and
                    np.array_equal(ut, np.broadcast_to(ut[:, :1], ut.shape)))
        rows.append({"step": done, "t": d["time"], "mass_rel": d["mass"] / d0["mass"] - 1.0,
                     "closure_rel": (d["mass"] - d["mass0"] - d["pole_flux"]) / d["mass0"],
                     "pole_flux_rel": d["pole_flux"] / d["mass0"], "energy_rel": d["energy"] / d0["energy"] - 1.0,
                     "nonfinite": d["nonfinite"], "axisymmetric": axis, "max_u_phi": float(np.abs(up).max()),
                     "rho_min": float(r.min()), "rho_max": float(r.max())})
    wall = time.perf_counter() - t_wall
    print("| step | t | mass / mass0 - 1 | (mass - mass0 - pole flux) / mass0 | pole flux / mass0 | energy / energy0 - 1 "
          "| non-finite | rho, u^theta the same in every column | max abs(u^phi) | rho min, max |")
    print("|---|---|---|---|---|---|---|---|---|---|")
    for x in rows:
        print(f"| {x['step']} | {x['t']:.4f} | {x['mass_rel']:.3e} | {x['closure_rel']:.3e} | {x['pole_flux_rel']:.3e} "
              f"| {x['energy_rel']:.3e} | {x['nonfinite']} | {'yes' if x['axisymmetric'] else 'no'} "
              f"| {x['max_u_phi']:.2e} | {x['rho_min']:.4f}, {x['rho_max']:.4f} |")
    print(json.dumps({"steps": a.steps, "device_ms_steps": dev_ms, "ms_per_step": dev_ms / a.steps,
                      "mlups": nt * np_ * a.steps / (dev_ms * 1e-3) / 1e6, "wall_s": wall, "records": rows}))
    s.close()


if __name__ == "__main__":
    main()
