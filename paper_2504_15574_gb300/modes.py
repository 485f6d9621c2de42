"""Sound and shear modes of degree l on a 256 x 512 grid against their closed-form evolution
(arXiv 2504.15574 Sec. 4.1, 4.2, App. B; the non-axisymmetric sets of the reading that every
Y_l^m mode of a degree evolves as the axisymmetric one).

Starts (inputs.sound_legendre / shear_legendre): rho = 1 + A f_l, u = 0, and the toroidal flow
of the stream function A f_l, with f_l = sum_{m <= l} P_l^m(cos theta) cos(m phi + alpha_m) / (l + 1)
(Schmidt semi-normalised, seeded phases), A = 1e-3.  Both are eigenfields of the linearised
isothermal Navier-Stokes operator on the unit sphere (c_s^2 = 1, nu = nu_v = tau for the Q = 4
BGK model), so the whole field keeps its shape and its amplitude obeys, with lam2 = l (l + 1):
  sound:  a(t) = e^{-g t} (cos w t + (g / w) sin w t),  g = tau (lam2 - 1),  w = sqrt(lam2 - g^2);
  shear:  a(t) = e^{-k t},                                k = tau (lam2 - 2).
The amplitude of a run is its projection on the initial field (area-weighted: rho - 1 for sound,
(u^theta, u^phi) for shear).  Both time-step choices of the configuration are run: the clamped
dt (8.064e-6 at 256 x 512, filter off, 10^4 steps to t = 0.081) and the literal
dt = 0.25 dtheta / v_max with the polar filter (1.314e-3, 10^4 steps to t = 13.1).  Reported per
run: the largest |a_run - a_closed| over the report times, in units of the initial amplitude,
and the device throughput.  FP32 for every run, FP64 for two (its steps are 1/64-rate FP64).

Not a parity test: the closed forms are the Navier-Stokes limit, which the kinetic model meets
up to corrections of order tau.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import inputs, vlbm

VMAX = {"d2q16": math.sqrt(3 + math.sqrt(6)), "d2q9": math.sqrt(3.0)}


def closed_form(kind, ell, tau, t):
    lam2 = ell * (ell + 1)
    if kind == "sound":
        g = tau * (lam2 - 1)
        w = math.sqrt(lam2 - g * g)
        return math.exp(-g * t) * (math.cos(w * t) + g / w * math.sin(w * t))
    return math.exp(-tau * (lam2 - 2) * t)


def run(kind, ell, tau, literal, precision, nt=256, np_=512, steps=10000, reports=10, velocity_set="d2q16"):
    dth, vmax = math.pi / nt, VMAX[velocity_set]
    if literal:
        dt = 0.25 * dth / vmax
    else:
        dt = min(0.25 * min(dth, math.sin(dth / 2) * 2 * math.pi / np_) / vmax, tau)
    start = inputs.sound_legendre(nt, np_, ell) if kind == "sound" else inputs.shear_legendre(nt, np_, ell)
    s = vlbm.Solver(nt, np_, tau, dt, precision=precision, polar_filter=literal, velocity_set=velocity_set)
    s.init_moments(*start[:3])
    T, _ = inputs.cell_centres(nt, np_)
    w = np.sin(T)[:, None] * np.ones((1, np_))
    if kind == "sound":
        ref = [start[0] - 1.0]
    else:
        ref = [start[1], start[2]]
    norm = sum((w * r * r).sum() for r in ref)
    worst, done, dev_s, rows = 0.0, 0, 0.0, []
    for k in range(1, reports + 1):
        n = steps * k // reports - done
        s.sync()
        t0 = time.perf_counter()
        s.step(n)
        s.sync()
        dev_s += time.perf_counter() - t0
        done += n
        rho, ut, up = s.moments()
        cur = [rho - 1.0] if kind == "sound" else [ut, up]
        a = sum((w * c * r).sum() for c, r in zip(cur, ref)) / norm
        t = done * dt
        cf = closed_form(kind, ell, tau, t)
        worst = max(worst, abs(a - cf))
        rows.append((t, a, cf))
    s.close()
    return {"kind": kind, "ell": ell, "tau": tau, "dt": dt, "filter": literal, "precision": precision,
            "velocity_set": velocity_set,
            "t_end": done * dt, "a_end": rows[-1][1], "closed_end": rows[-1][2], "max_abs_dev": worst,
            "mlups": nt * np_ * done / dev_s / 1e6}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--out", default=None)
    ap.add_argument("--velocity-set", default="d2q16", choices=["d2q16", "d2q9"],
                    help="d2q9: the FP32 runs only")
    a = ap.parse_args(argv)
    vlbm.load()
    res = []
    if a.velocity_set == "d2q9":
        for literal in (False, True):
            for tau in (0.005, 0.02):
                for kind in ("sound", "shear"):
                    for ell in (1, 2, 3, 4):
                        r = run(kind, ell, tau, literal, "fp32", steps=a.steps, velocity_set="d2q9")
                        res.append(r)
                        print(json.dumps(r), flush=True)
        if a.out:
            with open(a.out, "w") as fh:
                json.dump(res, fh)
        return
    for literal in (False, True):
        for tau in (0.005, 0.02):
            for kind in ("sound", "shear"):
                for ell in (1, 2, 3, 4):
                    r = run(kind, ell, tau, literal, "fp32", steps=a.steps)
                    res.append(r)
                    print(json.dumps(r), flush=True)
    for kind, ell in (("sound", 2), ("shear", 3)):
        r = run(kind, ell, 0.02, False, "fp64", steps=a.steps)
        res.append(r)
        print(json.dumps(r), flush=True)
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(res, fh)


if __name__ == "__main__":
    main()
