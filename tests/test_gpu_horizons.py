"""Long horizons of the CUDA path against the FP64 oracle.  The expected values were written by
tests/golden/make_oracle_horizons.py, which calls only oracle/: the 256 x 512 degree-l sound and
shear sets after 10^4 steps (rows sampled at every 4th column) and the 1024 x 2048 shock cap after
100 steps (axisymmetric: one column holds them all).

FP64: relative max error <= 1e-12 in rho and u on every stored cell, and the diagnostics.
FP32: the error against the oracle stated per case (FP32_BOUND), and the pole mass-flux budget
of the FP32 state closing to a stated bound."""
import math
import os

import numpy as np
import pytest

from parity import errors, require_gpu
from paper_2504_15574_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_horizons.npz")
VMAX = math.sqrt(3 + math.sqrt(6))
NT2, NP2, STEPS2, TAU2 = 256, 512, 10000, 0.02
NT3, NP3, STEPS3, TAU3 = 1024, 2048, 100, 1e-3
CASES2 = {"sound_l2": lambda: inputs.sound_legendre(NT2, NP2, 2), "shear_l3": lambda: inputs.shear_legendre(NT2, NP2, 3)}
# Stated FP32 errors against the FP64 oracle, about 3x the values measured on GB300: rho, drho, u
# as the relative max errors of reading R17 over the stored cells; mass and energy relative to the
# oracle's; pole: |pole flux - oracle's pole budget| / mass; closure: |mass - mass0 - pole flux| /
# mass0 of the FP32 state.  (shear_l3's density deviation is second order in the flow speed,
# ~1e-6 of rho, so its drho measures FP32 rounding on that small scale.)
FP32_BOUND = {
    "sound_l2": {"rho": 3e-7, "drho": 4e-4, "u": 1e-3, "mass": 5e-9, "pole": 1e-11, "closure": 5e-9},
    "shear_l3": {"rho": 2e-7, "drho": 1.2e-2, "u": 5e-4, "mass": 6e-10, "pole": 1e-11, "closure": 6e-10},
    "shock_cap": {"rho": 3e-6, "drho": 4e-6, "u": 3e-6, "mass": 6e-8, "energy": 5e-8, "pole": 3e-11,
                  "closure": 6e-8},
}


@pytest.fixture(scope="module")
def V():
    require_gpu()
    from paper_2504_15574_gb300 import build, vlbm
    build.build()
    vlbm.load()
    return vlbm


@pytest.fixture(scope="module")
def G():
    return dict(np.load(GOLDEN))


def clamped_dt(nt, np_, tau):
    dth = math.pi / nt
    return min(0.25 * min(dth, math.sin(dth / 2) * 2 * math.pi / np_) / VMAX, tau)


def sampled(m, G):
    return [a[G["rows"]][:, G["cols"]] for a in m]


def diag_of(s):
    d = s.diagnostics()
    return d, np.array([d["mass"], d["px"], d["py"], d["pz"], d["energy"], d["pole_flux"], d["mass0"]])


@pytest.mark.parametrize("name", sorted(CASES2))
def test_fp64_10k_steps_256x512(V, G, name):
    s = V.Solver(NT2, NP2, TAU2, clamped_dt(NT2, NP2, TAU2))
    s.init_moments(*CASES2[name]())
    s.step(STEPS2)
    e = errors(sampled(s.moments(), G), G[name + "_moments"])
    print(name, "fp64", e)
    assert e["rho"] <= 1e-12 and e["u"] <= 1e-12, e
    _, dg = diag_of(s)
    do = G[name + "_diag"]
    mass = do[0]
    assert abs(dg[0] - do[0]) <= 1e-12 * mass and abs(dg[4] - do[4]) <= 1e-12 * do[4]
    assert np.abs(dg[1:4] - do[1:4]).max() <= 1e-12 * mass
    assert abs(dg[5] - do[5]) <= 1e-12 * mass   # pole budget
    s.close()


@pytest.mark.parametrize("name", sorted(CASES2))
def test_fp32_10k_steps_256x512(V, G, name):
    s = V.Solver(NT2, NP2, TAU2, clamped_dt(NT2, NP2, TAU2), precision="fp32")
    s.init_moments(*CASES2[name]())
    s.step(STEPS2)
    e = errors(sampled(s.moments(), G), G[name + "_moments"])
    d, dg = diag_of(s)
    do = G[name + "_diag"]
    closure = abs(d["mass"] - d["mass0"] - d["pole_flux"]) / d["mass0"]
    print(name, "fp32", e, "mass", dg[0] / do[0] - 1, "pole flux", dg[5], do[5], "closure", closure)
    b = FP32_BOUND[name]
    assert e["rho"] <= b["rho"] and e["drho"] <= b["drho"] and e["u"] <= b["u"], e
    assert abs(dg[0] / do[0] - 1) <= b["mass"] and abs(dg[5] - do[5]) <= b["pole"] * do[0], (dg, do)
    assert closure <= b["closure"], closure
    s.close()


def test_fp32_shock_cap_100_steps_1024x2048(V, G):
    """The throughput workload (1024 x 2048 shock cap, WENO-5, polar filter, literal dt) over
    100 steps: every cell against the oracle, the state still axisymmetric bit for bit, and the
    FP32 diagnostics against the oracle's."""
    s = V.Solver(NT3, NP3, TAU3, 0.25 * (math.pi / NT3) / VMAX, precision="fp32", polar_filter=True)
    s.init_moments(*inputs.shock_cap(NT3, NP3))
    s.step(STEPS3)
    r, ut, up = s.moments()
    for a in (r, ut):
        assert np.array_equal(a, np.broadcast_to(a[:, :1], a.shape))
    ref = [np.broadcast_to(G["shock_cap_moments"][k][:, None], r.shape) for k in range(3)]
    e = errors((r, ut, up), ref)
    d, dg = diag_of(s)
    do = G["shock_cap_diag"]
    closure = abs(d["mass"] - d["mass0"] - d["pole_flux"]) / d["mass0"]
    print("shock_cap fp32", e, "mass", dg[0] / do[0] - 1, "energy", dg[4] / do[4] - 1, "pole flux", dg[5], do[5],
          "closure", closure)
    b = FP32_BOUND["shock_cap"]
    assert e["rho"] <= b["rho"] and e["drho"] <= b["drho"] and e["u"] <= b["u"], e
    assert abs(dg[0] / do[0] - 1) <= b["mass"] and abs(dg[4] / do[4] - 1) <= b["energy"], (dg, do)
    assert abs(dg[5] - do[5]) <= b["pole"] * do[0] and closure <= b["closure"], (dg, do, closure)
    s.close()
