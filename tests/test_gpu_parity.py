"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on
the same seeded inputs.

FP64 path: relative max error <= 1e-12 in rho and u (the bar the project sets
for FP64), and the populations themselves.  FP32 deviation path: the error
bound stated per case and derived in the design notes (FP32 rounding of
deviation-sized quantities, 2^-24 relative, accumulated over the steps run).
"""
import math

import numpy as np
import pytest

import oracle
from parity import clamped_dt, errors, literal_dt, require_gpu
from paper_2504_15574_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def V():
    require_gpu()
    from paper_2504_15574_gb300 import build, vlbm
    build.build()
    vlbm.load()
    return vlbm


def run_pair(V, nt, np_, tau, dt, ic, steps, precision="fp64", polar_filter=False, eps=1e-6, scheme="weno5",
             komissarov=False, velocity_set="d2q16", tile_rows=0):
    rho, ut, up, T = ic
    o = oracle.Oracle(nt, np_, tau=tau, dt=dt, eps=eps, polar_filter=polar_filter, scheme=scheme,
                      komissarov=komissarov, q=3 if velocity_set == "d2q9" else 4)
    o.init_moments(rho, ut, up, T)
    g = V.Solver(nt, np_, tau, dt, precision=precision, polar_filter=polar_filter, eps=eps, scheme=scheme,
                 komissarov=komissarov, velocity_set=velocity_set, tile_rows=tile_rows)
    g.init_moments(rho, ut, up, T)
    o.step(steps)
    g.step(steps)
    return o, g


CASES = {
    # name: (nt, np, tau, dt, ic-factory, steps, filter)
    "shear_p21_32x64_literal_dt": (32, 64, 0.02, literal_dt(32), lambda: inputs.shear_p21(32, 64), 500, False),
    "vortices_ragged_13x10": (13, 10, 0.05, clamped_dt(13, 10, 0.05), lambda: inputs.gaussian_vortices(13, 10, 3), 60,
                              False),
    "sound_1d_64x1": (64, 1, 2e-3, 1e-4, lambda: inputs.sound_parabola(64, 1, 1e-3), 200, False),
    "shock_cap_T_24x16": (24, 16, 1e-3, clamped_dt(24, 16, 1e-3), lambda: inputs.shock_cap(24, 16, cap=0.3), 80, False),
    "legendre3_32x64": (32, 64, 0.02, clamped_dt(32, 64, 0.02), lambda: inputs.sound_legendre(32, 64, 3), 100, False),
    "filter_vortices_16x32": (16, 32, 0.01, literal_dt(16) / 2, lambda: inputs.gaussian_vortices(16, 32, 5), 60, True),
    "minimum_6x2": (6, 2, 0.05, 1e-3, lambda: inputs.gaussian_vortices(6, 2, 8, umax=0.1), 40, False),
    "wide_row_8x4096": (8, 4096, 0.05, clamped_dt(8, 4096, 0.05), lambda: inputs.gaussian_vortices(8, 4096, 2), 3,
                        False),
    # polar filter blocks wider than a warp's 256 columns (b = 1024 on the first rows)
    "filter_wide_blocks_64x8192": (64, 8192, 0.01, literal_dt(64) / 2,
                                   lambda: inputs.gaussian_vortices(64, 8192, 6), 3, True),
    # polar filter blocks wider than one 2048-column window (b = 8192 on the pole rows)
    "filter_window_blocks_8x32768": (8, 32768, 0.01, 0.01, lambda: inputs.gaussian_vortices(8, 32768, 7), 3, True),
    # filtered rows 0-9 and 118-127: the FP32 stage runs its tile rows 2-13 on a second stream
    # beside the filter of the polar rows
    "filter_bands_128x256": (128, 256, 0.01, literal_dt(128) / 2, lambda: inputs.gaussian_vortices(128, 256, 7), 40,
                             True),
    # the sound wave about an axis in the equatorial plane (App. C, alpha = -pi/2): flow across the
    # pole rows and the phi seam
    "sound_rotated_32x32": (32, 32, 2e-3, 1e-4, lambda: inputs.sound_parabola_rotated(32, 32, 1e-3), 200, False),
    # the spherical shock tube of Sec. 4.3 (density ratio 8), through shock formation
    "riemann_256x1": (256, 1, 2e-4, 2e-5, lambda: inputs.riemann_cap(256, 1), 400, False),
    # the shock tube about an axis in the grid's equatorial plane (App. C, Fig. riemann_2D), to
    # t = 1: the shock crosses the rotated grid's pole rows; without and with the polar filter
    "riemann_rotated_32x32": (32, 32, 0.02, clamped_dt(32, 32, 0.02), lambda: inputs.riemann_cap_rotated(32, 32), 969,
                              False),
    "riemann_rotated_filter_32x32": (32, 32, 0.02, literal_dt(32), lambda: inputs.riemann_cap_rotated(32, 32), 95,
                                     True),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_matches_oracle(V, name):
    nt, np_, tau, dt, ic, steps, filt = CASES[name]
    o, g = run_pair(V, nt, np_, tau, dt, ic(), steps, polar_filter=filt)
    e = errors(g.moments(), o.moments())
    assert e["rho"] <= FP64_TOL and e["u"] <= FP64_TOL, e
    fo, fg = o.get_populations(), g.get_populations()
    assert np.abs(fg - fo).max() <= FP64_TOL * np.abs(fo).max()


def test_fp64_full_size_256x512(V):
    """The FP64 sound/shear configuration's grid, a few steps, every output compared."""
    nt, np_, tau = 256, 512, 0.02
    for ic in (inputs.sound_legendre(nt, np_, 2), inputs.shear_legendre(nt, np_, 3)):
        o, g = run_pair(V, nt, np_, tau, clamped_dt(nt, np_, tau), ic, 3)
        e = errors(g.moments(), o.moments())
        assert e["rho"] <= FP64_TOL and e["u"] <= FP64_TOL, e


def test_fp64_diagnostics_and_pole_budget(V):
    nt, np_ = 16, 24
    o, g = run_pair(V, nt, np_, 0.05, 5e-4, inputs.gaussian_vortices(nt, np_, 11, umax=0.1), 40)
    do, dg = o.diagnostics(), g.diagnostics()
    assert dg["mass"] == pytest.approx(do["mass"], rel=1e-13)
    assert dg["energy"] == pytest.approx(do["energy"], rel=1e-13)
    for c in ("px", "py", "pz"):
        assert dg[c] == pytest.approx(do[c], abs=1e-13 * do["mass"])
    assert dg["pole_flux"] == pytest.approx(do["pole_budget"], rel=1e-9)
    assert abs(dg["mass"] - dg["mass0"] - dg["pole_flux"]) < 1e-13 * dg["mass0"]
    assert dg["steps"] == 40 and dg["time"] == pytest.approx(40 * 5e-4)


def test_fp64_checkpoint_resume_is_bitwise(V):
    nt, np_ = 12, 16
    ic = inputs.gaussian_vortices(nt, np_, 21)
    a = V.Solver(nt, np_, 0.05, 5e-4)
    a.init_moments(*ic)
    a.step(10)
    f10 = a.get_populations()
    a.step(10)
    b = V.Solver(nt, np_, 0.05, 5e-4)
    b.set_populations(f10)
    b.step(10)
    assert np.array_equal(a.get_populations(), b.get_populations())


SCHEME_CASES = [
    # (scheme, komissarov, nt, np, filter)
    ("u1", False, 13, 10, False),
    ("u2", False, 16, 32, False),
    ("u3", False, 16, 32, False),
    ("u3", True, 16, 32, False),
    ("u2", True, 13, 10, False),
    ("weno5", True, 16, 32, False),
    ("u3", True, 16, 32, True),
]


@pytest.mark.parametrize("scheme,komissarov,nt,np_,filt", SCHEME_CASES)
def test_fp64_schemes_match_oracle(V, scheme, komissarov, nt, np_, filt):
    """Upwind fluxes U1-U3 and the Komissarov theta flux (Sec. 3.5) on the FP64 path,
    against the oracle's FP64 evaluation of the same scheme."""
    tau = 0.02
    dt = literal_dt(nt) / 2 if filt else clamped_dt(nt, np_, tau)
    ic = inputs.gaussian_vortices(nt, np_, 3, umax=0.08)
    o, g = run_pair(V, nt, np_, tau, dt, ic, 40, polar_filter=filt, scheme=scheme, komissarov=komissarov)
    e = errors(g.moments(), o.moments())
    assert e["rho"] <= FP64_TOL and e["u"] <= FP64_TOL, e
    if komissarov:
        # no flux crosses a pole
        assert g.diagnostics()["pole_flux"] == 0.0


D2Q9_CASES = [
    # (name, nt, np, filter, scheme, komissarov, ic-factory with T)
    ("vortices_16x32", 16, 32, False, "weno5", False, lambda nt, np_: inputs.gaussian_vortices(nt, np_, 5, umax=0.08)),
    ("shock_T_24x16", 24, 16, False, "weno5", False, lambda nt, np_: inputs.shock_cap(nt, np_, cap=0.3)),
    ("filter_u3_komissarov_16x32", 16, 32, True, "u3", True,
     lambda nt, np_: inputs.gaussian_vortices(nt, np_, 6, umax=0.08)),
    ("ragged_13x10_u2", 13, 10, False, "u2", False, lambda nt, np_: inputs.gaussian_vortices(nt, np_, 2)),
]


@pytest.mark.parametrize("case", D2Q9_CASES, ids=[c[0] for c in D2Q9_CASES])
def test_fp64_d2q9_matches_oracle(V, case):
    """The D2Q9 velocity set (App. A.1, Eqs. feq_Q=3, Q3_kernels) on the FP64 path."""
    name, nt, np_, filt, scheme, kom, ic = case
    tau, dth, vmax = 0.02, math.pi / nt, math.sqrt(3.0)
    dt = 0.125 * dth / vmax if filt else min(0.25 * min(dth, math.sin(dth / 2) * 2 * math.pi / np_) / vmax, tau)
    o, g = run_pair(V, nt, np_, tau, dt, ic(nt, np_), 40, polar_filter=filt, scheme=scheme, komissarov=kom,
                    velocity_set="d2q9")
    e = errors(g.moments(), o.moments())
    assert e["rho"] <= FP64_TOL and e["u"] <= FP64_TOL, e
    assert g.get_populations().shape == (9, nt, np_)
    d_g, d_o = g.diagnostics(), o.diagnostics()
    assert d_g["mass"] == pytest.approx(d_o["mass"], rel=1e-12)


# ---- FP32 deviation path ------------------------------------------------------------
# Stated bounds of the FP32 deviation path (derivation in the design notes):
# rounding of deviation-sized fluxes (2^-24 relative) amplified by 1/(R sin(theta) dtheta)
# near the poles and accumulated over the run gives ~1e-9 of rho and 1e-5..1e-4 of the
# flow speed over these horizons; each bound below lies above the worst value measured on GB300
# (by 1.3x for sound_1d_64x1's rho - mean, the tightest; by 3x or more for most).
FP32_CASES = {
    # name: (tol_rho, tol_drho, tol_u)
    "shear_p21_32x64_literal_dt": (1e-8, None, 1e-4),
    "vortices_ragged_13x10": (1e-7, 2e-4, 2e-5),
    "sound_1d_64x1": (1e-8, 2e-5, 2e-5),
    "shock_cap_T_24x16": (1e-5, 1e-5, 1e-4),
    "legendre3_32x64": (1e-8, 2e-5, 2e-4),
    "filter_vortices_16x32": (1e-7, 2e-4, 2e-5),
    "minimum_6x2": (1e-7, 2e-4, 2e-5),
    "wide_row_8x4096": (1e-7, 1e-3, 5e-7),
    "filter_wide_blocks_64x8192": (1e-7, 2e-4, 2e-5),
    "filter_window_blocks_8x32768": (1e-7, 2e-4, 2e-5),
    "filter_bands_128x256": (1e-7, 2e-4, 2e-5),
    "sound_rotated_32x32": (1e-8, 5e-5, 2e-5),
    "riemann_256x1": (2.5e-5, 3e-5, 2e-5),
    "riemann_rotated_32x32": (4e-6, 1e-5, 1e-5),
    "riemann_rotated_filter_32x32": (4e-6, 1e-5, 1e-5),
}


# stated bounds of the FP32 populations (max |df| / max |f| over all 16 populations and cells),
# about 3x the worst GB300 value
FP32_POP_TOL = {
    "shear_p21_32x64_literal_dt": 4e-8, "vortices_ragged_13x10": 4e-8, "sound_1d_64x1": 1e-8,
    "shock_cap_T_24x16": 5e-6, "legendre3_32x64": 2e-9, "filter_vortices_16x32": 4e-7, "minimum_6x2": 1e-8,
    "wide_row_8x4096": 4e-8, "filter_wide_blocks_64x8192": 4e-8, "filter_window_blocks_8x32768": 5e-8,
    "filter_bands_128x256": 1e-7, "sound_rotated_32x32": 2e-8, "riemann_256x1": 2e-5,
    "riemann_rotated_32x32": 4e-6, "riemann_rotated_filter_32x32": 4e-6,
}


@pytest.mark.parametrize("name", sorted(FP32_CASES))
def test_fp32_matches_oracle_within_stated_bound(V, name):
    nt, np_, tau, dt, ic, steps, filt = CASES[name]
    tol_rho, tol_drho, tol_u = FP32_CASES[name]
    o, g = run_pair(V, nt, np_, tau, dt, ic(), steps, precision="fp32", polar_filter=filt)
    e = errors(g.moments(), o.moments())
    # the 16 populations themselves, relative to the largest population
    fg, fo = g.get_populations(), o.get_populations()
    e_f = np.abs(fg - fo).max() / np.abs(fo).max()
    print(name, e, "populations", e_f)
    assert e["rho"] <= tol_rho, e
    if tol_drho is not None:
        assert e["drho"] <= tol_drho, e
    assert e["u"] <= tol_u, e
    assert e_f <= FP32_POP_TOL[name], e_f


# stated bounds of the FP32 upwind schemes (same origin as above; ~3x the worst GB300 value)
FP32_SCHEME_TOL = {"rho": 5e-8, "drho": 2e-5, "u": 1e-5}


@pytest.mark.parametrize("scheme,komissarov,nt,np_,filt", SCHEME_CASES)
def test_fp32_schemes_match_oracle_within_stated_bound(V, scheme, komissarov, nt, np_, filt):
    """The FP32 deviation path with the upwind fluxes (the reference state's part of their linear
    flux differences is exact in the FP64-derived tendency) and the Komissarov theta flux
    (reconstruction on df = dg / sin, interface sines), against the oracle."""
    tau = 0.02
    dt = literal_dt(nt) / 2 if filt else clamped_dt(nt, np_, tau)
    ic = inputs.gaussian_vortices(nt, np_, 3, umax=0.08)
    o, g = run_pair(V, nt, np_, tau, dt, ic, 40, precision="fp32", polar_filter=filt, scheme=scheme,
                    komissarov=komissarov)
    e = errors(g.moments(), o.moments())
    print(scheme, komissarov, e)
    assert e["rho"] <= FP32_SCHEME_TOL["rho"] and e["drho"] <= FP32_SCHEME_TOL["drho"], e
    assert e["u"] <= FP32_SCHEME_TOL["u"], e


# FP32 D2Q9: five pair planes (four pairs whose members share the sign of each nonzero velocity
# component, the rest population beside an always-zero slot), the same kernel as D2Q16.  Stated
# bounds of the same origin as above.
D2Q9_FP32_CASES = D2Q9_CASES + [
    # several 8 x 32 tiles in both directions with ragged last ones
    ("vortices_40x100", 40, 100, False, "weno5", False, lambda nt, np_: inputs.gaussian_vortices(nt, np_, 4, umax=0.08)),
    ("filter_sound_64x128", 64, 128, True, "weno5", False, lambda nt, np_: inputs.sound_legendre(nt, np_, 3)),
    # the smallest grid (every cell a pole-row cell beside a ghost column) and the axisymmetric one
    ("minimum_6x2", 6, 2, False, "weno5", False, lambda nt, np_: inputs.gaussian_vortices(nt, np_, 8, umax=0.1)),
    ("sound_1d_64x1", 64, 1, False, "weno5", False, lambda nt, np_: inputs.sound_parabola(nt, np_, 1e-3)),
    ("u1_vortices_24x48", 24, 48, False, "u1", False, lambda nt, np_: inputs.gaussian_vortices(nt, np_, 10, umax=0.08)),
    ("u3_filter_32x64", 32, 64, True, "u3", False, lambda nt, np_: inputs.gaussian_vortices(nt, np_, 11, umax=0.08)),
    # WENO-5 with the Komissarov theta flux
    ("w5k_vortices_16x32", 16, 32, False, "weno5", True, lambda nt, np_: inputs.gaussian_vortices(nt, np_, 12, umax=0.08)),
]
D2Q9_FP32_TOL = {
    # name: (tol_rho, tol_drho, tol_u), about 5x the worst GB300 value
    "vortices_16x32": (3e-8, 6e-6, 3e-6),
    "shock_T_24x16": (4e-7, 7e-7, 2e-6),
    "filter_u3_komissarov_16x32": (1e-7, 2e-5, 1e-5),
    "ragged_13x10_u2": (4e-8, 4e-6, 5e-6),
    # (its density deviation is ~3e-5 of rho: drho measures FP32 rounding on a tiny scale)
    "vortices_40x100": (5e-8, 2e-3, 3e-6),
    "filter_sound_64x128": (1e-9, 2e-6, 3e-6),
    "minimum_6x2": (1e-7, 1e-5, 8e-6),
    "sound_1d_64x1": (5e-9, 3e-6, 6e-6),
    "u1_vortices_24x48": (3e-8, 9e-6, 3e-6),
    "u3_filter_32x64": (4e-8, 1.1e-5, 5e-6),
    "w5k_vortices_16x32": (3e-8, 6e-6, 2e-6),
}


def d2q9_dt(nt, np_, tau, filt):
    dth, vmax = math.pi / nt, math.sqrt(3.0)
    return 0.125 * dth / vmax if filt else min(0.25 * min(dth, math.sin(dth / 2) * 2 * math.pi / np_) / vmax, tau)


@pytest.mark.parametrize("case", D2Q9_FP32_CASES, ids=[c[0] for c in D2Q9_FP32_CASES])
def test_fp32_d2q9_matches_oracle_within_stated_bound(V, case):
    """The D2Q9 velocity set (App. A.1, Eqs. feq_Q=3, Q3_kernels) on the FP32 deviation path."""
    name, nt, np_, filt, scheme, kom, ic = case
    tau = 0.02
    o, g = run_pair(V, nt, np_, tau, d2q9_dt(nt, np_, tau, filt), ic(nt, np_), 40, precision="fp32",
                    polar_filter=filt, scheme=scheme, komissarov=kom, velocity_set="d2q9")
    e = errors(g.moments(), o.moments())
    print(name, e)
    tol_rho, tol_drho, tol_u = D2Q9_FP32_TOL[name]
    assert e["rho"] <= tol_rho and e["drho"] <= tol_drho, e
    assert e["u"] <= tol_u, e
    f, fo = g.get_populations(), o.get_populations()
    assert f.shape == (9, nt, np_)
    np.testing.assert_allclose(f, fo, rtol=0, atol=1e-5 * np.abs(fo).max())
    # the populations in and out again through the five-pair layout: FP32 rounding of the deviations
    g.set_populations(fo)
    np.testing.assert_allclose(g.get_populations(), fo, rtol=0, atol=1e-7 * np.abs(fo).max())


def test_fp32_d2q9_full_size_1024x2048_one_step(V):
    """D2Q9 at the throughput grid size (shock cap at T = 1.5, WENO-5, polar filter): one step,
    every cell against the oracle."""
    nt, np_, tau = 1024, 2048, 1e-3
    dt = 0.25 * (math.pi / nt) / math.sqrt(3.0)
    o, g = run_pair(V, nt, np_, tau, dt, inputs.shock_cap(nt, np_), 1, precision="fp32", polar_filter=True,
                    velocity_set="d2q9")
    e = errors(g.moments(), o.moments())
    print(e)
    assert e["rho"] <= 1e-6 and e["drho"] <= 1e-6, e
    assert e["u"] <= 1e-5, e


@pytest.mark.parametrize("velocity_set,scheme", [("d2q16", "weno5"), ("d2q16", "u3"), ("d2q9", "weno5")])
def test_fp32_split_filter_schedule_equals_single_launch_schedule_bitwise(V, velocity_set, scheme):
    """With the polar filter, vlbm_step runs each stage as a polar-band launch (with the filter,
    on a second stream) and an interior-band launch; vlbm_profile_step runs the single-launch,
    single-stream schedule.  Same arithmetic per tile, so the states agree bit for bit."""
    nt, np_, tau = 128, 256, 0.01
    ic = inputs.gaussian_vortices(nt, np_, 9, umax=0.08)
    a = V.Solver(nt, np_, tau, literal_dt(nt) / 2, precision="fp32", polar_filter=True, scheme=scheme,
                 komissarov=scheme != "weno5", velocity_set=velocity_set)
    b = V.Solver(nt, np_, tau, literal_dt(nt) / 2, precision="fp32", polar_filter=True, scheme=scheme,
                 komissarov=scheme != "weno5", velocity_set=velocity_set)
    a.init_moments(*ic[:3])
    b.init_moments(*ic[:3])
    a.step(20)
    b.profile_step(20)
    assert np.array_equal(a.get_populations(), b.get_populations())
    a.close()
    b.close()


# 4-row stage tiles (128-thread CTAs; vlbm_options.tile_rows = 4): every case against the oracle
# with the bounds stated above, and for D2Q16 against the 8-row tiles, whose walkers form every
# face and flux difference with the same operations (a tile's first face takes the differences
# its predecessor carried): bit for bit for WENO-5 and the upwind schemes.  WENO-5 with the
# Komissarov flux agrees to the last bits only (GB300, 16 x 32: max|df| / max|f| 2.6e-11 after one
# step, 3.7e-9 after 40; deterministic at each tile height; the differing cells lie beside faces
# that are tile boundaries for 4-row tiles only): stated bound 1e-8.  D2Q9 8-row tiles add their
# phi and theta differences in two arrays, the 4-row ones in one, so D2Q9 is compared with the
# oracle only.
W5K_TILE_ROWS_TOL = 1e-8
FOUR_ROW_CASES = [
    # (name, nt, np, filter, scheme, komissarov, velocity set, (tol_rho, tol_drho, tol_u)); the
    # named cases are those of the tables above (same start, steps, dt and stated bounds)
    ("vortices_ragged_13x10", 13, 10, False, "weno5", False, "d2q16", FP32_CASES["vortices_ragged_13x10"]),
    ("shock_cap_T_24x16", 24, 16, False, "weno5", False, "d2q16", FP32_CASES["shock_cap_T_24x16"]),
    ("filter_bands_128x256", 128, 256, True, "weno5", False, "d2q16", FP32_CASES["filter_bands_128x256"]),
    ("minimum_6x2", 6, 2, False, "weno5", False, "d2q16", FP32_CASES["minimum_6x2"]),
    ("u3_komissarov_16x32", 16, 32, False, "u3", True, "d2q16", (FP32_SCHEME_TOL["rho"], FP32_SCHEME_TOL["drho"], FP32_SCHEME_TOL["u"])),
    ("u3_komissarov_filter_16x32", 16, 32, True, "u3", True, "d2q16",
     (FP32_SCHEME_TOL["rho"], FP32_SCHEME_TOL["drho"], FP32_SCHEME_TOL["u"])),
    ("weno5_komissarov_16x32", 16, 32, False, "weno5", True, "d2q16",
     (FP32_SCHEME_TOL["rho"], FP32_SCHEME_TOL["drho"], FP32_SCHEME_TOL["u"])),
    # several tiles both ways; its density deviation is ~1e-4 of rho, so drho would measure FP32
    # rounding on a tiny scale (as for the D2Q9 40 x 100 case): rho and u bounds only
    ("u3_komissarov_40x100", 40, 100, False, "u3", True, "d2q16", (FP32_SCHEME_TOL["rho"], None, FP32_SCHEME_TOL["u"])),
    ("vortices_40x100", 40, 100, False, "weno5", False, "d2q9", D2Q9_FP32_TOL["vortices_40x100"]),
    ("u3_filter_32x64", 32, 64, True, "u3", False, "d2q9", D2Q9_FP32_TOL["u3_filter_32x64"]),
]


@pytest.mark.parametrize("case", FOUR_ROW_CASES, ids=[c[0] for c in FOUR_ROW_CASES])
def test_fp32_four_row_tiles(V, case):
    name, nt, np_, filt, scheme, kom, vs, tol = case
    steps, tau = 40, 0.02
    if vs == "d2q9":
        dt = d2q9_dt(nt, np_, tau, filt)
        ic = dict((c[0], c[6]) for c in D2Q9_FP32_CASES)[name](nt, np_)
    elif name in CASES:
        _, _, tau, dt, icf, steps, filt = CASES[name]
        ic = icf()
    else:
        # the upwind-scheme cases' start and time step (test_fp32_schemes_match_oracle_within_stated_bound)
        dt = literal_dt(nt) / 2 if filt else clamped_dt(nt, np_, tau)
        ic = inputs.gaussian_vortices(nt, np_, 3, umax=0.08)
    kw = dict(precision="fp32", polar_filter=filt, scheme=scheme, komissarov=kom, velocity_set=vs)
    o, g = run_pair(V, nt, np_, tau, dt, ic, steps, tile_rows=4, **kw)
    e = errors(g.moments(), o.moments())
    print(name, e)
    tol_rho, tol_drho, tol_u = tol
    assert e["rho"] <= tol_rho and e["u"] <= tol_u, e
    if tol_drho is not None:
        assert e["drho"] <= tol_drho, e
    if vs == "d2q16":
        h = V.Solver(nt, np_, tau, dt, tile_rows=8, **kw)
        h.init_moments(*ic)
        h.step(steps)
        f4, f8 = g.get_populations(), h.get_populations()
        d4, d8 = g.diagnostics(), h.diagnostics()
        if scheme == "weno5" and kom:
            e_f = np.abs(f4 - f8).max() / np.abs(f8).max()
            print(name, "4- against 8-row tiles", e_f)
            assert e_f <= W5K_TILE_ROWS_TOL, e_f
            assert abs(d4["mass"] - d8["mass"]) <= 16 * W5K_TILE_ROWS_TOL * abs(d8["mass"]), (d4, d8)
        else:
            assert np.array_equal(f4, f8)
            assert d4["mass"] == d8["mass"], (d4, d8)
        assert d4["pole_flux"] == d8["pole_flux"], (d4, d8)
        h.close()
    g.close()


def test_fp32_weno_with_komissarov_full_size_1024x2048_one_step(V):
    """WENO-5 with the Komissarov theta flux (the paper's W5+K variant, Sec. 3.5) at the throughput
    grid size on the FP32 path, every cell against the oracle."""
    nt, np_, tau = 1024, 2048, 1e-3
    o, g = run_pair(V, nt, np_, tau, literal_dt(nt), inputs.shock_cap(nt, np_), 1, precision="fp32",
                    polar_filter=True, scheme="weno5", komissarov=True)
    e = errors(g.moments(), o.moments())
    print("w5k full size", e)
    assert e["rho"] <= 1e-6 and e["drho"] <= 1e-6, e
    assert e["u"] <= 1e-5, e
    assert g.diagnostics()["pole_flux"] == 0.0


def test_fp32_u3_komissarov_full_size_1024x2048_one_step(V):
    """U3 with the Komissarov flux at the throughput grid size, every cell against the oracle."""
    nt, np_, tau = 1024, 2048, 1e-3
    o, g = run_pair(V, nt, np_, tau, literal_dt(nt), inputs.shock_cap(nt, np_), 1, precision="fp32",
                    polar_filter=True, scheme="u3", komissarov=True)
    e = errors(g.moments(), o.moments())
    assert e["rho"] <= 1e-6 and e["drho"] <= 1e-6, e
    assert e["u"] <= 1e-5, e


def test_fp32_full_size_1024x2048_one_step(V):
    """The throughput configuration itself (1024 x 2048, shock cap at T = 1.5):
    one step on the GPU against one step of the oracle, every cell compared."""
    nt, np_, tau = 1024, 2048, 1e-3
    dt = literal_dt(nt)
    ic = inputs.shock_cap(nt, np_)
    o, g = run_pair(V, nt, np_, tau, dt, ic, 1, precision="fp32", polar_filter=True)
    e = errors(g.moments(), o.moments())
    assert e["rho"] <= 1e-6 and e["drho"] <= 1e-6, e
    assert e["u"] <= 1e-5, e


def test_fp32_axisymmetric_state_stays_bitwise_axisymmetric(V):
    nt, np_ = 1024, 2048
    g = V.Solver(nt, np_, 1e-3, literal_dt(nt), precision="fp32", polar_filter=True)
    g.init_moments(*inputs.shock_cap(nt, np_))
    g.step(20)
    r, ut, up = g.moments()
    assert np.array_equal(r, np.broadcast_to(r[:, :1], r.shape))
    assert np.array_equal(ut, np.broadcast_to(ut[:, :1], ut.shape))
    # u^phi stays at the rounding level of the populations mirrored in v_phi (the FP32
    # sums over k_phi and 3 - k_phi are not evaluated in mirrored order)
    assert np.abs(up).max() < 1e-6


def test_fp32_is_deterministic(V):
    nt, np_ = 40, 64
    ic = inputs.gaussian_vortices(nt, np_, 4)
    out = []
    for _ in range(2):
        g = V.Solver(nt, np_, 0.01, clamped_dt(nt, np_, 0.01), precision="fp32")
        g.init_moments(*ic)
        g.step(25)
        out.append(g.get_populations())
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_guard_reports_nonfinite(V, precision):
    nt, np_ = 8, 8
    g = V.Solver(nt, np_, 0.05, 1e-4, precision=precision)
    g.init_moments(*inputs.gaussian_vortices(nt, np_, 1))
    f = g.get_populations()
    f[3, 2, 5] = np.nan
    g.set_populations(f)
    with pytest.raises(V.VlbmError) as e:
        g.step(1)
    assert e.value.code == V.VLBM_ERR_NONFINITE


def test_rest_state_fp32_tendency_matches_oracle(V):
    """rho = 1, u = 0: the FP32 path's reference tendency (FP64 tables) reproduces
    the oracle's WENO truncation residual."""
    nt, np_ = 64, 128
    one = np.ones((nt, np_))
    o, g = run_pair(V, nt, np_, 0.02, 1e-4, (one, 0 * one, 0 * one, None), 10, precision="fp32")
    fo, fg = o.get_populations(), g.get_populations()
    v, w = oracle.quadrature()
    W = np.outer(w, w).reshape(16, 1, 1)
    assert np.abs((fg - W) - (fo - W)).max() <= 1e-9


@pytest.mark.parametrize("scheme", ["weno5", "u3"])
def test_fp32_tile_wait_that_runs_out_reports_a_timeout(V, scheme):
    """The stage kernels' bounded wait for a tile's copies: with a limit of 0 (give up when the
    copies have not landed at the first test), kernels give up (after recording the timeout and
    letting their copies land),
    vlbm_step returns VLBM_ERR_TIMEOUT, and a fresh handle then steps normally (the one-tile
    WENO-5 kernel and the persistent kernel of the upwind schemes)."""
    nt, np_ = 256, 512
    kw = dict(precision="fp32", polar_filter=True, scheme=scheme, komissarov=scheme != "weno5")
    ic = inputs.gaussian_vortices(nt, np_, 2)
    g = V.Solver(nt, np_, 0.01, literal_dt(nt) / 2, **kw)
    g.init_moments(*ic)
    V.vlbm_set_wait_limit(g.h, 0.0)
    with pytest.raises(V.VlbmError) as ex:
        g.step(4)
    assert ex.value.code == V.VLBM_ERR_TIMEOUT
    g.close()
    h = V.Solver(nt, np_, 0.01, literal_dt(nt) / 2, **kw)
    h.init_moments(*ic)
    h.step(4)
    r, ut, up = h.moments()
    assert np.isfinite(r).all() and abs(r.mean() - 1.0) < 1e-2
    h.close()
