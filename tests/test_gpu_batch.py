"""Batched ensembles (vlbm_batch_*): every member of a batch of uneven grids
advances exactly as a standalone FP32 solver does (the batch only schedules the
same stage computation), for every launch schedule; the autotuner picks a
schedule, restores the state and caches its choice."""
import json
import os

import numpy as np
import pytest

from parity import clamped_dt, require_gpu
from paper_2504_15574_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    require_gpu()
    from paper_2504_15574_gb300 import build, vlbm
    build.build()
    vlbm.load()
    return vlbm


GRIDS = [(16, 32), (24, 48), (13, 10), (64, 128), (32, 64), (6, 2)]
TAU = 2e-3


def _batch(V, **kw):
    dts = [clamped_dt(nt, np_, TAU) for nt, np_ in GRIDS]
    b = V.Batch(GRIDS, TAU, dts, **kw)
    for r, (nt, np_) in enumerate(GRIDS):
        b.init_moments(r, *inputs.gaussian_vortices(nt, np_, run=100 + r))
    return b, dts


def _singles(V, dts, steps, **kw):
    out = []
    for r, (nt, np_) in enumerate(GRIDS):
        s = V.Solver(nt, np_, TAU, dts[r], precision="fp32", **kw)
        s.init_moments(*inputs.gaussian_vortices(nt, np_, run=100 + r))
        s.step(steps)
        out.append(s.moments())
        s.close()
    return out


@pytest.mark.parametrize("schedule", [(8, 0), (4, 0), (8, 1), (4, 2), (8, -1), (4, -1)])
def test_batch_members_equal_standalone_solvers_bitwise(V, schedule):
    b, dts = _batch(V)
    b.set_schedule(*schedule)
    b.step(20)
    ref = _singles(V, dts, 20)
    for r in range(len(GRIDS)):
        got = b.moments(r)
        for x, y in zip(got, ref[r]):
            assert np.array_equal(x, y), (r, schedule)
    b.close()


@pytest.mark.parametrize("schedule", [(8, 0), (4, 2), (8, -1)])
def test_batch_with_polar_filter_equals_standalone_solvers_bitwise(V, schedule):
    """One batched filter launch per stage over the filtered rows of every run gives each
    member the state of a standalone solver with its own filter launches (which, for the
    64 x 128 member, run beside its tile rows clear of the filtered rows)."""
    b, dts = _batch(V, polar_filter=True)
    b.set_schedule(*schedule)
    b.step(20)
    ref = _singles(V, dts, 20, polar_filter=True)
    for r in range(len(GRIDS)):
        for x, y in zip(b.moments(r), ref[r]):
            assert np.array_equal(x, y), (r, schedule)
    ms, launches = b.profile(2)
    assert launches == 6
    b.close()


def test_batch_with_upwind_scheme_equals_standalone_solvers_bitwise(V):
    """A batch runs the upwind-scheme stage (U3, Komissarov theta flux) for every member."""
    b, dts = _batch(V, scheme="u3", komissarov=True)
    b.set_schedule(8, 0)
    b.step(20)
    ref = _singles(V, dts, 20, scheme="u3", komissarov=True)
    for r in range(len(GRIDS)):
        for x, y in zip(b.moments(r), ref[r]):
            assert np.array_equal(x, y), r
    b.close()


def test_autotuner_restores_state_and_caches(V, tmp_path):
    cache = str(tmp_path / "tune.json")
    b, dts = _batch(V)
    choice = b.tune(cache)
    assert choice["tile_rows"] in (4, 8) and choice["ctas_per_sm"] in [-1] + list(range(1, 9)) and choice["ms_per_step"] > 0
    entries = json.load(open(cache))
    assert len(entries) == 1
    (key, val), = entries.items()
    assert val["tile_rows"] == choice["tile_rows"] and "x64x128" in key
    b.step(10)
    ref = _singles(V, dts, 10)
    for r in range(len(GRIDS)):
        assert np.array_equal(b.moments(r)[0], ref[r][0])
    # a second tune of the same grid mix comes from the cache
    b2, _ = _batch(V)
    again = b2.tune(cache)
    assert (again["tile_rows"], again["ctas_per_sm"]) == (choice["tile_rows"], choice["ctas_per_sm"])
    assert again["ms_per_step"] == pytest.approx(choice["ms_per_step"], rel=1e-4)
    b.close()
    b2.close()


def test_batch_rejects_fp64(V):
    import ctypes
    with pytest.raises(V.VlbmError) as e:
        o = V.vlbm_default_options()
        h = V._H()
        nt = (ctypes.c_int * 1)(16)
        np_ = (ctypes.c_int * 1)(32)
        t = np.array([1e-3])
        V._bcheck(V.load().vlbm_batch_create(1, nt, np_, V._p(t), V._p(t), ctypes.byref(o), ctypes.byref(h)))
    assert e.value.code == V.VLBM_ERR_UNSUPPORTED


@pytest.mark.parametrize("schedule,scheme,filt", [((8, 0), "weno5", False), ((8, -1), "weno5", True),
                                                  ((4, 2), "u3", True)])
def test_d2q9_batch_members_equal_standalone_solvers_bitwise(V, schedule, scheme, filt):
    """A batch of D2Q9 runs (App. A.1; five pair planes per member, the batched filter over
    them): every member advances as a standalone D2Q9 FP32 solver with the same tile rows, bit
    for bit.  (With 8-row tiles the D2Q9 tile walks its phi and theta faces on different warps
    into two tendency arrays that the cell adds; with 4-row tiles on the same warp into one:
    the last bit of a flux difference may differ between the two tile shapes.)"""
    vmax = 3.0 ** 0.5
    dts = [min(0.25 * min(np.pi / nt, np.sin(np.pi / nt / 2) * 2 * np.pi / np_) / vmax, TAU) for nt, np_ in GRIDS]
    kw = dict(polar_filter=filt, scheme=scheme, komissarov=scheme != "weno5")
    b = V.Batch(GRIDS, TAU, dts, velocity_set="d2q9", **kw)
    for r, (nt, np_) in enumerate(GRIDS):
        b.init_moments(r, *inputs.gaussian_vortices(nt, np_, run=200 + r))
    b.set_schedule(*schedule)
    b.step(20)
    for r, (nt, np_) in enumerate(GRIDS):
        s = V.Solver(nt, np_, TAU, dts[r], precision="fp32", velocity_set="d2q9", tile_rows=schedule[0], **kw)
        s.init_moments(*inputs.gaussian_vortices(nt, np_, run=200 + r))
        s.step(20)
        for x, y in zip(b.moments(r), s.moments()):
            assert np.array_equal(x, y), (r, schedule)
        assert np.array_equal(b.get_populations(r), s.get_populations())
        s.close()
    b.close()


def test_batch_refuses_weno_with_komissarov(V):
    with pytest.raises(V.VlbmError) as ex:
        V.Batch(GRIDS, TAU, 1e-4, komissarov=True)
    assert ex.value.code == V.VLBM_ERR_UNSUPPORTED
