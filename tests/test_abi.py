"""The C-ABI library loads on a machine without a GPU, exports every entry point
include/vlbm.h declares, and validates arguments before touching the device."""
import math
import os
import re
import subprocess

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "vlbm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2504_15574_gb300 import build, vlbm
    build.build()
    return vlbm.load()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"VLBM_API\s+[^;(]*?\b(vlbm_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("vlbm_create", "vlbm_init_moments", "vlbm_step", "vlbm_moments", "vlbm_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2504_15574_gb300 import vlbm
    out = subprocess.run(["nm", "-D", "--defined-only", vlbm.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(vlbm_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)
    # the Python binding covers every declared entry point
    assert set(declared_functions()) <= set(vlbm.SIGNATURES)


def test_max_stable_dt_needs_no_gpu(lib):
    from paper_2504_15574_gb300 import vlbm
    vmax = math.sqrt(3 + math.sqrt(6))
    dt = vlbm.vlbm_max_stable_dt(32, 64, 1.0)
    dth = math.pi / 32
    assert dt == pytest.approx(0.25 * min(dth, math.sin(dth / 2) * (2 * math.pi / 64)) / vmax, rel=1e-15)
    assert vlbm.vlbm_max_stable_dt(32, 64, 1.0, polar_filter=True) == pytest.approx(0.25 * dth / vmax, rel=1e-15)
    assert vlbm.vlbm_max_stable_dt(32, 64, 1e-9) == 1e-9      # capped at tau
    # D2Q9: the largest velocity is sqrt(3)
    assert vlbm.vlbm_max_stable_dt(32, 64, 1.0, polar_filter=True, velocity_set=vlbm.VLBM_D2Q9) == \
        pytest.approx(0.25 * dth / math.sqrt(3.0), rel=1e-15)
    with pytest.raises(vlbm.VlbmError) as e:
        vlbm.vlbm_max_stable_dt(32, 64, 1.0, velocity_set=5)
    assert e.value.code == vlbm.VLBM_ERR_ARG


@pytest.mark.parametrize("args,code", [
    ((5, 64, 4, 0.1, 1e-3), -1),      # n_theta < 6
    ((32, 63, 4, 0.1, 1e-3), -1),     # odd n_phi
    ((32, 64, 4, 0.0, 1e-3), -1),     # tau <= 0
    ((32, 64, 4, 0.1, -1.0), -1),     # dt <= 0
    ((32, 64, 7, 0.1, 1e-3), -1),     # unknown velocity set
])
def test_create_rejects_bad_arguments_before_the_gpu(lib, args, code):
    from paper_2504_15574_gb300 import vlbm
    with pytest.raises(vlbm.VlbmError) as e:
        vlbm.vlbm_create(*args)
    assert e.value.code == code
    assert vlbm.vlbm_last_error()


@pytest.mark.parametrize("tile_rows", [1, 5, 16, -4])
def test_create_rejects_a_tile_height_other_than_4_or_8(lib, tile_rows):
    from paper_2504_15574_gb300 import vlbm
    o = vlbm.vlbm_default_options()
    o.precision = vlbm.VLBM_FP32
    o.tile_rows = tile_rows
    with pytest.raises(vlbm.VlbmError) as e:
        vlbm.vlbm_create(32, 64, 4, 0.1, 1e-3, o)
    assert e.value.code == vlbm.VLBM_ERR_ARG
    assert "tile_rows" in vlbm.vlbm_last_error()


@pytest.mark.parametrize("velocity_set", ["d2q16", "d2q9"])
def test_batch_refuses_weno_with_komissarov_before_the_gpu(lib, velocity_set):
    # single runs take WENO-5 with the Komissarov theta flux on both paths; batches
    # offer that flux with the upwind schemes only
    from paper_2504_15574_gb300 import vlbm
    with pytest.raises(vlbm.VlbmError) as e:
        vlbm.Batch([(32, 64), (16, 32)], 0.1, 1e-3, scheme="weno5", komissarov=True,
                   velocity_set=velocity_set)
    assert e.value.code == vlbm.VLBM_ERR_UNSUPPORTED
    assert "upwind" in str(e.value)


def test_null_handles_are_argument_errors(lib):
    import ctypes
    assert lib.vlbm_step(None, 1) == -1
    assert lib.vlbm_moments(None, None, None, None, None) == -1
    assert lib.vlbm_lc_set_output_form(None, 1, 1.0) == -1
    lib.vlbm_destroy(None)   # NULL-safe
