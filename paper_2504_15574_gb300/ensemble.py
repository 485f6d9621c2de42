"""Batched vortex-dynamics ensemble: throughput of vlbm_batch_* on mixed grids.

Workload: `runs_per_class` runs of each grid class 64x128, 128x256, 256x512 and
512x1024 (equal counts), each started from its own seeded Gaussian-vortex field
(inputs.gaussian_vortices, run index = seed), FP32, tau = 2e-3, per-grid dt =
min(rule, tau) with the rule of vlbm_max_stable_dt (0.25 dtheta / v_max with the
polar filter, the clamped pole-row rule without it).  All runs advance together:
one persistent stage kernel per RK3 stage over the batch's (run, tile) work list,
the step loop captured as CUDA graphs, the launch schedule chosen by the
autotuner.  Reported: cells, device time per step (CUDA events), MLUPS, the HBM
fraction of the 512 B per cell per step the stages move, the chosen schedule,
and, for comparison, the same runs advanced one standalone solver at a time.

Not the paper's experiment; the ensemble form of its solver.
"""
from __future__ import annotations

import argparse
import json
import os
import time

from . import inputs, vlbm

CLASSES = ((64, 128), (128, 256), (256, 512), (512, 1024))
TAU = 2e-3
BYTES_PER_CELL_STEP = 512


def measured_hbm_gbs():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    try:
        with open(os.path.join(root, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except Exception:
        return None


def build(runs_per_class, polar_filter):
    grids, dts = [], []
    for g in CLASSES:
        dt = vlbm.vlbm_max_stable_dt(g[0], g[1], TAU, polar_filter=polar_filter)
        for _ in range(runs_per_class):
            grids.append(g)
            dts.append(dt)
    b = vlbm.Batch(grids, TAU, dts, polar_filter=polar_filter, guard=False)
    for r, g in enumerate(grids):
        b.init_moments(r, *inputs.gaussian_vortices(g[0], g[1], run=r)[:3])
    return b, grids, dts


def sequential_ms_per_step(grids, dts, polar_filter, steps):
    """Device time per step of the same runs advanced one standalone solver at a time
    (one solver per grid class, timed on its own stream, times the run count)."""
    total = 0.0
    for g in CLASSES:
        count = sum(1 for x in grids if x == g)
        dt = dts[grids.index(g)]
        s = vlbm.Solver(g[0], g[1], TAU, dt, precision="fp32", polar_filter=polar_filter, guard=False)
        s.init_moments(*inputs.gaussian_vortices(g[0], g[1], run=0)[:3])
        s.step(3)
        s.sync()
        t0 = time.perf_counter()
        s.step(steps)
        s.sync()
        total += (time.perf_counter() - t0) / steps * 1e3 * count
        s.close()
    return total


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--runs-per-class", type=int, default=64)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--polar-filter", action="store_true")
    ap.add_argument("--tune-cache", default=None)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    vlbm.load()
    t0 = time.perf_counter()
    b, grids, dts = build(a.runs_per_class, a.polar_filter)
    t_init = time.perf_counter() - t0
    cells = b.cells()
    sched = b.tune(a.tune_cache)
    ms, launches = b.profile(a.steps)
    seq = sequential_ms_per_step(grids, dts, a.polar_filter, 50)
    peak = measured_hbm_gbs()
    achieved = cells * BYTES_PER_CELL_STEP / (ms * 1e-3) / 1e9
    out = {"workload": f"{len(grids)} runs ({a.runs_per_class} each of " +
                       ", ".join(f"{g[0]}x{g[1]}" for g in CLASSES) + "), Gaussian vortices, FP32, tau=2e-3",
           "polar_filter": a.polar_filter, "cells": cells, "steps": a.steps,
           "ms_per_step": ms, "mlups": cells / (ms * 1e-3) / 1e6, "launches_per_step": launches,
           "schedule": sched, "hbm_gbs_algorithmic": achieved,
           "hbm_frac_of_measured": (achieved / peak) if peak else None,
           "sequential_ms_per_step": seq, "batch_speedup_vs_sequential": seq / ms,
           "seconds_init": t_init}
    b.close()
    line = json.dumps(out)
    print(line)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(line + "\n")


if __name__ == "__main__":
    main()
