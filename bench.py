#!/usr/bin/env python3
"""Throughput of the vLBM RK3 step on GB300 (arXiv 2504.15574 Sec. 3.7, Eq. Lf).

Workload: the 1024 x 2048 axisymmetric shock cap (rho = 4, T = 1.5 for
theta < 0.2; rho = 1, T = 1 elsewhere; u = 0), D2Q16, WENO-5 with active
nonlinear weights, tau = 1e-3, FP32 deviation storage with FP64 tables and an
FP64 non-finite guard per call, polar ring filter on with dt = 0.25 dtheta /
v_max.  A step is one SSP-RK3 step of all 16 populations on all 2,097,152
cells (MLUPS = million cell updates per second, Q = 16 populations).

One JSON line on rank 0.  ``--impl reference`` times the FP64 CPU oracle on
the host cores instead (a deliberately slow baseline).  Under torchrun every
rank runs an independent replica of the workload (the method shards only by
independent runs here), timing is max over ranks, value sums all ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & % HBM roofline per RK3 step; learned-coarse vs plain-fine time at equal error"
NT, NP = 1024, 2048
TAU = 1e-3
VMAX = math.sqrt(3 + math.sqrt(6))
DT = 0.25 * (math.pi / NT) / VMAX
# algorithmic HBM bytes per cell per RK3 step (FP32): stage 1 reads f, writes f1 (2 x 64 B);
# stages 2 and 3 read the stage input and f and write one array (3 x 64 B each)
BYTES_PER_CELL_STAGE = (128, 192, 192)
WORKLOAD = ("shock cap 1024x2048, D2Q16 (Q=16), FP32 deviation storage, WENO-5, polar filter, "
            "tau=1e-3, dt=0.25*dtheta/v_max")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    # profiling only (ncu captures of a smaller grid); the benchmark line uses the defaults
    ap.add_argument("--n-theta", type=int, default=1024)
    ap.add_argument("--n-phi", type=int, default=2048)
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle cpu_baseline leg")
    ap.add_argument("--repeats", type=int, default=0,
                    help="repeats of the timed steps (0: at least 5, until ~0.5 s of steps, at most 50)")
    ap.add_argument("--scheme", default="weno5", choices=["weno5", "u1", "u2", "u3"],
                    help="advection scheme (the headline workload is weno5)")
    ap.add_argument("--komissarov", action="store_true", help="Komissarov theta flux (upwind schemes)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"],
                    help="population storage (the headline workload is fp32)")
    ap.add_argument("--velocity-set", default="d2q16", choices=["d2q16", "d2q9"])
    args = ap.parse_args()
    global NT, NP, DT
    NT, NP = args.n_theta, args.n_phi
    DT = 0.25 * (math.pi / NT) / VMAX
    return args


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def repeat_times(time_one, repeats, world, device):
    """Times repeats of the timed region: time_one() runs one repeat (barriers inside) and returns
    its milliseconds.  At least 5 repeats and until ~0.5 s has run (at most 50), or exactly
    `repeats` when > 0; with world > 1 every rank takes rank 0's decision after each repeat, and
    the returned times are the max over ranks, repeat by repeat."""
    import torch
    times = []
    while True:
        times.append(float(time_one()))
        done = (len(times) >= repeats) if repeats > 0 else \
            (len(times) >= 5 and (sum(times) >= 500.0 or len(times) >= 50))
        if world > 1:
            flag = torch.tensor([1 if done else 0], device=device)
            torch.distributed.broadcast(flag, 0)
            done = bool(int(flag.item()))
        if done:
            break
    t = torch.tensor(times, dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def whole_job_mlups(cells, steps, world, ms):
    """Lattice updates of all ranks' replicas over the (max-over-ranks) time, in millions per second."""
    return cells * steps * world / (ms * 1e-3) / 1e6


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def committed_traffic(args):
    """DRAM bytes of the three stage launches of one step from the committed ncu summary of
    this scheme at 1024 x 2048 (null there once the kernel has changed since the capture,
    and null for another grid or a scheme without a summary)."""
    if (NT, NP) != (1024, 2048) or args.precision != "fp32":
        return None
    vs = "_d2q9" if args.velocity_set == "d2q9" else ""
    name = f"stage_f32{vs}_1024x2048.md" if args.scheme == "weno5" else \
        f"stage_f32{vs}_{args.scheme}{'k' if args.komissarov else ''}_1024x2048.md"
    path = os.path.join(ROOT, "profiles", name)
    try:
        for line in open(path):
            if line.startswith("traffic_bytes_per_step:"):
                v = line.split(":", 1)[1].strip()
                return None if v == "null" else float(v)
    except OSError:
        pass
    return None


def committed_lane_ops(args):
    """FP32 lane operations per cell and stage of the stage kernel, from the instruction classes of
    the committed ncu summary (the default workload's WENO-5 D2Q16 FP32 stage only; else None)."""
    if (NT, NP) != (1024, 2048) or args.precision != "fp32" or args.scheme != "weno5" or args.komissarov \
            or args.velocity_set != "d2q16":
        return None
    try:
        for line in open(os.path.join(ROOT, "profiles", "stage_f32_1024x2048.md")):
            if line.startswith("fp32_lane_ops_per_cell_stage:"):
                return float(line.split(":", 1)[1].strip())
    except OSError:
        pass
    return None


class Clocks:
    """Samples the SM clock, power and clock-event reasons of one GPU every 10 ms during the
    timed region, through NVML (read-only queries of the driver's library); falls back to
    nvidia-smi at its fastest loop if NVML cannot be loaded."""

    # NVML clock-event reason bits
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local):
        self.local = local
        self.rows = []          # (sm_mhz, max_mhz, reasons set)
        self.stop = threading.Event()
        self.proc = None
        self.thread = None
        self.source = None
        self.nvml = None
        self.handle = None

    def _nvml_handle(self):
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            return None, None
        h = ctypes.c_void_p()
        # the NVML device of this process's CUDA device: by PCI bus id, else by the visible-device list
        try:
            import torch
            p = torch.cuda.get_device_properties(self.local)
            bus = f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0".encode()
            if lib.nvmlDeviceGetHandleByPciBusId_v2(bus, ctypes.byref(h)) == 0:
                return lib, h
        except Exception:
            pass
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [x.strip() for x in vis.split(",") if x.strip()]
        if ids and self.local < len(ids):
            if ids[self.local].isdigit():
                if lib.nvmlDeviceGetHandleByIndex_v2(int(ids[self.local]), ctypes.byref(h)) == 0:
                    return lib, h
            elif lib.nvmlDeviceGetHandleByUUID(ids[self.local].encode(), ctypes.byref(h)) == 0:
                return lib, h
        if lib.nvmlDeviceGetHandleByIndex_v2(self.local, ctypes.byref(h)) == 0:
            return lib, h
        return None, None

    def _poll_nvml(self):
        import ctypes
        lib, h = self.nvml, self.handle
        get_reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self.stop.is_set():
            sm, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
            if lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(sm)) == 0 and \
                    lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:
                reasons = set()
                if get_reasons(h, ctypes.byref(rs)) == 0:
                    reasons = {n for b, n in self.REASONS.items() if rs.value & b}
                self.rows.append((float(sm.value), float(mx.value), reasons))
            self.stop.wait(0.01)

    def _read_smi(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.proc.stdout:
            r = [x.strip() for x in line.split(",")]
            if len(r) > 8 and r[1].replace(".", "").isdigit() and r[2].replace(".", "").isdigit():
                self.rows.append((float(r[1]), float(r[2]),
                                  {n for n, v in zip(names, r[5:9]) if v.lower() == "active"}))

    def __enter__(self):
        try:
            self.nvml, self.handle = self._nvml_handle()
        except OSError:
            self.nvml = None
        if self.nvml is not None:
            self.source = "nvml, 10 ms"
            self.thread = threading.Thread(target=self._poll_nvml, daemon=True)
            self.thread.start()
            return self
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.local), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.source = "nvidia-smi -lms 20"
            self.thread = threading.Thread(target=self._read_smi, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.stop.set()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)

    def summary(self):
        sm = [r[0] for r in self.rows]
        mx = [r[1] for r in self.rows]
        reasons = set()
        for r in self.rows:
            reasons |= r[2]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "sm_mhz_min": min(sm) if sm else None, "reasons": sorted(reasons), "samples": len(sm),
                "source": self.source}


def oracle_sample(steps, warmup, budget_s, scheme="weno5", komissarov=False, q=4):
    """The FP64 CPU oracle on the same workload (1024 x 2048 shock cap): `warmup` untimed full RK3
    steps (stopping early once they pass a quarter of `budget_s`), then up to `steps` timed full
    RK3 steps, stopping once `budget_s` seconds of timed work have run.  Returns (MLUPS, seconds,
    steps timed, threads, warm-up steps run)."""
    import oracle
    from paper_2504_15574_gb300 import inputs
    o = oracle.Oracle(NT, NP, tau=TAU, dt=DT, polar_filter=True, scheme=scheme, komissarov=komissarov, q=q)
    o.init_moments(*inputs.shock_cap(NT, NP))
    warm, t_w = 0, time.perf_counter()
    while warm < warmup and time.perf_counter() - t_w < budget_s / 4:
        o.step(1)
        warm += 1
    done, el = 0, 0.0
    while done < steps and el < budget_s:
        t0 = time.perf_counter()
        o.step(1)
        el += time.perf_counter() - t0
        done += 1
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return NT * NP * done / el / 1e6, el, done, cores, warm


def qcount(args):
    return 9 if getattr(args, "velocity_set", "d2q16") == "d2q9" else 16


def array_mb(args):
    """Bytes of one population array (with ghost rows and columns) in MB: FP32 stores pair
    planes of float2 (8 for D2Q16, 5 for D2Q9), FP64 one plane of doubles per population."""
    pitch = (NP + 8 + 3) // 4 * 4
    planes = (5 if args.velocity_set == "d2q9" else 8) if args.precision == "fp32" else qcount(args)
    return planes * (NT + 6) * pitch * 8 / 1e6


def workload_name(args):
    w = WORKLOAD.replace("1024x2048", f"{NT}x{NP}")
    if getattr(args, "velocity_set", "d2q16") == "d2q9":
        w = w.replace("D2Q16 (Q=16)", "D2Q9 (Q=9)")
    if getattr(args, "precision", "fp32") == "fp64":
        w = w.replace("FP32 deviation storage", "FP64 populations")
    if args.scheme != "weno5":
        w = w.replace("WENO-5", args.scheme.upper() + (" + Komissarov theta flux" if args.komissarov else ""))
    return w


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    val, el, done, cores, warm = oracle_sample(args.steps, args.warmup, 60.0, args.scheme, args.komissarov,
                                               3 if args.velocity_set == "d2q9" else 4)
    sample = (f"{done} of the {args.steps} requested full RK3 steps of the 1024x2048 workload "
              f"(timed work bounded at 60 s; {el:.1f} s) after {warm} of the {args.warmup} requested "
              f"warm-up steps")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": done, "warmup": warm, "ms_per_step": el / done * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args), "n_theta": NT, "n_phi": NP, "Q": qcount(args), "parallelism": "host cores"},
        "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_ours(args):
    import torch
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2504_15574_gb300 import inputs, vlbm
    vlbm.load()
    stream = torch.cuda.Stream()          # a real stream: the library captures CUDA graphs on it
    torch.cuda.set_stream(stream)
    rho, ut, up, T = inputs.shock_cap(NT, NP)
    s = vlbm.Solver(NT, NP, TAU, DT, precision=args.precision, polar_filter=True, stream=stream.cuda_stream,
                    scheme=args.scheme, komissarov=args.komissarov, velocity_set=args.velocity_set)
    s.init_moments(rho, ut, up, T)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    # warm-up (also builds and caches the CUDA graphs)
    s.step(max(args.warmup, 3))
    barrier()
    # The timed region, K steps through the public call (graph-launched, one FP64 guard per
    # call), is repeated: at least 5 times and until about half a second of steps has run (at
    # most 50 times); each repeat is bracketed by a barrier and a synchronize and timed with CUDA
    # events on the library's stream, the repeat's time is the max over ranks, and the line
    # reports the median repeat with the spread.  The clocks are sampled over all repeats.
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def time_one():
        barrier()
        ev0.record(stream)
        s.step(args.steps)
        ev1.record(stream)
        barrier()
        return ev0.elapsed_time(ev1)

    with Clocks(local) as clk:
        times = repeat_times(time_one, args.repeats, world, "cuda")
    ms = statistics.median(times)
    cells = NT * NP
    value = whole_job_mlups(cells, args.steps, world, ms)

    # per-kernel time, CUDA events on the launching stream (vlbm_profile_step): the three
    # stage kernels and the polar filter after each
    stage_ms, filter_ms, launches_per_step = s.profile_step(max(5, min(args.steps, 20)))
    # 64 B per cell per array for FP32 D2Q16; scaled by the population count and element size
    scale = (9 if args.velocity_set == "d2q9" else 16) / 16 * (2 if args.precision == "fp64" else 1)
    alg_bytes = cells * sum(BYTES_PER_CELL_STAGE) * scale
    achieved = alg_bytes / (sum(stage_ms) * 1e-3) / 1e9
    peak, peak_kind = measured_peak()
    traffic = committed_traffic(args)

    # end to end through the C ABI with host buffers in pinned memory: H2D of the moments, K
    # steps, D2H of the moments
    e2e_steps = args.steps

    def pinned(a=None):
        t = torch.empty((NT, NP), dtype=torch.float64).pin_memory()
        if a is not None:
            t.copy_(torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)))
        return t

    host_in = [pinned(a) for a in (rho, ut, up, T)]
    host_out = [pinned() for _ in range(3)]
    ins, outs = [t.numpy() for t in host_in], [t.numpy() for t in host_out]
    barrier()
    t0 = time.perf_counter()
    s.init_moments(*ins)
    s.step(e2e_steps)
    vlbm.vlbm_moments(s.h, *outs)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_val = whole_job_mlups(cells, e2e_steps, world, e2e_s * 1e3)
    h2d = 4 * cells * 8
    d2h = 3 * cells * 8

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu:
            val, el, done, cores, warm = oracle_sample(1000, 1, 15.0, args.scheme, args.komissarov,
                                                       3 if args.velocity_set == "d2q9" else 4)
            cpu = {"value": val, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                   "sample": f"{done} full RK3 steps of the 1024x2048 workload after {warm} warm-up step "
                             f"(bounded at 15 s of timed work; {el:.1f} s)"}
        clocks = clk.summary()
        # the stage kernel against its FMA pipe: FP32 lane operations (committed ncu instruction
        # classes) over the same event time, against 128 FP32 lanes per SM x SMs x the median SM
        # clock sampled during the timed region
        fma_roof = None
        lane_ops = committed_lane_ops(args)
        if lane_ops is not None and clocks.get("sm_mhz"):
            nsm = torch.cuda.get_device_properties(local).multi_processor_count
            ops = lane_ops * cells * 3 / (sum(stage_ms) * 1e-3) / 1e12
            pk = 128 * nsm * clocks["sm_mhz"] * 1e6 / 1e12
            fma_roof = {"bound": "alu", "pipe": "fma (FP32)", "achieved": ops, "peak": pk, "unit": "T lane-op/s",
                        "frac": ops / pk, "lane_ops_per_cell_stage": lane_ops,
                        "peak_from": f"128 FP32 lanes per SM x {nsm} SMs x {clocks['sm_mhz']:.0f} MHz (sampled)"}
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "repeats": {"count": len(times), "statistic": "median",
                        "ms_per_step": {"min": min(times) / args.steps, "median": ms / args.steps,
                                        "max": max(times) / args.steps},
                        "value_spread": [whole_job_mlups(cells, args.steps, world, max(times)),
                                         whole_job_mlups(cells, args.steps, world, min(times))]},
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
            "data": "synthetic",
            "config": {"workload": workload_name(args), "n_theta": NT, "n_phi": NP,
                       "Q": qcount(args), "global_batch": world,
                       "parallelism": f"replicas x{world}",
                       "l2": f"inputs larger than L2 (three {array_mb(args):.0f} MB population arrays per replica)"},
            "fma_roofline": fma_roof,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": ("stage_f32_kernel" if args.precision == "fp32" else "stage_f64 kernels")
                         + " (3 stages per step; bytes and traffic per step)",
                         "stage_ms": stage_ms, "filter_ms": filter_ms},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": "MLUPS", "h2d_bytes_per_step": h2d / e2e_steps,
                    "d2h_bytes_per_step": d2h / e2e_steps, "host_buffers": "pinned"},
            "gpu_launches": launches_per_step * args.steps + 1,
            "clocks": clocks,
        }), flush=True)
    s.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
