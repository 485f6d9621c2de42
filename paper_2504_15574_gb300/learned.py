"""Learned-coarse vLBM: training data from fine runs, training, and evaluation.

A coarse FP32 solver (4x fewer cells per direction) advances one coarse step,
then the correction network (``vlbm_lc_*``, BF16 tensor-core kernels) nudges its
moments toward the block-averaged state of a fine run.  Pieces:

- ``downsample``: 4x4 sin(theta)-area-weighted block means of rho, of rho u as a
  Cartesian 3-vector (projected back on the coarse cell's vielbein frame, so the
  rotating frame near the poles is not averaged component-wise) and of T;
- ``make_samples``: fine runs (a ``Batch`` of FP32 solvers, Gaussian-vortex
  starts) advanced ``factor`` fine steps per coarse step; coarse rollouts beside
  them start from the block-averaged fine populations; after each coarse step the
  sample is (coarse moments, downsampled fine moments minus them);
- ``train``: Adam on those samples, with the correction in the "direct" form
  (drho, du^theta, du^phi) or the "stream" form (the centred curl of a predicted
  stream function: divergence-free, drho = 0);
- ``evaluate``: rollouts of plain coarse, coarse + correction and the fine run
  on held-out seeds; area-weighted relative L2 error of the vorticity (and of
  rho) against the downsampled fine run, and wall time per coarse step.

Not in the paper: a project extension whose arithmetic lives in the CUDA
library; this module only drives it and computes the judging metrics.
"""
from __future__ import annotations

import json
import math
import time

import numpy as np

from . import inputs, vlbm


def _frames(H, W):
    th, ph = inputs.cell_centres(H, W)
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    e_th = np.stack([np.cos(TH) * np.cos(PH), np.cos(TH) * np.sin(PH), -np.sin(TH)])
    e_ph = np.stack([-np.sin(PH), np.cos(PH), np.zeros_like(PH)])
    return np.sin(TH), e_th, e_ph


def downsample(rho, ut, up, T, factor=4):
    """Block means of a fine (rho, u^theta, u^phi, T) onto the coarse grid."""
    Hf, Wf = rho.shape
    H, W = Hf // factor, Wf // factor
    s, e_th, e_ph = _frames(Hf, Wf)
    w = s
    mom = rho[None] * (ut[None] * e_th + up[None] * e_ph)

    def block(a):
        return a.reshape(a.shape[:-2] + (H, factor, W, factor)).sum(axis=(-3, -1))

    wsum = block(w)
    rc = block(w * rho) / wsum
    mc = block(w[None] * mom) / wsum[None]
    Tc = block(w * T) / wsum
    _, ce_th, ce_ph = _frames(H, W)
    uc = mc / rc[None]
    return rc, (uc * ce_th).sum(0), (uc * ce_ph).sum(0), Tc


def downsample_populations(f, factor=4):
    """sin(theta)-area-weighted block means of every population [16][Hf][Wf] -> [16][H][W].
    Keeps the non-equilibrium part of the fine state (a coarse start from moments alone
    would begin with an equilibrium transient)."""
    _, Hf, Wf = f.shape
    H, W = Hf // factor, Wf // factor
    s = np.sin((np.arange(Hf) + 0.5) * math.pi / Hf)[:, None] * np.ones((1, Wf))
    ws = s.reshape(H, factor, W, factor).sum(axis=(1, 3))
    return (f * s[None]).reshape(16, H, factor, W, factor).sum(axis=(2, 4)) / ws[None]


def vorticity(ut, up):
    """Relative vorticity on the cell grid: [d_theta(sin u^phi) - d_phi u^theta] / sin, centred
    differences, pole ghost rows from the opposite meridian with vector components negated."""
    H, W = ut.shape
    dth, dph = math.pi / H, 2 * math.pi / W
    s = np.sin((np.arange(H) + 0.5) * dth)
    half = W // 2
    sup = s[:, None] * up
    north = np.roll(sup[0], -half)      # (-sin)(-u^phi) at the opposite meridian
    south = np.roll(sup[-1], -half)
    ext = np.vstack([north[None], sup, south[None]])
    d_th = (ext[2:] - ext[:-2]) / (2 * dth)
    d_ph = (np.roll(ut, -1, axis=1) - np.roll(ut, 1, axis=1)) / (2 * dph)
    return (d_th - d_ph) / s[:, None]


def rel_l2(a, ref):
    H, W = ref.shape
    w = np.sin((np.arange(H) + 0.5) * math.pi / H)[:, None]
    return float(np.sqrt((w * (a - ref) ** 2).sum() / (w * ref**2).sum()))


def clamped_dt(n_theta, n_phi, tau):
    """0.25 min(dtheta, sin(dtheta/2) dphi) / v_max, capped at tau (the stable step without the polar filter)."""
    dth = math.pi / n_theta
    lim = min(dth, math.sin(dth / 2) * 2 * math.pi / n_phi)
    return min(0.25 * lim / math.sqrt(3 + math.sqrt(6)), tau)


class Setup:
    """Grids, time steps and relaxation time of one learned-coarse experiment.

    With the polar filter, dt follows the theta spacing (0.25 dtheta / v_max, capped at
    tau) and a coarse step is `factor` fine steps.  Without it, dt follows the pole
    rows (clamped rule, ~ 1 / (n_theta n_phi)) and a coarse step is `substeps` fine
    steps (factor^2 for equal aspect ratios).  tile_rows: the stage tile height of the
    coarse and plain solvers (4 or 8; 0: the library's default)."""

    def __init__(self, coarse=(128, 256), factor=4, tau=2e-3, polar_filter=True, tile_rows=0):
        self.coarse = tuple(coarse)
        self.tile_rows = int(tile_rows)
        self.factor = int(factor)
        self.fine = (self.coarse[0] * factor, self.coarse[1] * factor)
        self.tau = float(tau)
        self.polar_filter = bool(polar_filter)
        vmax = math.sqrt(3 + math.sqrt(6))
        if self.polar_filter:
            self.dt_c = min(0.25 * (math.pi / self.coarse[0]) / vmax, self.tau)
            self.substeps = self.factor
        else:
            self.dt_c = clamped_dt(*self.coarse, self.tau)
            self.substeps = math.ceil(self.dt_c / clamped_dt(*self.fine, self.tau) - 1e-9)
        self.dt_f = self.dt_c / self.substeps

    def coarse_solver(self):
        return vlbm.Solver(*self.coarse, self.tau, self.dt_c, precision="fp32", polar_filter=self.polar_filter,
                           guard=False, tile_rows=self.tile_rows)

    def fine_batch(self, seeds):
        b = vlbm.Batch([self.fine] * len(seeds), self.tau, self.dt_f, polar_filter=self.polar_filter, guard=False)
        for r, sd in enumerate(seeds):
            b.init_moments(r, *inputs.gaussian_vortices(*self.fine, run=sd)[:3])
        return b


def make_samples(setup: Setup, seeds, n_steps, spinup=0, net=None, reinit_every=1, stride=1):
    """(inputs [N,4,H,W], targets [N,3,H,W]) from coarse rollouts beside fine runs.

    One coarse solver per seed starts from the block-averaged fine populations and
    is re-started from them every `reinit_every` coarse steps (default: every step,
    so each target is the one-step gap of a coarse step taken from the fine state,
    the correction a per-step nudge has to supply); after each coarse step the
    sample is (coarse moments, downsampled fine moments minus them).  With
    reinit_every = 1, the fine runs advance `stride` coarse steps between samples.
    With a network and reinit_every > 1, its correction is applied after each
    sample (so later rounds see the states the corrected rollout visits)."""
    fb = setup.fine_batch(seeds)
    if spinup:
        fb.step(spinup * setup.substeps)
    cs = [setup.coarse_solver() for _ in seeds]
    X, Y = [], []
    for k in range(n_steps):
        if k % reinit_every == 0:
            if reinit_every == 1 and k and stride > 1:
                fb.step((stride - 1) * setup.substeps)
            for r in range(len(seeds)):
                cs[r].set_populations(downsample_populations(fb.get_populations(r), setup.factor))
        fb.step(setup.substeps)
        for r in range(len(seeds)):
            cs[r].step(1)
            c = cs[r].moments(with_T=True)
            d = downsample(*fb.moments(r, with_T=True))
            X.append(np.stack(c))
            Y.append(np.stack([d[0] - c[0], d[1] - c[1], d[2] - c[2]]))
            if net is not None:
                net.apply(cs[r])
    for c in cs:
        c.close()
    fb.close()
    return np.array(X), np.array(Y)


def make_drift_samples(setup: Setup, seeds, windows, settle=64, span=32, spans=4, spinup=0):
    """(inputs [N,4,H,W], targets [N,3,H,W]): per-step drift of the coarse run away from the fine run.

    Each window restarts the coarse solvers from the block-averaged fine populations,
    lets the restart transient settle for `settle` coarse steps, then records `spans`
    samples: after each further `span` steps, the coarse moments and the growth of the
    gap (downsampled fine minus coarse) over that span divided by `span`.  The restart
    offset cancels in the difference, so the target is the error the coarse scheme
    adds per step, which a per-step correction has to remove."""
    fb = setup.fine_batch(seeds)
    if spinup:
        fb.step(spinup * setup.substeps)
    cs = [setup.coarse_solver() for _ in seeds]

    def gaps():
        out = []
        for r in range(len(seeds)):
            c = cs[r].moments(with_T=True)
            d = downsample(*fb.moments(r, with_T=True))
            out.append((np.stack(c), np.stack([d[0] - c[0], d[1] - c[1], d[2] - c[2]])))
        return out

    X, Y = [], []
    for _ in range(windows):
        for r in range(len(seeds)):
            cs[r].set_populations(downsample_populations(fb.get_populations(r), setup.factor))
        fb.step(settle * setup.substeps)
        for c in cs:
            c.step(settle)
        prev = gaps()
        for _ in range(spans):
            fb.step(span * setup.substeps)
            for c in cs:
                c.step(span)
            cur = gaps()
            for (x, g1), (_, g0) in zip(cur, prev):
                X.append(x)
                Y.append((g1 - g0) / span)
            prev = cur
    for c in cs:
        c.close()
    fb.close()
    return np.array(X), np.array(Y)


def _extend_theta(a, odd, halo=3):
    """[..., H, W] -> [..., H + 2 halo, W]: rows beyond a pole from the opposite meridian."""
    W = a.shape[-1]
    sgn = -1.0 if odd else 1.0
    north = sgn * np.roll(a[..., :halo, :][..., ::-1, :], -(W // 2), axis=-1)
    south = sgn * np.roll(a[..., -halo:, :][..., ::-1, :], -(W // 2), axis=-1)
    return np.concatenate([north, a, south], axis=-2)


def _differences(X):
    """The ten difference channels the network's feature kernel forms (for their scales)."""
    D4, D6 = [1.0, -4.0, 6.0, -4.0, 1.0], [1.0, -6.0, 15.0, -20.0, 15.0, -6.0, 1.0]

    def diff(a, odd, st, axis):
        h = len(st) // 2
        if axis == 1:
            return sum(w * np.roll(a, h - m, axis=-1) for m, w in enumerate(st))
        e = _extend_theta(a, odd)
        H = a.shape[-2]
        return sum(w * e[..., 3 + m - h:3 + m - h + H, :] for m, w in enumerate(st))

    rho, ut, up = X[:, 0], X[:, 1], X[:, 2]
    return [diff(rho, False, D6, 0), diff(rho, False, D6, 1), diff(ut, True, D6, 0), diff(ut, True, D6, 1),
            diff(up, True, D6, 0), diff(up, True, D6, 1), diff(ut, True, D4, 0), diff(ut, True, D4, 1),
            diff(up, True, D4, 0), diff(up, True, D4, 1)]


def scales(X, Y):
    """Per-channel input and output scales from the sample spread: the largest |value| of
    rho-1, u^theta, u^phi, T-1 (T floored at 1e-3), the std of each difference channel, and
    the std of each target channel."""
    ins = [max(np.abs(X[:, 0] - 1).max(), 1e-12), max(np.abs(X[:, 1]).max(), 1e-12),
           max(np.abs(X[:, 2]).max(), 1e-12), max(np.abs(X[:, 3] - 1).max(), 1e-3)]
    ins += [max(float(d.std()), 1e-30) for d in _differences(X)]
    outs = [max(Y[:, c].std(), 1e-16) for c in range(3)]
    return ins, outs


def stream_scale(setup: Setup, outs):
    """Output scale of the stream function: the velocity targets' spread times R times 8
    coarse theta spacings (a correction varying over ~8 cells has that stream-function size)."""
    return 0.5 * (outs[1] + outs[2]) * 8.0 * math.pi / setup.coarse[0]


def vorticity_scale(setup: Setup, outs):
    """Output scale of the vorticity correction: the velocity targets' spread over R times 4
    coarse theta spacings (a velocity correction varying over ~4 cells has that vorticity)."""
    return 0.5 * (outs[1] + outs[2]) / (4.0 * math.pi / setup.coarse[0])


def train(setup: Setup, X, Y, epochs=4, lr=2e-3, seed=1, log=None, net=None, form="direct"):
    if net is None:
        ins, outs = scales(X, Y)
        if form == "stream":
            outs = [stream_scale(setup, outs), outs[1], outs[2]]
        elif form == "vorticity":
            outs = [vorticity_scale(setup, outs), outs[1], outs[2]]
        net = vlbm.LearnedCorrection(*setup.coarse, seed=seed, in_scale=ins, out_scale=outs, form=form)
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        order = rng.permutation(len(X))
        lr_ep = lr * (0.5 ** ep)
        tot = 0.0
        for i in order:
            tot += net.train_step(X[i], Y[i], lr_ep)
        hist.append(tot / len(X))
        if log:
            log(f"epoch {ep}: mean loss {hist[-1]:.4e}")
    return net, hist


def evaluate(setup: Setup, net, seeds, n_steps, spinup=20, start="fine"):
    """Rollouts of n_steps coarse steps after a spin-up of `spinup` coarse steps: errors against
    the downsampled fine run and wall times.  start = "fine": the coarse runs start from the
    downsampled fine state after the spin-up (the fine run does the spin-up); "analytic": every run
    starts from the analytic start on its own grid at t = 0 and runs spin-up + n_steps (the
    protocol of plain_runs_at)."""
    fb = setup.fine_batch(seeds)
    fb.step(spinup * setup.substeps)
    if start == "fine":
        starts = [downsample_populations(fb.get_populations(r), setup.factor) for r in range(len(seeds))]
    t0 = time.perf_counter()
    fb.step(n_steps * setup.substeps)
    t_fine = (time.perf_counter() - t0) / (n_steps * len(seeds))
    refs = [downsample(*fb.moments(r, with_T=True)) for r in range(len(seeds))]
    fb.close()
    # learned_u (direct form only): the same network with its density output dropped
    modes = ("plain", "learned", "learned_u") if net.form == "direct" else ("plain", "learned")
    res = {m: [] for m in modes}
    times = {}
    for mode in modes:
        cs = setup.coarse_solver()
        el = 0.0
        if mode == "learned_u":
            # the velocity-only correction: the same network with its density output dropped
            out_scale = net.out_scale.copy()
            net.set_scales(net.in_scale, (0.0, out_scale[1], out_scale[2]))
        for r in range(len(seeds)):
            if start == "fine":
                cs.set_populations(starts[r])
            else:
                cs.init_moments(*inputs.gaussian_vortices(*setup.coarse, run=seeds[r])[:3])
                if mode != "plain":
                    net.rollout(cs, spinup)
                else:
                    cs.step(spinup)
            t0 = time.perf_counter()
            if mode != "plain":
                net.rollout(cs, n_steps)
            else:
                cs.step(n_steps)
            el += time.perf_counter() - t0
            rho, ut, up = cs.moments()
            ref = refs[r]
            res[mode].append({"vort": rel_l2(vorticity(ut, up), vorticity(ref[1], ref[2])),
                              "rho": rel_l2(rho - 1.0, ref[0] - 1.0)})
        times[mode] = el / (n_steps * len(seeds))
        cs.close()
        if mode == "learned_u":
            net.set_scales(net.in_scale, out_scale)
    # a coarse step stands for `substeps` fine steps; the batch advanced all seeds together
    out = {"seeds": list(seeds), "coarse_steps": n_steps, "t_end": n_steps * setup.dt_c, "start": start,
           "grid_coarse": list(setup.coarse), "grid_fine": list(setup.fine),
           "vort_err_plain_per_seed": [e["vort"] for e in res["plain"]],
           "vort_err_learned_per_seed": [e["vort"] for e in res["learned"]],
           "vort_err_plain": float(np.mean([e["vort"] for e in res["plain"]])),
           "vort_err_learned": float(np.mean([e["vort"] for e in res["learned"]])),
           "rho_err_plain": float(np.mean([e["rho"] for e in res["plain"]])),
           "rho_err_learned": float(np.mean([e["rho"] for e in res["learned"]])),
           "rho_err_plain_per_seed": [e["rho"] for e in res["plain"]],
           "rho_err_learned_per_seed": [e["rho"] for e in res["learned"]],
           "form": net.form,
           "ms_per_coarse_step_plain": times["plain"] * 1e3, "ms_per_coarse_step_learned": times["learned"] * 1e3,
           "ms_fine_per_coarse_step": t_fine * 1e3}
    if "learned_u" in res:
        out.update({"vort_err_learned_u_per_seed": [e["vort"] for e in res["learned_u"]],
                    "rho_err_learned_u_per_seed": [e["rho"] for e in res["learned_u"]],
                    "vort_err_learned_u": float(np.mean([e["vort"] for e in res["learned_u"]])),
                    "rho_err_learned_u": float(np.mean([e["rho"] for e in res["learned_u"]]))})
    out["speedup_learned_vs_fine"] = out["ms_fine_per_coarse_step"] / out["ms_per_coarse_step_learned"]
    return out


def plain_runs_at(setup: Setup, seeds, n_steps, grids, spinup=20, start="analytic"):
    """Plain FP32 runs at intermediate grids (integer multiples m of the coarse grid, m < factor)
    to the time the learned rollouts of `evaluate` reach (spin-up + n_steps coarse steps, each grid
    at its own clamped dt dividing the coarse one); their m x m block means on the coarse grid
    against the fine run's.  start = "analytic": each grid from the analytic start on itself at
    t = 0; "fine": from the fine state after the spin-up, block-averaged onto the grid (only for m
    dividing the fine factor; other grids are skipped), as `evaluate` starts the coarse runs.
    Returns per grid the mean vorticity and rho - 1 errors and the wall time per coarse-step span."""
    fb = setup.fine_batch(seeds)
    fb.step(spinup * setup.substeps)
    fstart = [fb.get_populations(r) for r in range(len(seeds))] if start == "fine" else None
    fb.step(n_steps * setup.substeps)
    refs = [downsample(*fb.moments(r, with_T=True)) for r in range(len(seeds))]
    fb.close()
    out = []
    for m in grids:
        if start == "fine" and setup.factor % m:
            continue
        g = (setup.coarse[0] * m, setup.coarse[1] * m)
        sub = setup.substeps if m == setup.factor else \
            math.ceil(setup.dt_c / clamped_dt(*g, setup.tau) - 1e-9)
        dt = setup.dt_c / sub
        ev, er, el = [], [], 0.0
        for k, sd in enumerate(seeds):
            s = vlbm.Solver(*g, setup.tau, dt, precision="fp32", polar_filter=setup.polar_filter, guard=False,
                            tile_rows=setup.tile_rows)
            if start == "fine":
                s.set_populations(downsample_populations(fstart[k], setup.factor // m))
            else:
                s.init_moments(*inputs.gaussian_vortices(*g, run=sd)[:3])
                s.step(spinup * sub)
            t0 = time.perf_counter()
            s.step(n_steps * sub)
            el += time.perf_counter() - t0
            rho, ut, up, T = s.moments(with_T=True)
            s.close()
            d = downsample(rho, ut, up, T, factor=m) if m > 1 else (rho, ut, up, T)
            ref = refs[seeds.index(sd)]
            ev.append(rel_l2(vorticity(d[1], d[2]), vorticity(ref[1], ref[2])))
            er.append(rel_l2(d[0] - 1.0, ref[0] - 1.0))
        out.append({"grid": list(g), "steps_per_coarse_step": sub, "vort_err": float(np.mean(ev)),
                    "rho_err": float(np.mean(er)), "vort_err_per_seed": ev,
                    "ms_per_coarse_step": el / (n_steps * len(seeds)) * 1e3})
    return out


def equal_error_grid(points, target):
    """The resolution multiple m* at which the plain error equals `target`, and the plain time per
    coarse-step span there, interpolated log-log between the two grids that bracket it; None if no
    pair brackets it.  points: [(m, error, ms)] in increasing m."""
    for (m0, e0, t0), (m1, e1, t1) in zip(points, points[1:]):
        if (e0 - target) * (e1 - target) <= 0 and e0 > 0 and e1 > 0 and e0 != e1:
            a = (math.log(target) - math.log(e0)) / (math.log(e1) - math.log(e0))
            m = math.exp(math.log(m0) + a * (math.log(m1) - math.log(m0)))
            ms = math.exp(math.log(t0) + a * (math.log(t1) - math.log(t0)))
            return m, ms
    return None


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--coarse", type=int, nargs=2, default=[128, 256])
    ap.add_argument("--polar-filter", action="store_true", help="filter on (dt by the theta spacing)")
    ap.add_argument("--tile-rows", type=int, choices=[0, 4, 8], default=0,
                    help="stage tile height of the coarse and plain solvers (0: the library's default, 8)")
    ap.add_argument("--targets", choices=["drift", "one-step"], default="drift")
    ap.add_argument("--train-seeds", type=int, default=32)
    ap.add_argument("--windows", type=int, default=16, help="drift targets: restart windows per seed")
    ap.add_argument("--steps", type=int, default=48, help="one-step targets: samples per seed")
    ap.add_argument("--spinup", type=int, default=20)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--eval-seeds", type=int, default=4)
    ap.add_argument("--eval-steps", type=int, nargs="+", default=[300, 1000])
    ap.add_argument("--out", default=None)
    ap.add_argument("--start", choices=["fine", "analytic"], default="fine",
                    help="rollout starts: the downsampled fine state after the spin-up, or every grid's own analytic start")
    ap.add_argument("--save-net", default=None, help="write the trained weights and scales (.npz)")
    ap.add_argument("--load-net", default=None, help="read weights and scales (.npz) instead of making data and training")
    ap.add_argument("--equal-error", type=int, nargs="*", default=[],
                    help="resolution multiples of the coarse grid for plain runs at each horizon (e.g. 2 3)")
    ap.add_argument("--save-data", default=None, help="write the training samples (.npz)")
    ap.add_argument("--load-data", default=None, help="read the training samples (.npz) instead of making them")
    ap.add_argument("--form", choices=["direct", "stream", "vorticity"], default="direct",
                    help="correction form: (drho, du) outputs, the curl of a predicted stream function, or of the "
                         "Poisson solution for a predicted vorticity")
    ap.add_argument("--timing-steps", type=int, default=0,
                    help="only time this many corrected coarse steps of an untrained network (no data, no training)")
    a = ap.parse_args(argv)
    setup = Setup(coarse=a.coarse, polar_filter=a.polar_filter, tile_rows=a.tile_rows)
    if a.timing_steps:
        net = vlbm.LearnedCorrection(*setup.coarse, seed=1, form=a.form)
        cs = setup.coarse_solver()
        cs.init_moments(*inputs.gaussian_vortices(*setup.coarse, run=5000)[:3])
        net.rollout(cs, 3)
        t0 = time.perf_counter()
        net.rollout(cs, a.timing_steps)
        ms = (time.perf_counter() - t0) / a.timing_steps * 1e3
        t0 = time.perf_counter()
        cs.step(a.timing_steps)
        ms_plain = (time.perf_counter() - t0) / a.timing_steps * 1e3
        print(json.dumps({"grid_coarse": list(setup.coarse), "steps": a.timing_steps,
                          "ms_per_corrected_step": ms, "ms_per_plain_step": ms_plain}))
        cs.close()
        net.close()
        return
    seeds = list(range(1000, 1000 + a.train_seeds))
    if a.load_net:
        z = np.load(a.load_net)
        form = str(z["form"]) if "form" in z else "direct"
        net = vlbm.LearnedCorrection(*setup.coarse, seed=1, in_scale=z["in_scale"], out_scale=z["out_scale"],
                                     form=form)
        net.set_weights(z["weights"])
        X, hist, t_data, t_train = [], [], 0.0, 0.0
    else:
        t0 = time.perf_counter()
        if a.load_data:
            z = np.load(a.load_data)
            X, Y = z["X"], z["Y"]
        elif a.targets == "drift":
            X, Y = make_drift_samples(setup, seeds, a.windows, spinup=a.spinup)
        else:
            X, Y = make_samples(setup, seeds, a.steps, spinup=a.spinup)
        t_data = time.perf_counter() - t0
        if a.save_data:
            np.savez(a.save_data, X=X, Y=Y)
        t0 = time.perf_counter()
        net, hist = train(setup, X, Y, epochs=a.epochs, log=print, form=a.form)
        t_train = time.perf_counter() - t0
    if a.save_net:
        np.savez(a.save_net, weights=net.get_weights(), in_scale=net.in_scale, out_scale=net.out_scale,
                 form=net.form)
    out = {"form": net.form, "grid_coarse": list(setup.coarse), "grid_fine": list(setup.fine),
           "polar_filter": setup.polar_filter,
           "dt_coarse": setup.dt_c, "fine_steps_per_coarse_step": setup.substeps, "targets": a.targets,
           "samples": int(len(X)), "loss_history": hist, "seconds_data": t_data, "seconds_train": t_train,
           "horizons": []}
    for n in a.eval_steps:
        eseeds = list(range(5000, 5000 + a.eval_seeds))
        res = evaluate(setup, net, eseeds, n, spinup=a.spinup, start=a.start)
        if a.equal_error:
            pr = plain_runs_at(setup, eseeds, n, sorted(a.equal_error), spinup=a.spinup, start=a.start)
            res["plain_grids"] = pr
            pts = [(1, res["vort_err_plain"], res["ms_per_coarse_step_plain"])] + \
                  [(p["grid"][0] // setup.coarse[0], p["vort_err"], p["ms_per_coarse_step"]) for p in pr] + \
                  [(setup.factor, 1e-300, res["ms_fine_per_coarse_step"])]
            res["equal_error"] = {}
            for key in ("learned", "learned_u"):
                if f"vort_err_{key}" not in res:
                    continue
                hit = equal_error_grid(pts[:-1], res[f"vort_err_{key}"])
                res["equal_error"][key] = None if hit is None else {
                    "multiple": hit[0], "ms_plain": hit[1],
                    "time_ratio_plain_over_learned": hit[1] / res[f"ms_per_coarse_step_{'learned'}"]}
        out["horizons"].append(res)
        keys = ("coarse_steps", "vort_err_plain", "vort_err_learned", "vort_err_learned_u", "rho_err_plain",
                "rho_err_learned", "rho_err_learned_u", "speedup_learned_vs_fine", "plain_grids", "equal_error")
        print(json.dumps({k: res[k] for k in keys if k in res}))
    line = json.dumps(out)
    print(line)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(line + "\n")


if __name__ == "__main__":
    main()
