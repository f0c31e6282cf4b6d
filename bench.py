#!/usr/bin/env python3
"""Benchmark: IC-PBA iterations/s and residuals/s against FC on one GB300.

Workload (default): the 100-frame orbit bundle of the precision configuration
-- a reference frame and 100 target frames on a 30 deg orbit around a
textured sphere on a textured ground plane, 1280x720 BF16 images, f = 900,
200,000 points with an 8-pixel pattern (33.6 M residuals per iteration), a
600 x 600 reduced camera system -- perturbed by 2 deg / 0.02 / 5 %.
A step is one complete IC solve of the bundle from p_0 with the inputs
resident in HBM: precompute (J, H, Schur complement, factorisation and
inverse of the reduced system) + 20 IC iterations. `value` = IC iterations
per second over the timed steps (precompute amortised over the 20
iterations). FC solves of the same bundle (20 iterations each, Hessian,
Schur complement and factorisation rebuilt every iteration) are timed the
same way beside it. The working set (0.94 GB of stored Jacobian rows, 186 MB
of images) is far larger than L2; L2 is also flushed (512 MB write) between
timed steps, outside the per-step CUDA events. The other workloads
(helix30, ring5, batch256, learned, mlp) run with --workload.

The per-result error of the GPU path against the FP64 oracle (one IC step,
one FC step, the reduced camera system, the parameters after the step) is
measured on a point subset of the workload (every 16th point, all frames),
where the oracle also gives the CPU baseline.

--gpus N under torchrun runs N independent replicas (one bundle per rank,
seeded by rank; no collective on the data path) and reports the aggregate.
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "IC-PBA iterations/s & residuals/s vs FC on same GB300 at equal final RMS error"
UNIT = "iterations/s"
SCENE = "orbit101"
# point-subset stride of the oracle samples: the precision check and CPU
# baseline (ours), and each step of the reference arm
SAMPLE_STRIDE = {"orbit101": 16}
REFERENCE_STRIDE = {"orbit101": 32}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def max_over_ranks(values, dist=None, device="cuda"):
    """The slowest rank's timings: every rank's list reduced element-wise by
    MAX (the value all ranks report); the list itself without a process
    group."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def aggregate_rate(units_per_rank, world, total_ms):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (weak scaling: each rank does the same work)."""
    return world * units_per_rank / (total_ms / 1e3)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--iters", type=int, default=20, help="IC / FC iterations per solve")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--workload", choices=sorted(WORKLOAD_TEXT), default=SCENE,
                   help="orbit101 (the benchmark workload: 100 target frames, BF16 images), helix30 "
                        "(30 frames), ring5 (the 5-frame case), batch256, learned or mlp")
    p.add_argument("--no-autotune", dest="autotune", action="store_false",
                   help="keep the library's default launch shapes instead of letting it time its "
                        "candidates (residual-pass CTA size, factorisation cluster size) at the "
                        "first precompute and keep the fastest")
    p.add_argument("--res-warps", type=int, default=0, choices=[0, 4, 8, 16],
                   help="fix the residual pass at this many warps (entries) per CTA instead of "
                        "autotuning it (0: autotune, or the default with --no-autotune)")
    p.add_argument("--no-graphs", action="store_true",
                   help="submit every kernel with its own launch instead of replaying CUDA graphs")
    p.add_argument("--bundles", type=int, default=256,
                   help="batch workload: number of bundles (default 256)")
    p.add_argument("--train-bundles", type=int, default=2000, help="learned workload: training bundles")
    p.add_argument("--eval-bundles", type=int, default=64, help="learned workload: held-out bundles")
    p.add_argument("--render", choices=("gpu", "host"), default="gpu",
                   help="learned workload: scenes by the CUDA ray caster or the host renderer")
    p.add_argument("--epochs", type=int, default=20, help="learned workload: training epochs")
    p.add_argument("--points", type=int, default=262144, help="mlp workload: feature rows per inference")
    p.add_argument("--point-stride", type=int, default=1,
                   help="keep every k-th point of the workload (a smaller case of the same kernels, for "
                        "profiling; the default 1 is the workload itself)")
    return p.parse_args()


WORKLOAD_TEXT = {
    "ring5": "reference + 4 frames on a +-20 degree ring around a value-noise sphere",
    "helix30": "30-frame 2-turn helix around a value-noise sphere",
    "orbit101": "reference + 100 frames on a 30-degree orbit around a value-noise sphere on a "
                "textured ground plane",
    "mlp": "the learned proposal's network kernels alone on random features",
    "learned": "learned inverse-depth proposal: trained on the converged inverse depths of "
               "generated 30-frame 640x480 FP16 helix bundles, evaluated on held-out bundles against "
               "the constant-depth initialisation",
    "batch256": "independent bundles of uneven size solved together: frames uniform 4-64 on a "
                "helix (24 deg per frame), points log-uniform 500-50,000, sphere radius uniform "
                "0.5-2, texture seed = bundle index, 640x480 FP16, f=525",
}


def workload_config(sc, iters):
    return {"workload": f"{SCENE}: {WORKLOAD_TEXT[SCENE]}, {sc.W}x{sc.H} {sc.dtype.upper()}, "
                        f"f={sc.fx:g}, {sc.N} points x 8-pixel pattern, "
                        f"2 deg/0.02/5% perturbation, {iters} iterations per solve",
            "frames": sc.F, "points": sc.N, "pattern": sc.P,
            "residuals_per_iter": sc.n_residuals(), "reduced_system": 6 * (sc.F - 1),
            "image": f"{sc.W}x{sc.H} {sc.dtype}", "iterations_per_step": iters,
            "l2": "flushed (512 MB write) between timed steps"}


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str | None):
        self.dev = device_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.dev:
                cmd += ["-i", self.dev]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def device_uuid(torch):
    try:
        u = torch.cuda.get_device_properties(torch.cuda.current_device()).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------------------
# the FP64 oracle on a bounded sample: per-result errors of the GPU path and
# the CPU baseline
# ----------------------------------------------------------------------------
def _pose_errors(Pa, Pb):
    import numpy as np
    rot, tr = 0.0, 0.0
    for f in range(1, Pa.shape[0]):
        Ra, Rb = Pa[f, :9].reshape(3, 3), Pb[f, :9].reshape(3, 3)
        c = float(np.clip((np.trace(Ra @ Rb.T) - 1) / 2, -1, 1))
        rot = max(rot, math.degrees(math.acos(c)))
        tr = max(tr, float(np.abs(Pa[f, 9:] - Pb[f, 9:]).max()))
    return rot, tr


def precision_sample(sc, iters, stride, stream, tuning):
    """The GPU path against the FP64 oracle on the bundle restricted to every
    `stride`-th point (all frames and images): one IC step and one FC step
    from p_0 (relative error of the whole update), the anchored reduced
    camera system S (largest entry error over the largest entry), the poses
    and inverse depths after the IC step. The oracle's precompute and IC
    iteration times there, scaled by `stride` (its work is linear in the
    points), give the CPU baseline."""
    import numpy as np
    import oracle
    import synth
    from paper_1704_06967_gb300 import Bundle
    sub = synth.point_subset(sc, stride) if stride > 1 else sc
    pb = oracle.Problem.from_scene(sub)
    t0 = time.perf_counter()
    pre = oracle.ic_precompute(pb, sub.poses0, sub.depths0)
    t1 = time.perf_counter()
    o_dth, o_dd, o_P, o_D, o_st = oracle.ic_step(pb, pre, sub.poses0, sub.depths0, sub.poses0, sub.depths0)
    t2 = time.perf_counter()
    g_theta, g_d, _ = oracle.ic_gradient(pb, pre, sub.poses0, sub.depths0)
    _, _, S_or = oracle.schur_solve(pb.F, pb.N, pre.Hff, pre.Hfd, pre.Hdd, g_theta, g_d, sub.poses0[:, 9:],
                                    want_S=True)
    f_dth, f_dd, _, _, _ = oracle.fc_step(pb, sub.poses0, sub.depths0)

    def rel(dth, dd, r_dth, r_dd):
        got = np.concatenate([dth[1:].ravel(), dd])
        ref = np.concatenate([r_dth[1:].ravel(), r_dd])
        return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))

    b = Bundle.from_scene(sub, stream=stream)
    b.set_tuning(*tuning)
    b.precompute_ic()
    S_gpu = b.system(fc=False)["S"]
    b.iterate(1, stats=False)
    dth, dd = b.last_update()
    P1, D1 = b.params()
    rot, tr = _pose_errors(P1, o_P)
    drel = np.abs(D1 / o_D - 1)
    b.set_params(sub.poses0, sub.depths0)
    b.solve_fc(1, stats=False)
    fdth, fdd = b.last_update()
    b.close()
    errors = {"sample": f"every {stride}th point ({sub.N} points, {sub.n_residuals()} residuals), all "
                        f"{sub.F} frames, the same images; one step from p_0",
              "ic_step_rel_err": rel(dth, dd, o_dth, o_dd),
              "fc_step_rel_err": rel(fdth, fdd, f_dth, f_dd),
              "S_max_err_over_max": float(np.abs(S_gpu - S_or).max() / np.abs(S_or).max()),
              "poses_after_ic_step": {"rot_deg": rot, "trans": tr},
              "inv_depth_after_ic_step": {"max_rel": float(drel.max()), "median_rel": float(np.median(drel))},
              "tolerance": {"step": 1e-4, "rot_deg": 1e-3, "trans": 1e-5}}
    t_pre, t_it = (t1 - t0) * stride, (t2 - t1) * stride
    value = iters / (t_pre + iters * t_it)
    cpu = {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"FP64 oracle IC precompute ({t1 - t0:.2f} s) + one IC iteration ({t2 - t1:.2f} s) on "
                     f"every {stride}th point of the {SCENE} bundle ({sub.N} points, all frames), scaled by "
                     f"{stride} to the whole bundle and to a {iters}-iteration solve; single thread"}
    return errors, cpu


# The all-core leg of the CPU baseline: worker processes forked before the
# first CUDA call, each running the oracle as it stands on its own share of
# the point sample (the scene is shared with the parent copy-on-write).
_FORK_SCENE = None


def _oracle_share(args):
    """(precompute s, one IC iteration s, points) of the oracle on every
    `step`-th point from `offset` of the forked scene."""
    import oracle
    import synth
    step, offset = args
    sub = synth.point_subset(_FORK_SCENE, step, offset=offset)
    pb = oracle.Problem.from_scene(sub)
    t0 = time.perf_counter()
    pre = oracle.ic_precompute(pb, sub.poses0, sub.depths0)
    t1 = time.perf_counter()
    oracle.ic_step(pb, pre, sub.poses0, sub.depths0, sub.poses0, sub.depths0)
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1, sub.N


def fork_oracle_pool(sc):
    """A pool of min(16, host cores) oracle workers forked now, before any
    CUDA call (a process forked after CUDA is initialised can hang)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    global _FORK_SCENE
    _FORK_SCENE = sc
    parts = max(1, min(16, os.cpu_count() or 1))
    pool = cf.ProcessPoolExecutor(max_workers=parts, mp_context=mp.get_context("fork"))
    list(pool.map(time.sleep, [0.05] * parts))  # start every worker now
    return pool, parts


def oracle_all_cores(pool, parts, stride, iters):
    """The oracle on every `stride`-th point split over `parts` processes at
    once; the slowest share's times, scaled by `stride`, estimate a solve of
    the whole bundle on all of them."""
    shares = list(pool.map(_oracle_share, [(stride * parts, stride * k) for k in range(parts)]))
    t_pre = max(x[0] for x in shares) * stride
    t_it = max(x[1] for x in shares) * stride
    value = iters / (t_pre + iters * t_it)
    return {"value": value, "unit": UNIT, "cores": parts, "kind": "oracle",
            "sample": f"FP64 oracle IC precompute + one IC iteration on every {stride}th point of the {SCENE} "
                      f"bundle ({sum(x[2] for x in shares)} points, all frames) split over {parts} processes "
                      f"running at once (every {stride * parts}th point each); the slowest process's times, "
                      f"scaled by {stride} to the whole bundle and to a {iters}-iteration solve (each process "
                      f"also solves the whole reduced system)"}


# ----------------------------------------------------------------------------
# runs that converge: both methods over an image pyramid
# ----------------------------------------------------------------------------
def converged_leg(sc, stream, levels=3, iters=(10, 10, 20)):
    """IC (p_0 re-anchored every 3 iterations) and FC from the perturbed p_0
    over a 3-level image pyramid (coarsest first), untimed by the main
    loop: each level's solve call is timed with CUDA events (the image
    reduction and the per-level context set-up excluded). Reports each
    method's final RMS against the RMS at the true parameters, whether the
    Sec. 4.1 rule (largest pattern-centre displacement of a step < 5e-3 px)
    fired, and the time each needs to reach the higher of the two final RMS
    values (the finest level's time pro rata its iterations)."""
    import numpy as np

    from paper_1704_06967_gb300 import Bundle, pyramid
    from paper_1704_06967_gb300.pba import _scene_images
    img = _scene_images(sc)
    out, fin = {}, {}
    for method in ("ic", "fc"):
        ms = []
        _, _, stats = pyramid.solve_coarse_to_fine(
            img, sc.poses0, sc.intrinsics, sc.uv, sc.depths0, sc.vis, pattern=sc.pattern, huber_k=sc.huber_k,
            levels=levels, iters=iters, method=method, reanchor_every=3, stream=stream, level_ms=ms)
        f = stats[-1]
        fin[method] = f
        hit = np.nonzero(f[:-1, 3] < 5e-3)[0]
        out[method] = {"level_ms": ms, "total_ms": float(sum(ms)), "final_rms": float(f[-1, 1]),
                       "sec41_converged_at": int(hit[0]) + 1 if hit.size else None,
                       "max_disp_px_last_step": float(f[-2, 3])}
    g = Bundle(img, sc.poses_gt, sc.intrinsics, sc.uv, sc.depths_gt, sc.vis, pattern=sc.pattern,
               huber_k=sc.huber_k, stream=stream)
    gt_rms = float(g.solve_fc(0)[0, 1])
    g.close()
    target = max(out["ic"]["final_rms"], out["fc"]["final_rms"])
    n = iters[-1]
    for method in ("ic", "fc"):
        f, o = fin[method], out[method]
        k = int(np.argmax(f[:, 1] <= target * (1 + 1e-12)))
        o["iterations_to_common_rms"] = k
        o["ms_to_common_rms"] = float(sum(o["level_ms"][:-1]) + o["level_ms"][-1] * k / n)
    return {"levels": levels, "iterations_per_level": list(iters), "ic_reanchor_every": 3,
            "true_params_rms": gt_rms, "common_rms": target, "ic": out["ic"], "fc": out["fc"],
            "fc_over_ic_time_to_common_rms": (out["fc"]["ms_to_common_rms"] / out["ic"]["ms_to_common_rms"]
                                              if out["ic"]["ms_to_common_rms"] > 0 else None)}


def small_perturbation_leg(name, stream, tuning, iters=40):
    """The same scene perturbed by 0.25 deg / 0.0025 / 1 % (the class of the
    paper's 1e-3 parameter noise), IC, IC with p_0 re-anchored every 5
    iterations (pba_solve_ic) and FC at full resolution from p_0 for `iters`
    iterations each, timed whole with CUDA events (graph replays); reports
    the final RMS against the RMS at the true parameters, the Sec. 4.1 rule,
    and the time each needs to reach the highest of the final RMS values
    (per-iteration time pro rata, the IC precomputes included)."""
    import numpy as np
    import torch

    import synth
    from paper_1704_06967_gb300 import Bundle
    sc = synth.make_scene(name, rot_deg=0.25, trans=0.0025, sigma_d=0.01)
    b = Bundle.from_scene(sc, stream=stream, use_graphs=True)
    b.set_tuning(*tuning)

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), r
    for _ in range(2):  # capture the graphs
        b.set_params(sc.poses0, sc.depths0)
        b.precompute_ic()
        b.iterate(iters, stats=False)
        b.set_params(sc.poses0, sc.depths0)
        b.solve_fc(iters, stats=False)
    b.set_params(sc.poses0, sc.depths0)
    pre_ms, _ = timed(b.precompute_ic)
    it_ms, _ = timed(lambda: b.iterate(iters, stats=False))
    b.set_params(sc.poses0, sc.depths0)
    b.precompute_ic()
    st_ic = b.iterate(iters)
    b.set_params(sc.poses0, sc.depths0)
    b.solve_ic(iters, reanchor_every=5, stats=False)  # capture
    b.set_params(sc.poses0, sc.depths0)
    ra_ms, _ = timed(lambda: b.solve_ic(iters, reanchor_every=5, stats=False))
    b.set_params(sc.poses0, sc.depths0)
    st_ra = b.solve_ic(iters, reanchor_every=5)
    b.set_params(sc.poses0, sc.depths0)
    fc_ms, _ = timed(lambda: b.solve_fc(iters, stats=False))
    b.set_params(sc.poses0, sc.depths0)
    st_fc = b.solve_fc(iters)
    b.set_params(sc.poses_gt, sc.depths_gt)
    gt_rms = float(b.solve_fc(0)[0, 1])
    b.close()
    target = max(st_ic[-1, 1], st_fc[-1, 1], st_ra[-1, 1])
    out = {}
    for m, st, per, base in (("ic", st_ic, it_ms / iters, pre_ms), ("fc", st_fc, fc_ms / iters, 0.0),
                             ("ic_reanchored_every_5", st_ra, ra_ms / iters, 0.0)):
        k = int(np.argmax(st[:, 1] <= target * (1 + 1e-12)))
        hit = np.nonzero(st[:-1, 3] < 5e-3)[0]
        out[m] = {"final_rms": float(st[-1, 1]), "iteration_ms": per, "precompute_ms": base if m == "ic" else None,
                  "iterations_to_common_rms": k, "ms_to_common_rms": base + k * per,
                  "sec41_converged_at": int(hit[0]) + 1 if hit.size else None,
                  "max_disp_px_last_step": float(st[-2, 3]),
                  "rms_drop_last_5_iterations": float(st[-6, 1] - st[-1, 1])}
    return {"perturbation": "0.25 deg / 0.0025 / 1 %", "iterations": iters, "true_params_rms": gt_rms,
            "common_rms": float(target), "ic": out["ic"], "fc": out["fc"],
            "ic_reanchored_every_5": out["ic_reanchored_every_5"],
            "ic_over_fc_iterations_per_s": out["fc"]["iteration_ms"] / out["ic"]["iteration_ms"],
            "fc_over_ic_time_to_common_rms": (out["fc"]["ms_to_common_rms"] / out["ic"]["ms_to_common_rms"]
                                              if out["ic"]["ms_to_common_rms"] > 0 else None)}


# ----------------------------------------------------------------------------
# reference arm
# ----------------------------------------------------------------------------
def run_reference_batch(args):
    """The oracle on a sample of the batch: per step, one bundle (in batch
    order) gets its IC precompute and one IC iteration, extrapolated to a
    --iters iteration solve; the sample's bundle-iterations over its total
    solve time is the rate of a CPU solving the bundles one after another."""
    import numpy as np
    import oracle
    import synth
    draws = synth.draw_batch(args.bundles)
    n = args.warmup + args.steps
    times = []
    scenes = synth.make_batch(min(n, args.bundles), keep_f32=True, workers=1)
    for i, sc in enumerate(scenes):
        pb = oracle.Problem.from_scene(sc)
        t0 = time.perf_counter()
        pre = oracle.ic_precompute(pb, sc.poses0, sc.depths0)
        t1 = time.perf_counter()
        oracle.ic_step(pb, pre, sc.poses0, sc.depths0, sc.poses0, sc.depths0)
        t2 = time.perf_counter()
        if i >= args.warmup:
            times.append((t1 - t0) + args.iters * (t2 - t1))
    value = args.iters * len(times) / float(np.sum(times))
    sample = (f"{len(times)} bundles of the batch (in batch order, after {args.warmup} warm-up bundles): "
              f"FP64 oracle IC precompute + one IC iteration each, extrapolated to {args.iters} "
              f"iterations; single thread")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "bundle-iterations/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"batch{args.bundles}: {args.bundles} {WORKLOAD_TEXT['batch256']}",
                      "bundles": args.bundles, "frames_total": sum(d.n_frames for d in draws)},
           "cpu_baseline": {"value": value, "unit": "bundle-iterations/s", "cores": 1, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": "bundle-iterations/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if SCENE == "batch256":
        return run_reference_batch(args)
    if SCENE in ("learned", "mlp"):
        print(json.dumps({"impl": "reference", "unavailable": "the learned workloads have no CPU arm: the "
                          "FP64 oracle of the network (oracle/mlp.py) checks its kernels in tests"}), flush=True)
        return 0
    import numpy as np
    import oracle
    import synth
    sc = synth.make_scene(SCENE)
    stride = REFERENCE_STRIDE.get(SCENE, 1)
    sub = synth.point_subset(sc, stride) if stride > 1 else sc
    pb = oracle.Problem.from_scene(sub)
    t0 = time.perf_counter()
    pre = oracle.ic_precompute(pb, sub.poses0, sub.depths0)
    t_pre = (time.perf_counter() - t0) * stride
    poses, depths = sub.poses0, sub.depths0
    for _ in range(args.warmup):
        _, _, poses, depths, _ = oracle.ic_step(pb, pre, sub.poses0, sub.depths0, poses, depths)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, _, poses, depths, _ = oracle.ic_step(pb, pre, sub.poses0, sub.depths0, poses, depths)
        times.append((time.perf_counter() - t0) * stride)
    t_it = float(np.mean(times))
    value = args.iters / (t_pre + args.iters * t_it)
    where = (f"every {stride}th point of the {SCENE} bundle ({sub.N} points, all frames), times scaled by "
             f"{stride} to the whole bundle" if stride > 1 else f"the full {SCENE} bundle")
    sample = (f"one FP64 oracle IC iteration per step on {where}; precompute ({t_pre:.2f} s) timed once and "
              f"amortised over {args.iters} iterations")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * t_it, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(sc, args.iters),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "residuals_per_s": value * sc.n_residuals()}
    print(json.dumps(out), flush=True)
    return 0


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    import synth
    from paper_1704_06967_gb300 import Bundle
    from paper_1704_06967_gb300 import build as pkg_build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus:
        log(f"warning: --gpus {args.gpus} but WORLD_SIZE {world}")
    iters = args.iters
    sc = synth.make_scene(SCENE, seed_offset=rank)
    if args.point_stride > 1:
        sc = synth.point_subset(sc, args.point_stride)
    pool = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool, parts = fork_oracle_pool(sc)  # before the first CUDA call
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        pkg_build.build()
    if dist is not None:
        dist.barrier()

    # a stream of our own (the legacy stream cannot be captured): every
    # library call, L2 flush and timing event below is ordered on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    b = Bundle.from_scene(sc, stream=stream, use_graphs=not args.no_graphs, autotune=args.autotune)
    if args.res_warps:
        b.set_tuning(args.res_warps, b.tuning()[1])  # fixed shape: no autotuning
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def l2_flush(k):
        flush.fill_(k & 0xFF)

    def ic_solve(stats=False):
        b.set_params(sc.poses0, sc.depths0)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        b.precompute_ic()
        e1.record(stream)
        st = b.iterate(iters, stats=stats)
        e2.record(stream)
        e2.synchronize()
        return e0.elapsed_time(e1), e0.elapsed_time(e2), st

    def fc_solve(stats=False):
        b.set_params(sc.poses0, sc.depths0)
        e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
        e0.record(stream)
        st = b.solve_fc(iters, stats=stats)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), st

    # warm-up (the timing masks are those of the timed loops below, so the
    # graphs those loops replay are captured here)
    for i in range(args.warmup):
        l2_flush(i)
        b.enable_timing(1 << 1)
        ic_solve()
        l2_flush(i + 1)
        b.enable_timing(0)
        fc_solve()
    torch.cuda.synchronize()

    # timed IC steps (kernel events around the residual pass only)
    clocks = ClockSampler(device_uuid(torch))
    clocks.start()
    b.enable_timing(1 << 1)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    pre_ms, ic_ms = [], []
    for i in range(args.steps):
        l2_flush(i)
        p, t, _ = ic_solve()
        pre_ms.append(p)
        ic_ms.append(t)
    torch.cuda.synchronize()
    kms, launches, kcounts = b.timing()
    ic_launches = launches
    b.enable_timing(0)
    # FC steps, same protocol
    b.enable_timing(0)
    fc_ms = []
    for i in range(args.steps):
        l2_flush(i + 7)
        t, _ = fc_solve()
        fc_ms.append(t)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()

    total_ic, total_fc = max_over_ranks([sum(ic_ms), sum(fc_ms)], dist)
    R = sc.n_residuals()
    value = aggregate_rate(iters * args.steps, world, total_ic)
    fc_value = aggregate_rate(iters * args.steps, world, total_fc)

    # statistics trajectories for the equal-RMS comparison (untimed)
    _, _, st_ic = ic_solve(stats=True)
    _, st_fc = fc_solve(stats=True)
    pre_avg = statistics.mean(pre_ms)
    it_ic = (statistics.mean(ic_ms) - pre_avg) / iters
    it_fc = statistics.mean(fc_ms) / iters
    target = max(st_ic[-1, 1], st_fc[-1, 1])
    k_ic = int(np.argmax(st_ic[:, 1] <= target * (1 + 1e-12)))
    k_fc = int(np.argmax(st_fc[:, 1] <= target * (1 + 1e-12)))
    t_ic = pre_avg + k_ic * it_ic
    t_fc = k_fc * it_fc

    # sliding window: a frame leaves and enters again; the IC system is
    # updated from the stored products (only the entering frame's entries
    # are precomputed) instead of a full precompute
    def timed_call(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    b.set_params(sc.poses0, sc.depths0)
    full_ms = timed_call(b.precompute_ic)
    mid = sc.F // 2
    win = np.ones(sc.F, bool)
    win[mid] = False
    leave_ms, enter_ms = [], []
    for _ in range(3):
        b.set_window(win)
        leave_ms.append(timed_call(b.update_ic))
        b.set_window(np.ones(sc.F, bool))
        enter_ms.append(timed_call(b.update_ic))
    window = {"full_precompute_ms": full_ms, "frame_leaves_update_ms": min(leave_ms),
              "frame_enters_update_ms": min(enter_ms), "frame": int(mid)}

    # per-kernel breakdown of one IC and one FC solve (diagnostic, untimed)
    b.enable_timing(-1)
    l2_flush(3)
    ic_solve()
    ic_break, _, _ = b.timing()
    b.enable_timing(-1)
    l2_flush(4)
    fc_solve()
    fc_break, _, _ = b.timing()
    b.enable_timing(0)

    # roofline of the IC residual kernel (algorithmic bytes per launch): the
    # stored J rows (28 B per residual), the per-pair J_d^T w r it writes,
    # each point's template intensities, depth and centre once, and every
    # image pixel once
    V = R // sc.P
    img_bytes = sc.F * sc.H * sc.W * (4 if sc.dtype == "f32" else 2)
    alg_bytes = R * 28 + V * 4 + sc.N * sc.P * 4 + sc.N * 12 + img_bytes
    pass_ms = kms["pass"] / max(1, kcounts["pass"])
    hbm_peak, peak_src = measured_peaks()
    achieved = alg_bytes / (pass_ms * 1e-3) / 1e9
    roofline = {"kernel": "ic_residual_kernel", "bound": "hbm", "achieved": achieved,
                "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback",
                "traffic": None, "algorithmic_bytes_per_launch": alg_bytes,
                "avg_launch_ms": pass_ms, "launches": int(kcounts["pass"])}
    traffic_file = os.path.join(ROOT, "profiles", f"ic_residual_{SCENE}_traffic.txt")
    if os.path.exists(traffic_file):
        try:
            # one JSON record per line, one per launch shape
            for line in open(traffic_file):
                tr = json.loads(line) if line.strip() else {}
                # (the traffic of a launch does not depend on its CTA size)
                if tr.get("kernel_sha") == kernel_sha() and tr.get("residuals") == R:
                    roofline["traffic"] = tr["dram_bytes_per_launch"]
        except Exception:
            pass

    # end to end: host buffers through the C ABI (pinned host images)
    pinned = torch.from_numpy(sc.images_store).pin_memory()
    host_imgs = pinned.numpy()
    e2e_t, h2d_b, d2h_b = [], 0, 0
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eb = Bundle(host_imgs, sc.poses0, sc.intrinsics, sc.uv, sc.depths0, sc.vis,
                    pattern=sc.pattern, huber_k=sc.huber_k)
        eb.set_tuning(*b.tuning())  # the shapes found above: no autotuning per context
        eb.precompute_ic()
        eb.iterate(iters, stats=False)
        P, D = eb.params()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e_t.append(t1 - t0)
            h2d_b, d2h_b = eb.transfer_bytes()
        eb.close()
    (e2e_total,) = max_over_ranks([sum(e2e_t)], dist)
    e2e_value = aggregate_rate(iters * args.steps, world, 1e3 * e2e_total)

    try:
        converged = converged_leg(sc, stream)
    except Exception as ex:  # a diagnostic: the headline above stands without it
        converged = {"error": f"{type(ex).__name__}: {ex}"}
    small = None
    if rank == 0:
        try:
            small = small_perturbation_leg(SCENE, stream, b.tuning())
        except Exception as ex:  # a diagnostic, as above
            small = {"error": f"{type(ex).__name__}: {ex}"}

    cpu, precision, cpu_all = None, None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        precision, cpu = precision_sample(sc, iters, SAMPLE_STRIDE.get(SCENE, 1), stream, b.tuning())
        try:
            cpu_all = oracle_all_cores(pool, parts, SAMPLE_STRIDE.get(SCENE, 1), iters)
        except Exception as ex:  # a reported baseline, not the measurement
            cpu_all = {"error": f"{type(ex).__name__}: {ex}"}
        pool.shutdown()

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": total_ic / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": dict(workload_config(sc, iters),
                              submission="one launch per kernel" if args.no_graphs
                              else "one CUDA graph replay per library call",
                              launch_shapes=dict(zip(("residual_warps_per_cta", "ldl_ctas_per_bundle"),
                                                     b.tuning()),
                                                 chosen_by="fixed (--res-warps)" if args.res_warps
                                                 else "autotuner" if args.autotune else "defaults")),
               "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d_b,
                       "d2h_bytes_per_step": d2h_b},
               "gpu_launches": int(ic_launches), "roofline": roofline,
               "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all, "clocks": clk,
               "residuals_per_s": value * R,
               "ic": {"precompute_ms": pre_avg, "iteration_ms": it_ic,
                      "final_rms": float(st_ic[-1, 1])},
               "fc": {"iterations_per_s": fc_value, "residuals_per_s": fc_value * R,
                      "ms_per_solve": total_fc / args.steps, "iteration_ms": it_fc,
                      "final_rms": float(st_fc[-1, 1])},
               "ic_over_fc_iterations_per_s": value / fc_value,
               "equal_rms": {"target_rms": float(target), "ic_iterations": k_ic,
                             "fc_iterations": k_fc, "ic_ms": t_ic, "fc_ms": t_fc,
                             "fc_over_ic_time": (t_fc / t_ic) if t_ic > 0 else None},
               "kernel_ms_per_solve": {"ic": ic_break, "fc": fc_break},
               "sliding_window": window,
               "error_vs_fp64_oracle": precision,
               "coarse_to_fine": converged,
               "small_perturbation": small}
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    b.close()
    return 0


def kernel_sha():
    """Hash of the residual kernel's own source text and of the device
    helpers it calls: the stored DRAM traffic applies only while these are
    unchanged."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1704_06967_gb300", "csrc")

    def body(text, head):
        start = text.index(head)
        return text[start:text.index("\n}\n", start)]

    src = open(os.path.join(csrc, "pba_iter.cu")).read()
    h = hashlib.sha256(body(src, "ic_residual_kernel(DevProblem pb").encode())
    inc = open(os.path.join(csrc, "pba_internal.cuh")).read()
    for head in ("__device__ __forceinline__ float load_px_t(", "__device__ __forceinline__ void warp_sum(",
                 "__device__ __forceinline__ float warp_max1(", "__device__ __forceinline__ float huber_rho("):
        h.update(body(inc, head).encode())
    return h.hexdigest()[:16]


# ----------------------------------------------------------------------------
# batch workload: many independent bundles in one context vs a per-bundle loop
# ----------------------------------------------------------------------------
def run_batch(args):
    import numpy as np
    import torch

    import synth
    from paper_1704_06967_gb300 import Batch, Bundle, PbaError
    from paper_1704_06967_gb300 import build as pkg_build
    from paper_1704_06967_gb300.pba import _scene_images

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        pkg_build.build()
    if dist is not None:
        dist.barrier()
    iters = args.iters
    t0 = time.perf_counter()
    # replicas draw disjoint batches (seed per rank)
    scenes = synth.make_batch(args.bundles, seed=synth.BATCH_SEED + 1000 * rank)
    log(f"generated {len(scenes)} bundles in {time.perf_counter() - t0:.1f} s")
    B = len(scenes)
    R = sum(sc.n_residuals() for sc in scenes)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    imgs = [_scene_images(sc) for sc in scenes]
    s0 = scenes[0]
    items = [(imgs[i], sc.poses0, sc.intrinsics, sc.uv, sc.depths0, sc.vis) for i, sc in enumerate(scenes)]
    batch = Batch(items, pattern=s0.pattern, huber_k=s0.huber_k, stream=stream, use_graphs=True,
                  autotune=args.autotune)
    singles = [Bundle(imgs[i], sc.poses0, sc.intrinsics, sc.uv, sc.depths0, sc.vis, pattern=sc.pattern,
                      huber_k=sc.huber_k, stream=stream, use_graphs=True) for i, sc in enumerate(scenes)]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def reset():
        for i, sc in enumerate(scenes):
            batch.set_params(sc.poses0, sc.depths0, bundle=i)
            singles[i].set_params(sc.poses0, sc.depths0)

    def timed(fn, k):
        flush.fill_(k & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    ic_failed = set()

    def flagged(fn, ctx, failed, bundle=None):
        # a weakly observed bundle can have an indefinite system (flagged by
        # the library per bundle; the others are solved normally)
        try:
            return fn()
        except PbaError as e:
            if e.status not in (5, 6):
                raise
            errs = ctx.bundle_errors()
            failed.update([bundle] if bundle is not None else [int(b) for b in np.flatnonzero(errs)])
            return None

    def batch_ic():
        flagged(batch.precompute_ic, batch, ic_failed)
        flagged(lambda: batch.iterate(iters, stats=False), batch, ic_failed)

    def loop_ic():
        for i, b in enumerate(singles):
            flagged(b.precompute_ic, b, ic_failed, i)
            flagged(lambda: b.iterate(iters, stats=False), b, ic_failed, i)

    fc_failed = set()

    def batch_fc(stats=False):
        # a weakly observed bundle can make FC's system indefinite (the FP64
        # oracle agrees on such bundles); the library flags that bundle and
        # the others are solved normally
        try:
            return batch.solve_fc(iters, stats=stats)
        except PbaError as e:
            if e.status not in (5, 6):
                raise
            fc_failed.update(int(b) for b in np.flatnonzero(batch.bundle_errors()))
            return None

    for i in range(args.warmup):
        reset()
        batch.enable_timing(1 << 1)
        timed(batch_ic, i)
        batch.enable_timing(0)
        if i == 0 and args.autotune:
            # the per-bundle loop runs the shapes the batch's first precompute chose
            for b in singles:
                b.set_tuning(*batch.tuning())
        timed(loop_ic, i + 1)
        timed(batch_fc, i + 2)
    torch.cuda.synchronize()
    clocks = ClockSampler(device_uuid(torch))
    clocks.start()
    batch.enable_timing(1 << 1)
    if dist is not None:
        dist.barrier()
    ic_ms, loop_ms, fc_ms = [], [], []
    for i in range(args.steps):
        reset()
        ic_ms.append(timed(batch_ic, i))
    kms, launches, kcounts = batch.timing()
    batch.enable_timing(0)
    for i in range(args.steps):
        reset()
        loop_ms.append(timed(loop_ic, i + 3))
        fc_ms.append(timed(batch_fc, i + 5))
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    total_ic, total_loop, total_fc = max_over_ranks([sum(ic_ms), sum(loop_ms), sum(fc_ms)], dist)
    value = aggregate_rate(B * iters * args.steps, world, total_ic)
    loop_value = aggregate_rate(B * iters * args.steps, world, total_loop)
    fc_value = aggregate_rate(B * iters * args.steps, world, total_fc)

    # the batch and the loop must agree exactly (each bundle's sums keep their
    # order) on the same Schur path: the automatic choice goes by the size of
    # the whole context, so it is fixed to the exact-product SIMT path here
    from paper_1704_06967_gb300.pba import PBA_SCHUR_AUTO, PBA_SCHUR_SIMT
    batch.set_schur_path(PBA_SCHUR_SIMT)
    for sb in singles:
        sb.set_schur_path(PBA_SCHUR_SIMT)
    reset()
    batch_ic()
    loop_ic()
    torch.cuda.synchronize()
    mismatch = 0
    for i in range(0, B, max(1, B // 16)):
        if i in ic_failed:
            continue
        P1, D1 = batch.params(i)
        P2, D2 = singles[i].params()
        mismatch += int(not (np.array_equal(P1, P2) and np.array_equal(D1, D2)))
    batch.set_schur_path(PBA_SCHUR_AUTO)
    # final RMS of the batch's IC and FC solves (sums over the bundles)
    reset()
    flagged(batch.precompute_ic, batch, ic_failed)
    st_ic = flagged(lambda: batch.iterate(iters), batch, ic_failed)
    reset()
    st_fc = batch_fc(stats=True)

    # roofline of the residual kernel over all bundles. Image term: each
    # image once, capped at the four taps of every residual (the batch's
    # bundles hold 500-50,000 points, so most of an image is never sampled
    # and "every pixel once" would exceed what the pass has to read)
    V = R // s0.P
    img_bytes = min(sum(sc.F for sc in scenes) * s0.H * s0.W, 4 * R) * 2
    N = sum(sc.N for sc in scenes)
    alg_bytes = R * 28 + V * 4 + N * s0.P * 4 + N * 12 + img_bytes
    pass_ms = kms["pass"] / max(1, kcounts["pass"])
    hbm_peak, peak_src = measured_peaks()
    achieved = alg_bytes / (pass_ms * 1e-3) / 1e9
    roofline = {"kernel": "ic_residual_kernel", "bound": "hbm", "achieved": achieved, "peak": hbm_peak,
                "unit": "GB/s", "frac": achieved / hbm_peak,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback",
                "traffic": None, "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": pass_ms,
                "launches": int(kcounts["pass"]),
                "image_bytes": "each image once, capped at 4 taps x 2 B per residual"}

    # end to end through the C ABI with host images (pinned), one context
    e2e_t, h2d_b, d2h_b = [], 0, 0
    host = [torch.from_numpy(sc.images_store).pin_memory().numpy() for sc in scenes]
    for i in range(1 + min(args.steps, 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eb = Batch([(host[j], sc.poses0, sc.intrinsics, sc.uv, sc.depths0, sc.vis)
                    for j, sc in enumerate(scenes)], pattern=s0.pattern, huber_k=s0.huber_k)
        eb.set_tuning(*batch.tuning())  # the shapes found above
        flagged(eb.precompute_ic, eb, set())
        flagged(lambda: eb.iterate(iters, stats=False), eb, set())
        for j in range(B):
            eb.params(j)
        torch.cuda.synchronize()
        if i >= 1:
            e2e_t.append(time.perf_counter() - t0)
            h2d_b, d2h_b = eb.transfer_bytes()
        eb.close()
    e2e_value = world * B * iters * len(e2e_t) / sum(e2e_t)

    Fs = [sc.F for sc in scenes]
    Ns = [sc.N for sc in scenes]
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "bundle-iterations/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ic / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic",
               "config": {"workload": f"batch{B}: {B} {WORKLOAD_TEXT['batch256']}, 8-pixel pattern, "
                                      f"2 deg/0.02/5% perturbation; a step is one IC solve of every "
                                      f"bundle (precompute + {iters} iterations) in one context",
                          "bundles": B, "frames_total": sum(Fs), "frames_min_max": [min(Fs), max(Fs)],
                          "points_total": N, "points_min_max": [min(Ns), max(Ns)],
                          "residuals_per_iter": R, "iterations_per_step": iters,
                          "submission": "one CUDA graph replay per library call",
                          "l2": "flushed (512 MB write) between timed steps",
                          "launch_shapes": dict(zip(("residual_warps_per_cta", "ldl_ctas_per_bundle"),
                                                    batch.tuning()),
                                                chosen_by="autotuner" if args.autotune else "defaults")},
               "e2e": {"value": e2e_value, "unit": "bundle-iterations/s", "h2d_bytes_per_step": h2d_b,
                       "d2h_bytes_per_step": d2h_b},
               "gpu_launches": int(launches), "roofline": roofline, "cpu_baseline": None, "clocks": clk,
               "residuals_per_s": value * R / B,
               "per_bundle_loop": {"value": loop_value, "unit": "bundle-iterations/s",
                                   "ms_per_step": total_loop / args.steps,
                                   "batch_over_loop": value / loop_value},
               "fc_batch": {"value": fc_value, "unit": "bundle-iterations/s",
                            "ms_per_step": total_fc / args.steps,
                            "final_rms": float(st_fc[-1, 1]) if st_fc is not None else None,
                            "bundles_not_positive_definite": sorted(fc_failed)},
               "ic_final_rms": float(st_ic[-1, 1]) if st_ic is not None else None,
               "ic_bundles_not_positive_definite": sorted(ic_failed),
               "ic_over_fc_iterations_per_s": value / fc_value,
               "batch_equals_loop": {"schur_path": "SIMT (exact products) on both",
                                     "bundles_checked": len(range(0, B, max(1, B // 16))),
                                     "mismatches": mismatch}}
        print(json.dumps(out), flush=True)
    for b in singles:
        b.close()
    batch.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0 if mismatch == 0 else 1


# ----------------------------------------------------------------------------
# learned workload: depth proposal trained on the method's own solutions
# ----------------------------------------------------------------------------
def learned_scene(i, device=None):
    """30-frame 640x480 FP16 helix bundle around a sphere (radius uniform
    0.7-1.5) on a ground plane, poses known to 0.1 deg / 0.001: the
    proposal's setting, new points of tracked frames whose depths are
    unknown. device="cuda": rendered by the CUDA ray caster."""
    import synth
    rng = __import__("numpy").random.default_rng(synth.BATCH_SEED + 7 + i)
    cfg = synth.SceneConfig(f"learned{i}", 640, 480, 525.0, 5000, "helix", n_frames=30, spacing=1,
                            sphere_r=float(rng.uniform(0.7, 1.5)), plane=True, dtype="f16", rot_deg=0.1,
                            trans=0.001, allow_fewer_points=True)
    return synth.make_scene(cfg, seed_offset=5000 + i, device=device)


def _learned_scene_star(i):
    sc = learned_scene(i)
    sc.images_f32 = None
    return sc


def run_learned(args):
    import concurrent.futures as cf
    import multiprocessing as mp

    import numpy as np
    import torch

    from paper_1704_06967_gb300 import Bundle, PbaError
    from paper_1704_06967_gb300 import build as pkg_build
    from paper_1704_06967_gb300.learned import DepthMLP, training_pairs
    from paper_1704_06967_gb300.pba import _scene_images

    pkg_build.build()
    ntr, nev, iters = args.train_bundles, args.eval_bundles, args.iters
    t0 = time.perf_counter()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    Xs, Ts = [], []

    def add_pairs(sc):
        tp = training_pairs(sc, iters=iters, stream=stream)
        if tp is not None:
            X, d, use = tp
            Xs.append(X[torch.tensor(use, device="cuda")])
            Ts.append(torch.tensor(d[use], dtype=torch.float32, device="cuda"))

    if args.render == "gpu":
        # rendered on the device one bundle at a time (the CUDA ray caster);
        # each training bundle is solved and dropped
        import synth
        synth.build_renderer_gpu()
        for i in range(ntr):
            add_pairs(learned_scene(i, device="cuda"))
        held = [learned_scene(i, device="cuda") for i in range(ntr, ntr + nev)]
    else:
        with cf.ProcessPoolExecutor(max_workers=max(1, min(8, (os.cpu_count() or 2) // 2)),
                                    mp_context=mp.get_context("spawn")) as ex:
            scenes = list(ex.map(_learned_scene_star, range(ntr + nev)))
        held = scenes[ntr:]
        for sc in scenes[:ntr]:
            add_pairs(sc)
    gen_s = time.perf_counter() - t0
    log(f"generated and solved {ntr + nev} bundles ({args.render} rendering) in {gen_s:.1f} s")
    X, T = torch.cat(Xs).contiguous(), torch.cat(Ts).contiguous()
    net = DepthMLP(seed=0, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    hist = net.train(X, T, epochs=args.epochs, batch=1024, lr=2e-3)
    e1.record(stream)
    e1.synchronize()
    train_ms = e0.elapsed_time(e1)
    n_samples = (X.shape[0] // 1024) * 1024 * args.epochs

    # inference throughput of the tensor-core kernel on the held-out features
    feats = []
    for sc in held:
        b = Bundle(_scene_images(sc), sc.poses0, sc.intrinsics, sc.uv, np.ones(sc.N), sc.vis,
                   pattern=sc.pattern, huber_k=sc.huber_k, stream=stream)
        feats.append(b.depth_features())
        b.close()
    Fe = torch.cat(feats).contiguous()
    for _ in range(3):
        net.infer(Fe)
    reps = 10
    e0.record(stream)
    for _ in range(reps):
        net.infer(Fe)
    e1.record(stream)
    e1.synchronize()
    infer_ms = e0.elapsed_time(e1) / reps
    flops = 2.0 * Fe.shape[0] * (96 * 128 + 2 * 128 * 128 + 128)

    # held-out bundles: constant inverse depth 1 against the proposal, each
    # solved by IC with damping 0.01 and re-anchoring every 3 iterations
    rows = []
    for sc in held:
        out = {}
        for mode in ("constant", "proposal"):
            b = Bundle(_scene_images(sc), sc.poses0, sc.intrinsics, sc.uv, np.ones(sc.N), sc.vis,
                       pattern=sc.pattern, huber_k=sc.huber_k, stream=stream, damping=0.01)
            if mode == "proposal":
                net.propose(b)
            _, dinit = b.params()
            try:
                st = b.solve_ic(iters, reanchor_every=3)
            except PbaError:
                st = None
            _, d = b.params()
            conv = np.flatnonzero(st[:-1, 3] < 5e-3) if st is not None else np.zeros(0)
            seen = sc.vis[:, 1:].any(1)  # the points the bundle adjustment estimates
            ratio = d[seen] / sc.depths_gt[seen]
            # the monocular scale is a gauge freedom: the depth error after
            # the solve is taken with the median ratio divided out
            scale = float(np.median(ratio)) if np.isfinite(ratio).all() else float("nan")
            out[mode] = (float(st[-1, 0]) if st is not None else float("nan"),
                         float(st[-1, 1]) if st is not None else float("nan"),
                         int(conv[0]) + 1 if conv.size else None,
                         float(np.median(np.abs(ratio / scale - 1.0))),
                         float(np.median(np.abs(dinit[seen] / sc.depths_gt[seen] - 1.0))),
                         float(st[-1, 2]) if st is not None else 0.0)
            b.close()
        rows.append(out)
    ec = np.array([r["constant"][3] for r in rows])
    ep = np.array([r["proposal"][3] for r in rows])
    res = {"metric": "learned inverse-depth proposal vs constant-depth initialisation: median inverse-depth "
                     f"error against the truth after {iters} IC iterations on held-out bundles, the monocular "
                     "scale (median ratio) divided out (mean ratio constant / proposal)",
           "value": float(np.mean(ec / ep)), "unit": "error ratio", "higher_is_better": True,
           "n_gpus": 1, "dtype": "bf16 inference (FP32 accumulation), f32 training", "data": "synthetic",
           "config": {"workload": f"learned: {WORKLOAD_TEXT['learned']}; {ntr} training and {nev} held-out "
                                  f"bundles of up to 5,000 points (sphere radius 0.7-1.5 on a ground plane, "
                                  f"poses known to 0.1 deg / 0.001), targets from {iters} IC iterations, "
                                  f"{args.epochs} epochs of Adam (batch 1024, lr 2e-3); held-out solves: IC "
                                  f"with damping 0.01, re-anchored every 3 iterations",
                      "training_samples": int(X.shape[0]),
                      "scene_generation": {"renderer": "CUDA ray caster (synth/render_gpu.cu)" if args.render == "gpu"
                                           else "host renderer (synth/render.c)",
                                           "seconds_with_training_solves": gen_s}},
           "held_out": {"energy_constant": [r["constant"][0] for r in rows],
                        "energy_proposal": [r["proposal"][0] for r in rows],
                        "valid_residuals_constant": [r["constant"][5] for r in rows],
                        "valid_residuals_proposal": [r["proposal"][5] for r in rows],
                        "initial_median_depth_error_constant": [r["constant"][4] for r in rows],
                        "initial_median_depth_error_proposal": [r["proposal"][4] for r in rows],
                        "rms_constant": [r["constant"][1] for r in rows],
                        "rms_proposal": [r["proposal"][1] for r in rows],
                        "iterations_to_convergence_constant": [r["constant"][2] for r in rows],
                        "iterations_to_convergence_proposal": [r["proposal"][2] for r in rows],
                        "scale_aligned_median_depth_error_constant": [r["constant"][3] for r in rows],
                        "scale_aligned_median_depth_error_proposal": [r["proposal"][3] for r in rows],
                        "convergence_rule": "max pattern-centre displacement of a step < 5e-3 px (Sec. 4.1); "
                                            "null: not reached"},
           "training": {"loss_per_epoch": hist, "ms": train_ms, "samples_per_s": n_samples / (train_ms / 1e3)},
           "inference": {"points": int(Fe.shape[0]), "ms": infer_ms, "points_per_s": Fe.shape[0] / (infer_ms / 1e3),
                         "tflops": flops / (infer_ms * 1e-3) / 1e12, "kernel": "mlp_infer_tc_kernel (tcgen05)"}}
    print(json.dumps(res), flush=True)
    return 0


# ----------------------------------------------------------------------------
# mlp workload: the proposal network's kernels alone (random features)
# ----------------------------------------------------------------------------
def run_mlp(args):
    import torch

    from paper_1704_06967_gb300 import build as pkg_build
    from paper_1704_06967_gb300.learned import DepthMLP

    pkg_build.build()
    n = args.points
    gen = torch.Generator(device="cpu").manual_seed(7)
    X = (torch.randn(n, 96, generator=gen) * 0.8).cuda()
    T = (torch.rand(n, generator=gen) + 0.5).cuda()
    net = DepthMLP(seed=1)
    st = net.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.warmup):
        net.infer(X)
    e0.record(st)
    for _ in range(args.steps):
        net.infer(X)
    e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    flops = 2.0 * n * (96 * 128 + 2 * 128 * 128 + 128)
    nt = min(n, 65536)
    net.train(X[:nt], T[:nt], epochs=1, batch=1024)
    e0.record(st)
    net.train(X[:nt], T[:nt], epochs=2, batch=1024)
    e1.record(st)
    e1.synchronize()
    tms = e0.elapsed_time(e1)
    out = {"metric": "learned-proposal network: tensor-core inference and FP32 training throughput",
           "value": n / (ms * 1e-3), "unit": "points/s", "higher_is_better": True, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "dtype": "bf16 inference (FP32 accumulation)",
           "data": "synthetic (random features)",
           "config": {"workload": f"mlp: 96-128-128-128-1 GELU network, {n} feature rows per inference call "
                                  "(each call synchronises to read the kernel's wait flag)"},
           "inference": {"ms_per_call": ms, "tflops": flops / (ms * 1e-3) / 1e12,
                         "kernel": "mlp_infer_tc_kernel (tcgen05.mma kind::f16, TMEM accumulator)"},
           "training": {"samples_per_s": 2 * (nt // 1024) * 1024 / (tms * 1e-3), "batch": 1024,
                        "kernels": "mlp_grad_kernel + mlp_adam_kernel per step"}}
    print(json.dumps(out), flush=True)
    return 0


def main():
    global SCENE
    args = parse()
    SCENE = args.workload
    if args.impl == "reference":
        return run_reference(args)
    if SCENE == "batch256":
        return run_batch(args)
    if SCENE == "learned":
        return run_learned(args)
    if SCENE == "mlp":
        return run_mlp(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
