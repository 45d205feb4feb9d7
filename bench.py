#!/usr/bin/env python3
"""Benchmark: one training step of differentiable tile-based Gaussian
splatting (project + SH, key emission + depth sort, compositing, image loss,
backward) on the 4M-Gaussian 3840x2160 workload, on N GPUs of one node.

Prints ONE JSON line on rank 0. `value` is Mpix/s of the whole job (rendered
and back-propagated pixels of all ranks / max-over-ranks time). With
--impl reference, the CPU oracle (the plain reference implementation of the
method) is timed instead on bounded window samples of the same workload.

Multi-GPU: the path needs no exchange on one GPU per scene, so --gpus N runs N
independent replicas (weak scaling, no collective on the data path; a
barrier and a max-reduction of the timings only).
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd ms/iter & Mpix/s @4M Gaussians 4K; batched vs per-view, same tol"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 200 for this implementation, about 0.8 s at 4K so that the clock "
                         "record holds several samples; 20 for the reference arm)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="diff_4k", choices=["diff_4k", "batch16", "train_1080p", "tiny", "street"])
    ap.add_argument("--mode", default="batched", choices=["batched", "per_view"])
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the per-view comparison leg")
    ap.add_argument("--tile", default=None, help="WxH tile override, e.g. 16x16 (skips the autotuner)")
    ap.add_argument("--raster", default=None,
                    help="explicit rasteriser configuration TWxTH/Ppx/fB/bB as the autotuner names them, e.g. "
                         "32x16/4px/f128/b256 (skips the autotuner)")
    ap.add_argument("--no-tune", action="store_true",
                    help="use the workload's tile shape and the default rasteriser configuration instead of the "
                         "autotuner's choice")
    ap.add_argument("--gaussians", type=int, default=None, help="override the workload's Gaussian count")
    ap.add_argument("--raster-px", type=int, default=4, choices=[2, 4], help="pixels per thread in the rasteriser")
    ap.add_argument("--loss", default="l1l2", choices=["l1l2", "ssim"],
                    help="image loss of the step: the workload's L1 + L2, or the fused SSIM loss")
    ap.add_argument("--no-morton", action="store_true", help="skip the Morton-order leg")
    ap.add_argument("--no-partitioned", action="store_true", help="skip the partitioned-sort leg")
    ap.add_argument("--kernel", default="step", choices=["step", "ssim_loss"],
                    help="step: the training step (default); ssim_loss: the fused SSIM loss kernel alone on a "
                         "seeded image pair of the workload's view sizes")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 20 if args.impl == "reference" else 200
    return args


# ---------------------------------------------------------------------------
# distributed plumbing (barrier + max over ranks only)
# ---------------------------------------------------------------------------
class Dist:
    def __init__(self, want_gpus):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch
            import torch.distributed as dist

            backend = "nccl" if torch.cuda.is_available() else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(self.local_rank)
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch

        dev = "cuda" if torch.cuda.is_available() and self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def max_over_ranks(values):
    """Combines per-rank step times the way the JSON line reports them."""
    return max(values)


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 50):
        self.gpu = gpu_index
        self.period_ms = int(period_ms)
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", str(self.period_ms)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def mark(self):
        """Wall-clock time of a timed-region boundary (local time, as nvidia-smi stamps its samples)."""
        return datetime.datetime.now()

    def stop(self, t0=None, t1=None):
        """Stops sampling; summary of the samples stamped within [t0, t1] (all
        samples when no window is given)."""
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        return self.summary(t0, t1)

    def summary(self, t0=None, t1=None):
        """Summary of the samples so far stamped within [t0, t1]."""
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in list(self.lines):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f")
                clk, clk_max = float(f[2]), float(f[3])
            except ValueError:
                continue
            if (t0 is not None and ts < t0) or (t1 is not None and ts > t1):
                continue
            sm.append(clk)
            mx.append(clk_max)
            for n, val in zip(names, f[6:10]):
                if val.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "window": "samples stamped inside the timed region"}


def clock_record(clocks, step, t_start, t_end, min_samples=3, extend_s=1.0):
    """The clock summary of the timed region. When the region is shorter than
    a few sampling periods (e.g. 20 steps of 3.7 ms), the same step keeps
    running, untimed, for extend_s more seconds and the summary covers the
    timed region plus that continuation, said so in `window`."""
    import torch

    time.sleep(2 * clocks.period_ms / 1000.0)  # let the sampler deliver the last in-region sample
    clk = clocks.summary(t_start, t_end)
    if (clk.get("samples") or 0) >= min_samples:
        clocks.stop()
        return clk
    t1 = time.perf_counter() + extend_s
    while time.perf_counter() < t1:
        for _ in range(8):
            step.run()
        torch.cuda.synchronize()
    t_ext = clocks.mark()
    clk = clocks.stop(t_start, t_ext)
    clk["window"] = (f"timed region ({(t_end - t_start).total_seconds() * 1e3:.0f} ms) and the same step replayed "
                     f"untimed for {extend_s:.1f} s right after it")
    clk["samples_in_timed_region"] = clocks.summary(t_start, t_end).get("samples", 0)
    return clk


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def make_scene(name, gaussians=None):
    from paper_2606_11390_gb300 import scenes

    return scenes.make(name) if gaussians is None else scenes.make(name, N=gaussians)


def workload_config(scene, args, tile):
    s = scene
    return {"workload": s["name"], "gaussians": int(s["means"].shape[0]), "views": int(s["sizes"].shape[0]),
            "resolutions": sorted({f"{w}x{h}" for w, h in s["sizes"]}), "pixels": int(
                (s["sizes"][:, 0].astype(np.int64) * s["sizes"][:, 1]).sum()),
            "tile": f"{tile[0]}x{tile[1]}", "sh_degree": int(s["cfg"]["sh_degree"]), "mode": args.mode,
            "cuda_graph": args.mode == "batched" and not args.no_graph, "adam": s["name"] == "street",
            "loss": (f"L1 + {s['loss'][1]} L2, computed in the forward kernel" if args.loss == "l1l2"
                     else "0.8 L1 + 0.2 (1 - SSIM), fused kernel"),
            "l2_flush": f"none: inputs (parameters {int(s['means'].shape[0]) * 236 / 1e9:.2f} GB, plus keys) exceed the 129 MB L2"}


# ---------------------------------------------------------------------------
# per-stage timing of an eager step (for the roofline of the dominant kernel)
# ---------------------------------------------------------------------------
def stage_times(step, iters=5):
    """Per-stage times of an eager step on the launching stream (CUDA events
    between the C-ABI calls; the backward timed as its two halves). With the
    L1 + L2 loss the forward kernel computes the loss too: its time is in
    raster_fwd and the loss stage is empty."""
    import torch

    from paper_2606_11390_gb300 import _native as gs
    from paper_2606_11390_gb300 import renderer as R

    names = ["project", "bin_sort", "raster_fwd", "loss", "raster_bwd", "project_bwd"]
    acc = {n: 0.0 for n in names}
    fr, cams = step.frames[0], step.frame_cams[0]
    stream = torch.cuda.current_stream()
    p, gr = step.params, step.grads
    for _ in range(iters):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)]
        # keep the GPU busy while the host enqueues the stages, so that no
        # stage's time includes the host's launch latency
        torch.cuda._sleep(200_000)
        ev[0].record(stream)
        R.project(p, cams, fr)
        ev[1].record(stream)
        R.bin_sort(fr)
        ev[2].record(stream)
        fr.image = step.image
        if step.loss_kind == "l1l2":  # the step's forward computes the loss itself
            R.rasterize_fwd_l1l2(fr, step.target, step.image.numel(), step.w_l1, step.w_l2, False, step.dL_dimage,
                                 step.loss)
            ev[3].record(stream)
        else:
            R.rasterize_fwd(fr)
            ev[3].record(stream)
            step.enqueue_loss()
        ev[4].record(stream)
        gs.gs_rasterize_bwd_pixels(fr.projected, fr.vals, fr.tile_ranges, cams.sizes, fr.cfg, fr.N, fr.final_T,
                                   fr.last, step.dL_dimage, fr.d_projected, cull_masks=fr.cull)
        ev[5].record(stream)
        gs.gs_project_bwd(p["means"], p["log_scales"], p["quats"], p["opacity_logits"], p["sh"], cams.dev,
                          cams.sizes, fr.cfg, fr.counts, fr.d_projected, gr["means"], gr["log_scales"],
                          gr["quats"], gr["opacity_logits"], gr["sh"], fr.status)
        ev[6].record(stream)
        torch.cuda.synchronize()
        for i, n in enumerate(names):
            acc[n] += ev[i].elapsed_time(ev[i + 1])
    return {n: acc[n] / iters for n in names}


def pair_counts(step):
    """Pixel-splat pair counts of the rasteriser on the step's own frame,
    from the pair-counting variants of the forward and backward kernels (the
    same cull and decisions as the timed kernels, run once outside the timed
    region): per kernel, pairs executed, evaluated and composited; plus
    sum(last), the pairs up to each pixel's last contributor."""
    import torch

    from paper_2606_11390_gb300 import _native as gs

    fr, cams = step.frames[0], step.frame_cams[0]
    img, fT, last = torch.empty_like(fr.image), torch.empty_like(fr.final_T), torch.empty_like(fr.last)
    cf = torch.zeros(3, dtype=torch.int64, device=fr.image.device)
    cb = torch.zeros_like(cf)
    dp = torch.empty_like(fr.d_projected)
    gs.gs_rasterize_fwd_counted(fr.projected, fr.vals, fr.tile_ranges, cams.sizes, fr.cfg, img, fT, last, cf)
    gs.gs_rasterize_bwd_pixels_counted(fr.projected, fr.vals, fr.tile_ranges, cams.sizes, fr.cfg, fr.N, fT, last,
                                       step.dL_dimage, dp, cb)
    torch.cuda.synchronize()
    names = ("executed", "evaluated", "composited")
    return {"raster_fwd": dict(zip(names, (int(x) for x in cf.cpu()))),
            "raster_bwd": dict(zip(names, (int(x) for x in cb.cpu()))),
            "sum_last": int(last.to(torch.int64).sum().item())}


# ---------------------------------------------------------------------------
# CPU oracle baseline
# ---------------------------------------------------------------------------
def host_cpu():
    """Host CPU description: logical CPUs available to this process and the
    model name (lscpu, else /proc/cpuinfo)."""
    ncpu = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Vendor ID") and ":" in ln:
                model = (model + " / " if model else "") + ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for ln in f:
                    if ln.lower().startswith(("model name", "cpu part")):
                        model = ln.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"nproc": ncpu, "model": model or "unknown"}


def _cpu_timed(scene, window, threads):
    """One timing of the oracle on the workload (see cpu_sample)."""
    import contextlib

    from oracle import oracle as O
    from paper_2606_11390_gb300 import scenes

    W, H = int(scene["sizes"][0, 0]), int(scene["sizes"][0, 1])
    ww, wh = window
    x0, y0 = (W - ww) // 2 // 16 * 16, (H - wh) // 2 // 16 * 16
    ctx = O.parallel(threads) if threads > 1 else contextlib.nullcontext(1)
    with ctx as used:
        t0 = time.perf_counter()
        proj = O.project(scene)
        t_proj = time.perf_counter() - t0
        d0 = np.zeros((proj["counts"].shape[0], 9))
        t0 = time.perf_counter()
        O.project_bwd(scene, d0)
        t_pbwd = time.perf_counter() - t0
        crop = scenes.crop_view(scene, x0, y0, ww, wh)
        cproj = O.project(crop)
        t0 = time.perf_counter()
        bins = O.bin_sort(crop, cproj)
        ras = O.raster_fwd(crop, cproj, bins)
        L, g = O.loss(ras["image"].astype(np.float32), crop["target"], *crop["loss"])
        O.raster_bwd(crop, cproj, bins, g)
        t_pix = time.perf_counter() - t0
    P = W * H
    total = t_proj + t_pbwd + t_pix * P / (ww * wh)
    return {"value": P / total / 1e6, "threads": int(used), "t_gauss": t_proj + t_pbwd, "t_pix": t_pix,
            "extrapolation": P / (ww * wh), "seconds_measured": round(t_proj + t_pbwd + t_pix, 2)}


def cpu_sample(scene, window=(512, 256)):
    """Times the oracle on the workload, single-threaded and with OpenMP on
    every host core: per-Gaussian stages (projection and its backward) over
    all Gaussians for the full view, per-pixel stages (key sort, compositing
    and its backward) on a centred window, then extrapolates the per-pixel
    stages to the full image. The key sort (std::stable_sort) stays serial in
    both builds."""
    host = host_cpu()
    W, H = int(scene["sizes"][0, 0]), int(scene["sizes"][0, 1])
    one = _cpu_timed(scene, window, 1)
    par = _cpu_timed(scene, window, host["nproc"])
    ww, wh = window

    def sample(r, what):
        return (f"{what} C++ oracle: projection fwd+bwd over all {scene['means'].shape[0]} Gaussians for the full "
                f"{W}x{H} view ({r['t_gauss']:.1f} s), sort+composite+backward on a {ww}x{wh} window "
                f"({r['t_pix']:.1f} s) extrapolated x{r['extrapolation']:.1f} to the full image")

    return {"value": par["value"], "unit": "Mpix/s", "cores": par["threads"], "kind": "oracle",
            "sample": sample(par, f"OpenMP ({par['threads']} threads)"),
            "seconds_measured": par["seconds_measured"], "host": host,
            "single_thread": {"value": one["value"], "unit": "Mpix/s", "cores": 1,
                              "sample": sample(one, "single-threaded"),
                              "seconds_measured": one["seconds_measured"]}}


def reference_arm(args, dist):
    """--impl reference: the oracle, as it stands, timed per step on a bounded
    window sample of the same workload."""
    if dist.rank != 0:
        return 0
    from oracle import oracle as O
    from paper_2606_11390_gb300 import scenes

    O.build()
    scene = make_scene(args.workload)
    W, H = int(scene["sizes"][0, 0]), int(scene["sizes"][0, 1])
    ww, wh = 256, 128
    x0, y0 = (W - ww) // 2 // 16 * 16, (H - wh) // 2 // 16 * 16
    crop = scenes.crop_view(scene, x0, y0, ww, wh)

    def one():
        proj = O.project(crop)
        bins = O.bin_sort(crop, proj)
        ras = O.raster_fwd(crop, proj, bins)
        L, g = O.loss(ras["image"].astype(np.float32), crop["target"], *crop["loss"])
        d = O.raster_bwd(crop, proj, bins, g)
        O.project_bwd(crop, d)

    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    dt = (time.perf_counter() - t0) / args.steps
    value = ww * wh / dt / 1e6
    sample = (f"single-threaded C++ oracle, full step (projection+SH of all {scene['means'].shape[0]} Gaussians, "
              f"sort, compositing, L1+L2 loss, backward) for a {ww}x{wh} window of the {W}x{H} view")
    line = {"metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "impl": "reference",
            "config": {"workload": scene["name"], "sample": f"{ww}x{wh} window", "gaussians": int(scene["means"].shape[0])},
            "cpu_baseline": {"value": value, "unit": "Mpix/s", "cores": 1, "kind": "oracle", "sample": sample,
                             "host": host_cpu()},
            "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# main arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    dist = Dist(args.gpus)
    if args.impl == "reference":
        rc = reference_arm(args, dist)
        dist.close()
        return rc
    import torch

    from paper_2606_11390_gb300 import _native as gs
    from paper_2606_11390_gb300 import renderer as R

    dev = dist.local_rank if torch.cuda.is_available() else 0
    torch.cuda.set_device(dev)
    gs.load()
    if args.kernel == "ssim_loss":
        rc = ssim_only(args, dist)
        dist.close()
        return rc
    scene = make_scene(args.workload, args.gaussians)
    if args.raster_px == 2:
        scene["cfg"] = dict(scene["cfg"], flags=gs.GS_FLAG_RASTER_2PX)
    tile = tuple(int(x) for x in args.tile.split("x")) if args.tile else (scene["cfg"]["tile_w"], scene["cfg"]["tile_h"])
    raster_kw = {"tile": tile}
    tune = None
    if args.raster:
        from paper_2606_11390_gb300 import autotune

        c = autotune.parse_name(args.raster)
        raster_kw = autotune.step_kwargs(c)
        tile = raster_kw["tile"]
        tune = {"choice": autotune.name(c), "ms": {}}
    elif not args.no_tune and not args.tile and args.raster_px == 4:
        # the rasteriser configuration (tile shape, pixels per thread, splats
        # per batch) from the autotuner, timed on this GPU for this workload
        from paper_2606_11390_gb300 import autotune

        best, tune_ms = autotune.best_config(scene, steps=5, mode=args.mode)
        raster_kw = autotune.step_kwargs(best)
        tile = raster_kw["tile"]
        tune = {"choice": autotune.name(best), "ms": {k: round(v, 4) for k, v in tune_ms.items()}}
    adam = scene["name"] == "street"  # the street workload's step includes the fused Adam update
    step = R.TrainStep(scene, mode=args.mode, graph=False if args.no_graph else None, adam=adam, loss=args.loss,
                       **raster_kw).prepare()
    P = step.cams.n_pixels
    launches = step.launches_per_step
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        step.run()
    torch.cuda.synchronize()
    step.check()

    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start = clocks.mark()
    e0.record(stream)
    for _ in range(args.steps):
        step.run()
    e1.record(stream)
    torch.cuda.synchronize()
    t_end = clocks.mark()
    clk = clock_record(clocks, step, t_start, t_end)
    dist.barrier()
    step.check()
    ms_local = e0.elapsed_time(e1) / args.steps
    ms = dist.max(ms_local)
    value = dist.world * P / (ms * 1e-3) / 1e6

    extra = {}
    if dist.rank == 0:
        # per-stage times from an instrumented eager step (same kernels, same stream)
        if args.mode == "batched":
            st = stage_times(step)
            extra["stage_ms"] = {k: round(v, 4) for k, v in st.items()}
            extra["n_isect"] = step.n_isect()
            pc = pair_counts(step)
            extra["raster_pairs"] = pc
            dom = max(st, key=st.get)
            peaks, src = measured_peaks()
            extra["roofline"] = roofline_for(dom, st[dom], step, peaks, src, scene["name"], pc)
            extra["stage_roofline"] = {k: roofline_for(k, v, step, peaks, src, scene["name"], pc)
                                       for k, v in st.items() if k in ROOFLINE_STAGES}
            if step.adam_on:
                extra["adam"] = adam_measure(step, peaks, src)
            extra["ssim_loss"] = ssim_kernel_measure(step.image, step.target, step.cams.sizes, peaks, src)
            extra["densify_stats"] = densify_measure(step, peaks, src)
            if not args.no_partitioned and scene["name"] != "street":
                extra["partitioned_sort"] = partitioned_sort_measure(step)
            if not args.no_morton and scene["name"] != "street":
                extra["morton"] = morton_measure(step, scene, args, raster_kw, ms)
        if not args.no_e2e:
            extra["e2e"] = e2e_measure(step, args, dist.world)
            extra["e2e_params_streamed"] = e2e_measure(step, args, dist.world, stream_params=True)
        del step
        torch.cuda.empty_cache()
        if not args.no_compare and args.workload == "diff_4k":
            extra["batched_vs_per_view"] = batched_vs_per_view(args)
        if not args.no_cpu_baseline:
            extra["cpu_baseline"] = cpu_sample(scene)

    if dist.rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": dist.world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(scene, args, tile), "clocks": clk,
                "gpu_launches": launches * args.steps}
        if tune is not None:
            line["config"]["raster"] = tune["choice"]
            line["autotune"] = tune
        line.update(extra)
        print(json.dumps(line), flush=True)
    dist.close()
    return 0


# Algorithmic FP32 work of the method per (pixel, splat) pair, mul and add
# counted separately, by what the compositing rule does with the pair.
# Forward, composited 24: offsets and power 9, exp 2, alpha 2 (opacity
# product, cap), threshold tests 2, transmittance 2, colour 7 (weight
# alpha T, three multiply-adds); evaluated and skipped (power < 0, alpha <
# alpha_min, or the stopping entry) 15: the first four groups only.
# Backward, composited 60: alpha recomputation 17 (offsets, power, exp,
# alpha, the skip tests and the cap test), transmittance recovery 2, colour
# gradient 7, alpha gradient and running colour sum 10, 2D-mean, conic and
# opacity gradients 15, accumulation into the splat's nine sums 9; evaluated
# and not composited 17 (the alpha recomputation that finds it skipped).
# Pairs the per-warp cull drops are work the kernel provably does not need
# and are not charged; pairs a lane executes for a pixel that has stopped or
# lies outside the image are waste, not work.
FLOP_PER_PAIR = {"raster_fwd": {"composited": 24, "skipped": 15},
                 "raster_bwd": {"composited": 60, "skipped": 17}}
ROOFLINE_STAGES = ("project", "bin_sort", "raster_fwd", "raster_bwd", "project_bwd")


# CUDA sources that make up each timed stage (plus the shared headers).
RASTER_SOURCES = ["raster.cu", "raster_kernels.cuh", "raster_launch.h", "raster_inst_fwd.cu", "raster_inst_bwd.cu",
                  "raster_inst_aux.cu"]
KERNEL_SOURCES = {"raster_fwd": RASTER_SOURCES, "raster_bwd": RASTER_SOURCES, "project": ["project.cu"],
                  "project_bwd": ["project.cu"], "bin_sort": ["binsort.cu"], "loss": ["loss_adam.cu"],
                  "ssim_loss": ["ssim.cu"]}
COMMON_SOURCES = ["gs_common.cuh", "gs_internal.h"]


def kernel_digest(kernel):
    """Digest of the CUDA sources of one stage, to tie recorded ncu traffic to
    the kernel it was measured on."""
    import hashlib

    from paper_2606_11390_gb300 import build as B

    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel] + COMMON_SOURCES:
        with open(os.path.join(B.CSRC, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def raster_variant(stage, cfg):
    """Template instance the rasteriser stage launches under a step
    configuration, e.g. raster_bwd<32,16,4,256> (tile, pixels per thread,
    splats per batch; a batch of 0 resolves to the kernel's default)."""
    from paper_2606_11390_gb300 import _native as gs

    tw, th = int(cfg["tile_w"]), int(cfg["tile_h"])
    ppt = 2 if (tw, th) == (8, 8) or int(cfg.get("flags", 0)) & gs.GS_FLAG_RASTER_2PX else 4
    nt = tw * th // ppt
    if stage == "raster_fwd":
        batch = int(cfg.get("raster_batch_fwd", 0)) or (nt if nt > 128 else 128)
    else:
        batch = int(cfg.get("raster_batch_bwd", 0)) or min(max(nt, 64), 256)
    return f"{stage}<{tw},{th},{ppt},{batch}>"


def recorded_traffic(kernel, workload, variant=None):
    """DRAM bytes per launch of `kernel` on `workload` from profiles/dram_traffic.json
    (entries keyed kernel|workload, or kernel|workload|instance for the
    rasteriser's template instances), if they were captured from the kernel's
    current sources and, where the entry names one, the same instance; else None."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    e = d.get(f"{kernel}|{workload}|{variant}") if variant is not None else None
    e = e or d.get(f"{kernel}|{workload}")
    if not e or kernel not in KERNEL_SOURCES or e.get("digest") != kernel_digest(kernel):
        return None
    if variant is not None and e.get("variant") not in (None, variant):
        return None
    return e.get("bytes_per_launch")


def raster_work(stage, pc):
    """Algorithmic FLOPs of one rasteriser launch from its pair counts, with
    the charge of each class."""
    c = pc[stage]
    f = FLOP_PER_PAIR[stage]
    comp, skipped = c["composited"], c["evaluated"] - c["composited"]
    flops = comp * f["composited"] + skipped * f["skipped"]
    return flops, {"composited": {"pairs": comp, "flop_per_pair": f["composited"]},
                   "evaluated_not_composited": {"pairs": skipped, "flop_per_pair": f["skipped"]},
                   "executed_lane_pairs": c["executed"], "sum_last": pc["sum_last"],
                   "lane_efficiency": c["evaluated"] / max(c["executed"], 1)}


def roofline_for(stage, ms, step, peaks, src, workload, pc=None):
    """Achieved vs peak of one stage. The rasteriser is bound by FP32 issue:
    algorithmic FLOPs = the pairs it evaluates, charged by class (composited
    or skipped; see FLOP_PER_PAIR), counted by the kernels' pair-counting
    variants; peak = SMs x 128 FP32 lanes x 2 (FMA) x max SM clock. The other
    stages are HBM-bound with the algorithmic bytes of their inputs and
    outputs."""
    import torch

    N, V, I, P = step.N, step.cams.V, step.n_isect(), step.cams.n_pixels
    variant = raster_variant(stage, step.cfg) if stage in FLOP_PER_PAIR else None
    traffic = recorded_traffic(stage, workload, variant)
    if stage in FLOP_PER_PAIR:
        pc = pc if pc is not None else pair_counts(step)
        flops, work = raster_work(stage, pc)
        sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
        n_sm = torch.cuda.get_device_properties(0).multi_processor_count
        peak = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12
        achieved = flops / (ms * 1e-3) / 1e12
        return {"kernel": stage, "variant": variant, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_source": f"{n_sm} SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz ({src} max SM clock; no measured FP32 peak)",
                "work": work, "flop": flops, "ms": ms}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    if stage == "project":
        bytes_ = N * 236 + V * N * (48 + 8 + 4)
    elif stage == "project_bwd":
        bytes_ = N * 236 * 2 + V * N * 40
    elif stage == "bin_sort":
        # the stage's minimal data movement: per record its depth key and tile
        # count read, per visible record its rectangle, per intersection its
        # 4-byte list entry written, per tile its range
        n_vis = int((step.frames[0].counts != 0).sum().item())
        bytes_ = V * N * 8 + n_vis * 8 + I * 4 + int(step.frames[0].n_tiles) * 8
    else:
        bytes_ = P * 3 * 4 * 3
    achieved = bytes_ / (ms * 1e-3) / 1e9
    return {"kernel": stage, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": traffic, "peak_source": f"{src} hbm_gbs", "ms": ms}


# Algorithmic FP32 work of the fused SSIM loss per pixel and channel, from the
# separable form without halo recomputation: five window sums (x, y, xx, yy,
# xy) as two 11-tap passes (5 x 2 x 11 x 2 = 220), SSIM and its three
# partials (30), three backward window sums (3 x 2 x 11 x 2 = 132) and the
# final combination with the L1 term (6).
SSIM_FLOP_PER_VALUE = 388


def ssim_kernel_measure(image, target, sizes, peaks, src, iters=20, warmup=3):
    """The fused SSIM loss kernel alone on an image and target (CUDA events
    on the launching stream; at 3840x2160 the three images together exceed
    L2). Bound: FP32 issue."""
    import torch

    from paper_2606_11390_gb300 import _native as gs

    sizes = np.asarray(sizes, np.int32).reshape(-1, 2)
    P = int((sizes[:, 0].astype(np.int64) * sizes[:, 1]).sum())
    g = torch.empty_like(image)
    loss = torch.zeros(1, dtype=torch.float64, device=image.device)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        gs.gs_ssim_loss(image, target, sizes, 0.2, g, loss)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(iters):
        gs.gs_ssim_loss(image, target, sizes, 0.2, g, loss)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / iters
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    peak = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12
    achieved = 3 * P * SSIM_FLOP_PER_VALUE / (ms * 1e-3) / 1e12
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    gbs = 3 * P * 12 / (ms * 1e-3) / 1e9
    return {"ms": ms, "loss": float(loss.item()), "launches": 1,
            "roofline": {"kernel": "ssim_loss", "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "work": f"{3 * P} values x {SSIM_FLOP_PER_VALUE} FLOP",
                         "peak_source": f"{n_sm} SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz ({src} max SM clock)"},
            "hbm": {"achieved_gbs": gbs, "peak_gbs": hbm, "frac": gbs / hbm, "bytes": 3 * P * 12}}


def partitioned_sort_measure(step, parts=(1, 2, 4, 8), iters=10):
    """gs_bin_sort_partitioned on the step's projected records for several
    partition counts (1 = the plain gs_bin_sort): the paper's multi-device
    depth sort (local sorts + merge-path merge tree) emulated on one GPU."""
    import torch

    from paper_2606_11390_gb300 import renderer as R

    fr0 = step.frames[0]
    stream = torch.cuda.current_stream()
    out = {}
    for P in parts:
        fr = R.Frame(step.N, fr0.cams, fr0.cfg, capacity=fr0.capacity, partitions=P)
        fr.projected.copy_(fr0.projected)
        fr.rects.copy_(fr0.rects)
        fr.counts.copy_(fr0.counts)
        fr.depth_keys.copy_(fr0.depth_keys)
        for _ in range(2):
            R.bin_sort(fr)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(iters):
            R.bin_sort(fr)
        b.record(stream)
        torch.cuda.synchronize()
        if fr.read_status() != 0:
            raise RuntimeError(f"partitioned sort status {fr.read_status()}")
        out[str(P)] = a.elapsed_time(b) / iters
        del fr
        torch.cuda.empty_cache()
    return {"bin_sort_ms_by_partitions": out}


def adam_measure(step, peaks, src, iters=10):
    """gs_adam_step (the fused Adam update of the step's optimiser) alone on
    the step's parameters, gradients and moments (CUDA events on the
    launching stream; at 64M Gaussians each array is 15 GB, far beyond L2).
    HBM-bound: per scalar p, g, m, v read and p, m, v written, 28 B. The
    extra updates move the parameters by iters x lr, after every timed step."""
    import torch

    from paper_2606_11390_gb300 import _native as gs

    stream = torch.cuda.current_stream()
    p, g = step.params.flat, step.grads.flat
    b1, b2 = step.betas

    def one():
        step.step_count.add_(1)
        gs.gs_adam_step(p, g, step.exp_avg, step.exp_avg_sq, step.lr, b1, b2, step.eps, step.step_count)

    one()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(iters)]
    for a, b in ev:
        step.step_count.add_(1)
        a.record(stream)
        gs.gs_adam_step(p, g, step.exp_avg, step.exp_avg_sq, step.lr, b1, b2, step.eps, step.step_count)
        b.record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / iters
    n = p.numel()
    bytes_ = 28 * n
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    gbs = bytes_ / (ms * 1e-3) / 1e9
    return {"ms": ms, "scalars": n, "launches": 1,
            "roofline": {"kernel": "adam", "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                         "frac": gbs / hbm, "traffic": None, "work": f"{n} scalars x 28 B",
                         "peak_source": f"{src} hbm_gbs"}}


def densify_measure(step, peaks, src, iters=20):
    """gs_densify_stats alone on the step's backward buffers (one launch per
    step when TrainStep(densify_stats=True)); HBM-bound: per (view, Gaussian)
    the tile count, the 2D-mean gradient and the radius (16 B), per Gaussian
    three running statistics read and written (24 B)."""
    import torch

    from paper_2606_11390_gb300 import _native as gs

    fr = step.frames[0]
    N, V = step.N, step.cams.V
    arrs = [torch.zeros(N, dtype=torch.float32, device=step.image.device) for _ in range(3)]
    stream = torch.cuda.current_stream()
    for _ in range(3):
        gs.gs_densify_stats(fr.projected, fr.counts, fr.d_projected, N, step.cams.sizes, *arrs)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(iters):
        gs.gs_densify_stats(fr.projected, fr.counts, fr.d_projected, N, step.cams.sizes, *arrs)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / iters
    bytes_ = V * N * 16 + N * 24
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    gbs = bytes_ / (ms * 1e-3) / 1e9
    return {"ms": ms, "launches": 1, "roofline": {"kernel": "densify_stats", "bound": "hbm", "achieved": gbs,
                                                  "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "traffic": None,
                                                  "peak_source": f"{src} hbm_gbs"}}


def morton_measure(step, scene, args, raster_kw, ms_input_order):
    """The same step after reordering the Gaussians along a 3D Morton curve
    (gs_morton_order + gs_gather_rows, timed separately), as the paper does at
    densification; the input order of the synthetic scenes is random."""
    import torch

    from paper_2606_11390_gb300 import renderer as R

    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    out = R.FlatParams(step.N)
    for _ in range(2):  # warm-up, then timed
        ev[0].record(stream)
        perm, status = R.morton_permutation(step.params)
        ev[1].record(stream)
        R.permute_gaussians(step.params, perm, out=out, status=status)
        ev[2].record(stream)
        torch.cuda.synchronize()
    if status.item() != 0:
        raise RuntimeError(f"morton status {status.item()}")
    order_ms, gather_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    st = R.TrainStep(scene, mode=args.mode, graph=False if args.no_graph else None, params=out, **raster_kw,
                     loss=args.loss).prepare()
    for _ in range(args.warmup):
        st.run()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        st.run()
    b.record(stream)
    torch.cuda.synchronize()
    st.check()
    ms = a.elapsed_time(b) / args.steps
    stages = stage_times(st)
    del st
    torch.cuda.empty_cache()
    return {"order_ms": order_ms, "gather_ms": gather_ms, "ms_per_step": ms,
            "Mpix_s": step.cams.n_pixels / (ms * 1e-3) / 1e6, "speedup_vs_input_order": ms_input_order / ms,
            "stage_ms": {k: round(v, 4) for k, v in stages.items()}}


def ssim_only(args, dist):
    """--kernel ssim_loss: the fused SSIM loss alone on a seeded image pair
    (uniform image, target = image + N(0, 0.05) clipped) of the workload's
    view sizes; K timed launches after W warm-up launches."""
    import torch

    from paper_2606_11390_gb300 import scenes

    sizes = scenes.make_sizes(args.workload)
    P = int((sizes[:, 0].astype(np.int64) * sizes[:, 1]).sum())
    rng = np.random.default_rng(2024)
    img = rng.uniform(0.0, 1.0, (P * 3,)).astype(np.float32)
    tgt = np.clip(img + 0.05 * rng.standard_normal(P * 3), 0.0, 1.0).astype(np.float32)
    image, target = torch.from_numpy(img).cuda(), torch.from_numpy(tgt).cuda()
    peaks, src = measured_peaks()
    r = ssim_kernel_measure(image, target, sizes, peaks, src, iters=args.steps, warmup=max(args.warmup, 1))
    ms = dist.max(r["ms"])
    if dist.rank == 0:
        line = {"metric": "fused SSIM loss fwd+bwd", "value": dist.world * P / (ms * 1e-3) / 1e6, "unit": "Mpix/s",
                "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": {"workload": f"ssim_loss@{args.workload}",
                                                "resolutions": sorted({f"{w}x{h}" for w, h in sizes}),
                                                "pixels": P, "l2_flush": "none: image, target and gradient exceed L2"
                                                if P * 36 > 129e6 else "none (fits L2)"},
                "roofline": r["roofline"], "hbm": r["hbm"], "gpu_launches": args.steps}
        print(json.dumps(line), flush=True)
    return 0


def batched_vs_per_view(args, tile=None):
    """The 16-view workload through the batched, graph-captured step and the
    plain per-view step on the same GPU; tile size from the autotuner."""
    import torch

    from paper_2606_11390_gb300 import autotune
    from paper_2606_11390_gb300 import renderer as R

    scene = make_scene("batch16")
    if tile is None:
        best, tune = autotune.best_config(scene, steps=2)
    else:
        best, tune = {"tile": tuple(tile), "ppt": 4, "batch_fwd": 0, "batch_bwd": 0}, {}
    kw = autotune.step_kwargs(best)
    out = {"workload": "batch16", "gaussians": int(scene["means"].shape[0]), "views": 16,
           "tile": f"{best['tile'][0]}x{best['tile'][1]}", "raster_config": autotune.name(best),
           "autotune_ms": {k: round(v, 3) for k, v in tune.items()}}
    n = max(3, args.steps // 4)
    res = {}
    params = None
    # batched: one launch per stage for all views, captured; per_view: one
    # launch per stage and view, eager (the plain per-camera loop);
    # per_view_graph: the same per-view launches captured in a graph, which
    # separates the gain of batching from that of graph capture
    for label, mode, graph in (("batched", "batched", True), ("per_view", "per_view", False),
                               ("per_view_graph", "per_view", True)):
        step = R.TrainStep(scene, mode=mode, graph=graph, params=params, **kw).prepare()
        params = step.params
        for _ in range(2):
            step.run()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(n):
            step.run()
        b.record()
        torch.cuda.synchronize()
        step.check()
        ms = a.elapsed_time(b) / n
        res[label] = {"ms_per_step": ms, "Mpix_s": step.cams.n_pixels / (ms * 1e-3) / 1e6,
                      "launches_per_step": step.launches_per_step, "n_isect": step.n_isect()}
        del step
        torch.cuda.empty_cache()
    out.update(res)
    out["batched_speedup"] = res["per_view"]["ms_per_step"] / res["batched"]["ms_per_step"]
    out["batched_speedup_vs_per_view_graph"] = res["per_view_graph"]["ms_per_step"] / res["batched"]["ms_per_step"]
    return out


def e2e_measure(step, args, world, stream_params=False):
    """Same metric through the public API with host buffers (HostFedStep):
    per step, the camera and the target image are copied in from pinned host
    memory and the loss read back, the Gaussians staying resident in device
    memory as model state (like the weights of a network) and their gradients
    there for an optimizer on the device. With stream_params the parameters
    are copied in and the gradients read back as well, every step. The copies
    of neighbouring steps overlap the compute on two copy streams. Timed from
    an event before the first input copy to one after the last output copy."""
    import torch

    from paper_2606_11390_gb300 import renderer as R

    host_params = host_grads = None
    if stream_params:
        host_params = torch.empty_like(step.params.flat, device="cpu").pin_memory()
        host_params.copy_(step.params.flat)
        host_grads = [torch.empty_like(step.grads.flat, device="cpu").pin_memory() for _ in range(2)]
    host_target = torch.empty_like(step.target, device="cpu").pin_memory()
    host_target.copy_(step.target)
    host_cams = torch.from_numpy(step.cams.host.copy()).pin_memory()
    host_loss = [torch.empty(1, dtype=torch.float64).pin_memory() for _ in range(2)]
    fed = R.HostFedStep(step, stream_params=stream_params)
    n = max(3, args.steps // 2)
    grads_of = (lambda i: host_grads[i & 1]) if stream_params else (lambda i: None)  # noqa: E731
    for i in range(2):
        fed.run(host_params, host_target, host_cams, grads_of(i), host_loss[i & 1])
    fed.sync()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    a.record(fed.h2d)
    for i in range(n):
        fed.run(host_params, host_target, host_cams, grads_of(i), host_loss[i & 1])
    b.record(fed.d2h)
    fed.sync()
    wall = (time.perf_counter() - t0) / n
    ms = a.elapsed_time(b) / n
    bi = host_target.numel() * 4 + host_cams.numel() * 4
    bo = 8
    if stream_params:
        bi += host_params.numel() * 4
        bo += host_grads[0].numel() * 4
    moved = ("camera and target image in, loss out; Gaussians resident in device memory" if not stream_params else
             "parameters, camera and target image in, gradients and loss out")
    return {"value": world * step.cams.n_pixels / (ms * 1e-3) / 1e6, "unit": "Mpix/s", "ms_per_step": ms,
            "wall_ms_per_step": wall * 1e3, "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo, "copies": moved,
            "overlap": "inputs of step k+1 and outputs of step k copied while step k computes (HostFedStep)"}


if __name__ == "__main__":
    sys.exit(main())
