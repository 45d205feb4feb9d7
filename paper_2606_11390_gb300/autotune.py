"""Rasteriser autotuner for the training step.

For a workload (Gaussian count, view sizes, SH degree) it searches the
rasteriser's launch configuration:
- tile shape (8x8, 16x16, 32x16, 32x32) together with the pixels each thread
  owns (2 or 4, so threads per tile = tile area / pixels per thread; 8x8 tiles
  take 2 only);
- splats staged per shared-memory batch in the forward (64, 128, 256, 512);
- splats staged per shared-memory batch in the backward (64, 128, 256, 512).
The search is coordinate descent: every tile shape and pixels per thread at
the default batch sizes, then the forward batch at the best of those, then
the backward batch; at most 15 timed configurations instead of the 150 of
the full product. Each is timed as the whole captured training step. Every
configuration produces the same image (tests/test_gpu_raster_variants.py),
so the choice is about time only.

Results are cached in a JSON file (default ~/.cache/gs_gb300/autotune.json,
override with GS_AUTOTUNE_CACHE) under the GPU name, the workload signature,
the step mode and a digest of the library's sources, so a rebuilt kernel is
tuned afresh.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

TILES = ((16, 16), (8, 8), (32, 16), (32, 32))
BATCHES = (64, 128, 256, 512)


def _cache_path():
    return os.environ.get("GS_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "gs_gb300", "autotune.json"))


def signature(scene) -> str:
    sizes = np.asarray(scene["sizes"]).reshape(-1, 2)
    key = f"N={int(scene['means'].shape[0])};views={sizes.tolist()};deg={scene['cfg']['sh_degree']}"
    return hashlib.sha1(key.encode()).hexdigest()[:16]


def library_digest() -> str:
    """Digest of the CUDA library's sources and build flags."""
    from . import build

    return build._digest()[:16]


def _load():
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d):
    p = _cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1)
        os.replace(tmp, p)
    except OSError:
        pass


def name(c: dict) -> str:
    """Short label of a configuration, e.g. 32x16/4px/f128/b0 (0: default batch)."""
    return f"{c['tile'][0]}x{c['tile'][1]}/{c['ppt']}px/f{c['batch_fwd']}/b{c['batch_bwd']}"


def parse_name(label: str) -> dict:
    """The configuration a name() label describes, e.g. 32x16/4px/f128/b256."""
    t, px, f, b = label.split("/")
    tw, th = (int(x) for x in t.split("x"))
    if not px.endswith("px") or not f.startswith("f") or not b.startswith("b"):
        raise ValueError(f"bad rasteriser configuration {label!r}")
    return {"tile": (tw, th), "ppt": int(px[:-2]), "batch_fwd": int(f[1:]), "batch_bwd": int(b[1:])}


def tile_candidates(tiles=TILES):
    """(tile, pixels per thread) pairs at the default batch sizes."""
    out = []
    for t in tiles:
        for ppt in ((2,) if t == (8, 8) else (4, 2)):
            out.append({"tile": tuple(t), "ppt": ppt, "batch_fwd": 0, "batch_bwd": 0})
    return out


def threads_per_tile(c: dict) -> int:
    return c["tile"][0] * c["tile"][1] // c["ppt"]


def batch_supported(c: dict, dim: str, b: int) -> bool:
    """Whether the library has the variant: the backward's batch must fit a
    CTA's shared memory (b x (80 + 2 x warps) + 4 x warps bytes, with an
    opt-in above 48 KB up to 227 KB), which every batch size does on every
    tile; the forward's always does."""
    warps = threads_per_tile(c) // 32
    return dim != "batch_bwd" or b * (80 + 2 * warps) + 4 * warps <= 227 * 1024


def search(measure, tiles=TILES, batches=BATCHES):
    """Coordinate descent over the configuration space with measure(config) ->
    ms; returns (best config, {label: ms} of every configuration timed)."""
    times = {}

    def timed(c):
        k = name(c)
        if k not in times:
            times[k] = float(measure(c))
        return times[k]

    best = min(tile_candidates(tiles), key=timed)
    for dim in ("batch_fwd", "batch_bwd"):
        cands = [best] + [dict(best, **{dim: b}) for b in batches if batch_supported(best, dim, b)]
        best = min(cands, key=timed)
    return best, times


def step_kwargs(c: dict) -> dict:
    """TrainStep keyword arguments of a configuration."""
    return {"tile": tuple(c["tile"]), "raster_px": int(c["ppt"]), "raster_batch": (int(c["batch_fwd"]),
                                                                                   int(c["batch_bwd"]))}


def _time_step(scene, c, steps, mode, params):
    import torch

    from . import renderer as R

    step = R.TrainStep(scene, mode=mode, params=params, **step_kwargs(c)).prepare()
    for _ in range(2):
        step.run()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        step.run()
    b.record()
    torch.cuda.synchronize()
    step.check()
    ms = a.elapsed_time(b) / steps
    return ms, step.params


def best_config(scene, steps=3, use_cache=True, mode="batched", measure=None, gpu=None, digest=None):
    """Returns (config, {label: ms}) of the fastest rasteriser configuration
    for the workload. `measure`, `gpu` and `digest` default to timing the
    captured step on the current GPU with the built library."""
    if gpu is None:
        import torch

        gpu = torch.cuda.get_device_name()
    digest = digest if digest is not None else library_digest()
    key = f"{gpu}|{signature(scene)}|{mode}|{digest}"
    cache = _load() if use_cache else {}
    if key in cache:
        e = cache[key]
        c = dict(e["config"], tile=tuple(e["config"]["tile"]))
        return c, dict(e["ms"])
    if measure is None:
        state = {"params": None}

        def measure(c):
            ms, state["params"] = _time_step(scene, c, steps, mode, state["params"])
            return ms
    best, times = search(measure)
    if use_cache:
        cache = _load()
        cache[key] = {"config": dict(best, tile=list(best["tile"])), "ms": times}
        _store(cache)
    return best, times
