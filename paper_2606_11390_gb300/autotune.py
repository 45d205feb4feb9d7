"""Tile-size autotuner for the batched step.

For a workload (Gaussian count, view sizes, SH degree) it times the captured
training step with each supported tile shape (8x8, 16x16, 32x16, 32x32) and
keeps the fastest. Results are cached per GPU name and workload signature in a JSON file
(default ~/.cache/gs_gb300/autotune.json, override with GS_AUTOTUNE_CACHE).
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

TILES = ((16, 16), (8, 8), (32, 16), (32, 32))


def _cache_path():
    return os.environ.get("GS_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "gs_gb300", "autotune.json"))


def signature(scene) -> str:
    sizes = np.asarray(scene["sizes"]).reshape(-1, 2)
    key = f"N={int(scene['means'].shape[0])};views={sizes.tolist()};deg={scene['cfg']['sh_degree']}"
    return hashlib.sha1(key.encode()).hexdigest()[:16]


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


def best_tile(scene, steps=3, use_cache=True, candidates=TILES, mode="batched"):
    """Returns ((tw, th), {tile: ms}) for the fastest tile shape."""
    import torch

    from . import renderer as R

    gpu = torch.cuda.get_device_name()
    key = f"{gpu}|{signature(scene)}|{mode}"
    cache = _load() if use_cache else {}
    if key in cache:
        t = tuple(cache[key]["tile"])
        return t, {tuple(map(int, k.split("x"))): v for k, v in cache[key]["ms"].items()}
    times = {}
    params = None
    for tile in candidates:
        step = R.TrainStep(scene, mode=mode, tile=tile, params=params).prepare()
        params = step.params
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
        times[tile] = a.elapsed_time(b) / steps
        del step
    best = min(times, key=times.get)
    cache[key] = {"tile": list(best), "ms": {f"{t[0]}x{t[1]}": v for t, v in times.items()}}
    if use_cache:
        _store(cache)
    return best, times
