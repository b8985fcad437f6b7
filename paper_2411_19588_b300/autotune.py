"""Autotuner for the batched form: picks the pixel-tile shape (16x16, 8x32,
32x8) and the number of Gaussians staged per blend step (64, 128, 256) by
timing one forward + backward of the caller's batch with each candidate
(CUDA events, after a warm-up), and caches the winner per GPU model,
Gaussian count, SH degree and view set.

Cache file: $SPLASH_AUTOTUNE_CACHE, else ~/.cache/splash_b300/autotune.json.
"""
from __future__ import annotations

import hashlib
import json
import os

import torch

from . import render as R

TILES = ((16, 16), (8, 32), (32, 8))
BATCHES = (64, 128, 256)


def cache_path() -> str:
    return os.environ.get("SPLASH_AUTOTUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "splash_b300",
                                                                   "autotune.json")


def cache_key(params: dict, cams) -> str:
    sizes = ",".join(f"{c.width}x{c.height}" for c in cams)
    h = hashlib.sha1(sizes.encode()).hexdigest()[:12]
    return f"{torch.cuda.get_device_name()}|n={params['means'].shape[0]}|sh={params['sh_degree']}|views={len(cams)}:{h}"


def _time_candidate(params, medium, cams, upstream, tile, batch, reps):
    r = R.Renderer(tile=tile, batch=batch)
    b = R.Batch(r, cams)
    b.calibrate(params, medium)
    grads = {k: torch.empty_like(params[k]) for k in R.PARAM_NAMES}
    grads["medium"] = torch.empty_like(medium)
    b.forward(params, medium)
    b.backward(params, medium, upstream, grads)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        b.forward(params, medium)
        b.backward(params, medium, upstream, grads)
    e1.record()
    torch.cuda.synchronize()
    r.sync_status()
    ms = e0.elapsed_time(e1) / reps
    b.close()
    r.close()
    return ms


def autotune(params: dict, medium: torch.Tensor, cams, upstream=None, reps: int = 3, force: bool = False,
             path: str | None = None) -> dict:
    """Returns {"tile": (tw, th), "batch": nb, "ms": best, "table": {...}, "cached": bool}."""
    path = path or cache_path()
    key = cache_key(params, cams)
    cache = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if key in cache and not force:
        e = cache[key]
        return {"tile": tuple(e["tile"]), "batch": e["batch"], "ms": e["ms"], "table": e["table"], "cached": True}
    if upstream is None:
        upstream = [torch.full((3, c.height, c.width), 1e-3, device=medium.device) for c in cams]
    table = {}
    for tile in TILES:
        for nb in BATCHES:
            table[f"{tile[0]}x{tile[1]}/{nb}"] = _time_candidate(params, medium, cams, upstream, tile, nb, reps)
    best = min(table, key=table.get)
    tw, th = (int(x) for x in best.split("/")[0].split("x"))
    out = {"tile": (tw, th), "batch": int(best.split("/")[1]), "ms": table[best], "table": table}
    cache[key] = {"tile": [tw, th], "batch": out["batch"], "ms": out["ms"], "table": table}
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, path)
    out["cached"] = False
    return out
