"""Autotuner for the launch shape of the whole path.

Searches the tile shape (8x8, 16x16, 32x8), the number of splats staged in
shared memory per round (32 ... 256) and the pixels per blend thread (1, 2, 4)
by timing complete passes (projection, binning, blending) on the caller's own
scene and cameras with CUDA events. The tile shape changes the binning too,
so every candidate is timed end to end. Results are cached in a JSON file,
keyed by GPU name, kernel kind, cull mode, splat count, launch mode and the
camera resolutions; a cached key is returned without timing anything.

The search is staged: tile shape x pixels per thread at the largest batch,
then the batch depth for the winner.
"""
from __future__ import annotations

import json
import os

import torch

from . import api
from .render import Rasterizer

TILES = ((16, 16), (8, 8), (32, 8), (32, 16))
BATCHES = (256, 128, 64, 32)
PPTS = (1, 2, 4)
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "gs_b300_autotune.json")


def _key(cams, kind, cull, P, persistent, last=False):
    res = sorted((int(c["width"]), int(c["height"])) for c in cams)
    counts = {}
    for r in res:
        counts[r] = counts.get(r, 0) + 1
    rs = ",".join(f"{w}x{h}*{n}" for (w, h), n in sorted(counts.items()))
    return f"{torch.cuda.get_device_name()}|{kind}|{cull}|P={P}|persistent={int(persistent)}|last={int(last)}|{rs}"


def _time(cams, kind, cull, sc, P, over, persistent, steps, last=False):
    """ms per pass, or inf for a candidate this workload cannot run (e.g.
    small tiles pushing the overlap count past the binning's 2^30 limit)."""
    cfg = api.make_config(kind, cull, **over)
    try:
        R = Rasterizer(cams, cfg, P, persistent=persistent, last=last)
        R.forward(sc, n_eval=False)
    except RuntimeError:
        torch.cuda.synchronize()
        return float("inf")
    torch.cuda.synchronize()
    R.run_async(sc)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        R.run_async(sc)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    del R
    return ms


def autotune(cams, kind: str, cull: str, sc: dict, P: int, persistent: bool = False,
             steps: int = 5, cache: str | None = DEFAULT_CACHE, verbose: bool = False,
             last: bool = False) -> dict:
    """Best {"tile", "batch", "px_per_thread"} for this workload, plus the
    timings that chose it (ms per pass). last: tune the blend that keeps each
    pixel's last contributor (a training forward) instead of the image-only
    one (a serving render)."""
    key = _key(cams, kind, cull, P, persistent, last)
    store = {}
    if cache and os.path.exists(cache):
        try:
            store = json.load(open(cache))
        except (OSError, ValueError):
            store = {}
        if key in store:
            return store[key]
    trials = {}
    for tile in TILES:
        for ppt in PPTS:
            over = {"tile": tile, "px_per_thread": ppt, "batch": BATCHES[0]}
            trials[f"{tile[0]}x{tile[1]}/b{BATCHES[0]}/p{ppt}"] = (
                _time(cams, kind, cull, sc, P, over, persistent, steps, last), over)
    best_name = min(trials, key=lambda k: trials[k][0])
    best = dict(trials[best_name][1])
    for b in BATCHES[1:]:
        over = dict(best, batch=b)
        trials[f"{over['tile'][0]}x{over['tile'][1]}/b{b}/p{over['px_per_thread']}"] = (
            _time(cams, kind, cull, sc, P, over, persistent, steps, last), over)
    best_name = min(trials, key=lambda k: trials[k][0])
    best_over = trials[best_name][1]
    result = {"tile": list(best_over["tile"]), "batch": int(best_over["batch"]),
              "px_per_thread": int(best_over["px_per_thread"]), "ms": trials[best_name][0],
              "trials_ms": {k: (v[0] if v[0] != float("inf") else None) for k, v in trials.items()}}
    if result["ms"] == float("inf"):
        raise RuntimeError("no candidate launch shape can run this workload")
    if verbose:
        print(json.dumps(result))
    if cache:
        store[key] = result
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        tmp = cache + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(store, f, indent=1)
        os.replace(tmp, cache)
    return result


def config_overrides(result: dict) -> dict:
    """Config overrides (for api.make_config) of an autotune result."""
    return {"tile": tuple(result["tile"]), "batch": result["batch"],
            "px_per_thread": result["px_per_thread"]}
