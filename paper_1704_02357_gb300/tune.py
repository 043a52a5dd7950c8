"""Autotune cache: the knob settings pspec_autotune picked, per GPU and plan shape, in JSON.

Key: GPU name, mesh side, precision, l_max, window, interlacing. The search itself runs in
libpspec (pspec_autotune); this module only stores and reapplies its answer.
"""
from __future__ import annotations

import json
import os
from typing import Optional

DEFAULT_PATH = os.environ.get("PSPEC_TUNING_CACHE",
                              os.path.join(os.path.expanduser("~"), ".cache", "pspec_gb300", "tuning.json"))


def key_for(est) -> str:
    import torch
    p = est.params
    name = torch.cuda.get_device_name(est.device).replace(" ", "_")
    prec = {0: "fp32", 1: "fp64", 2: "fp32_plain"}.get(p.precision, str(p.precision))
    return f"{name}|N{p.nmesh}|{prec}|l{p.ell_max}|w{p.window}|i{p.interlaced}"


def load_cache(path: str = DEFAULT_PATH) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str = DEFAULT_PATH) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tuned(est, data_pos, randoms_pos, ells, k_edges, path: Optional[str] = DEFAULT_PATH, reps: int = 2,
          keep_exact_paint: bool = True, **cat) -> dict:
    """Apply the cached tuning for this estimator's key, or run the autotuner and cache it.

    With `keep_exact_paint` (the default) a context that holds the tile-paint buffers keeps the
    exact tile-binned paint even where the search found the direct paint faster: the direct
    paint adds FP32 atomics in an order that changes from run to run, so it is not the same
    result at another speed."""
    key = key_for(est)
    cache = load_cache(path) if path else {}
    if key in cache:
        est.set_tuning(**cache[key])
        return dict(cache[key], cached=True)
    best = est.autotune(data_pos, randoms_pos, ells, k_edges, reps=reps, **cat)
    has_tiles = int(getattr(getattr(est, "params", None), "max_particles", 0) or 0) > 0
    if keep_exact_paint and has_tiles and best.get("paint_binned") == 0:
        best = dict(best, paint_binned=1)
        est.set_tuning(**best)
    if path:
        cache[key] = best
        save_cache(cache, path)
    return dict(best, cached=False)
