"""Cache of autotuned walk/build parameters.

nbody_autotune (in the CUDA library) times the candidates; this module only
remembers the winners in a JSON file keyed by the device, the problem size
bucket (nearest power of two of N), the number of systems bucket and
delta_acc, so later runs of the same shape skip the search.
"""
from __future__ import annotations

import json
import math
import os
import tempfile

TUNED_FIELDS = ("leaf_cap", "group_size", "ipl", "list_depth", "warps_per_block")


def cache_key(device: str, n: int, nsys: int, delta_acc: float) -> str:
    nb_ = int(round(math.log2(max(n, 1))))
    sb = int(round(math.log2(max(nsys, 1))))
    return f"{device}|n=2^{nb_}|nsys=2^{sb}|dacc={delta_acc:.6g}"


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(path: str, cache: dict) -> None:
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=d, suffix=".tmp")
    with os.fdopen(fd, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apply(cfg, entry: dict):
    for k in TUNED_FIELDS:
        if k in entry:
            setattr(cfg, k, int(entry[k]))
    return cfg


def tuned_config(ctx, device: str, offsets, eps_sys, x, y, z, m, a_old=None, space=None,
                 cache_path: str | None = None, tuner=None):
    """Return the tuned Config for this shape, from the cache or by running
    the autotuner (then stored).  The context is left configured with it."""
    from . import nbody as nbm
    tuner = tuner or nbm.nbody_autotune
    n = int(offsets[-1])
    cfg = nbm.nbody_get_config(ctx)
    key = cache_key(device, n, len(offsets) - 1, cfg.delta_acc)
    cache = load_cache(cache_path) if cache_path else {}
    if key in cache:
        cfg = apply(cfg, cache[key])
        nbm.nbody_set_config(ctx, cfg)
        return cfg, cache[key], True
    best, ms, tried = tuner(ctx, offsets, eps_sys, x, y, z, m, a_old, space)
    entry = {k: int(getattr(best, k)) for k in TUNED_FIELDS}
    entry.update(ms=ms, tried=tried)
    if cache_path:
        cache[key] = entry
        save_cache(cache_path, cache)
    return best, entry, False
