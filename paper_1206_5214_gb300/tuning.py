"""A JSON cache of autotuned hop block shapes, keyed by GPU name and problem shape.

``tuned(ctx, key_parts, prec, nrhs, path)`` looks the key up in the cache file,
applies a cached value with mdwf_set_tuning, or runs mdwf_autotune once and
stores the result. The cache path defaults to $MDWF_TUNE_CACHE or
~/.cache/mdwf/tune.json.
"""
from __future__ import annotations

import json
import os

from . import mdwf_autotune, mdwf_set_tuning

PREC = {0: "f64", 1: "f32", 2: "f16n"}


def default_path() -> str:
    return os.environ.get("MDWF_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "mdwf", "tune.json")


def cache_key(gpu_name: str, dims, Ls: int, prec: int, nrhs: int) -> str:
    return f"{gpu_name}|{'x'.join(str(int(d)) for d in dims)}|Ls{int(Ls)}|{PREC[int(prec)]}|nrhs{int(nrhs)}"


def load_cache(path: str | None = None) -> dict:
    path = path or default_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str | None = None) -> None:
    path = path or default_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tuned(ctx, gpu_name: str, dims, Ls: int, prec: int, nrhs: int = 1, path: str | None = None) -> int:
    """Apply the cached block shape for this key, or tune and cache it. Returns sites per block."""
    cache = load_cache(path)
    key = cache_key(gpu_name, dims, Ls, prec, nrhs)
    if key in cache:
        sb = int(cache[key])
        mdwf_set_tuning(ctx, prec, nrhs, sb)
        return sb
    sb = mdwf_autotune(ctx, prec, nrhs)
    cache[key] = sb
    save_cache(cache, path)
    return sb
