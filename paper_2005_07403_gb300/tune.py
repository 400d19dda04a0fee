"""Persistent cache of the autotuner's launch shapes.

The tuner itself is native (svd2_autotune_fwd / svd2_multi_autotune in the
library); this module remembers its winners per (GPU name, form, batch-size
bucket) in a JSON file next to the built library, and re-applies them.
"""
from __future__ import annotations

import json
import math
import os
import threading

import torch

from . import build as _build
from . import svd2 as S

CACHE = os.path.join(_build.BUILD, "tune_cache.json")
_lock = threading.Lock()


def _key(kind: str, n: int) -> str:
    name = torch.cuda.get_device_name()
    return f"{name}|{kind}|2^{int(math.log2(max(n, 1)))}"


def _load() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d: dict):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def tune(A: torch.Tensor, out: S.Svd2Result | None = None, reps: int = 5,
         use_cache: bool = True, form: str = "plain") -> dict:
    """Launch shape for A's form and size: from the cache, else measured by the
    native tuner on A (and cached).  The shape is applied with set_launch.
    ``form``: "plain" or "tan64" (the FP32 form with the FP64 tangent step,
    which has its own launch shape)."""
    rows, n = A.shape
    kind = S._kind(rows, A.dtype) + ("_tan64" if form == "tan64" else "")
    key = _key(kind, n)
    with _lock:
        cache = _load()
        hit = cache.get(key) if use_cache else None
    if hit is not None:
        S.set_launch(kind, hit["block"], hit["mpt"], hit["unroll"], hit["waves"])
        return dict(hit, cached=True)
    best = S.autotune_fwd(A, out, reps, form=form)
    with _lock:
        cache = _load()
        cache[key] = best
        _store(cache)
    return dict(best, cached=False)
