"""Autotuner for the batched conv2d kernel: the tile shape per filter side is
chosen by measurement on the GPU it will run on (the profile-driven tuning
step of the paper's flow, Sec. 2).

For each filter side present in a batch, the images with that side are run
alone under every tile variant the kernel offers; the fastest variant (CUDA
events around `reps` runs after a warm-up, measured in the library by
pencil_tune) is set on the plan.  Results are cached
in a JSON file keyed by GPU name, SM count, CUDA driver version, library
version, storage dtype and filter side, so later processes on the same kind
of GPU and build skip the search; a record that cannot be read counts as
absent.  The cache path is $PENCIL_TUNE_CACHE, else
~/.cache/pencil/batch_tune.json.
"""
from __future__ import annotations

import json
import os

from . import _binding as b


def cache_path() -> str:
    return os.environ.get("PENCIL_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "pencil", "batch_tune.json")


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _key(dtype: int, ks: int) -> str:
    name, sms, drv = b.pencil_device_info()
    return (f"{name}|sm{sms}|drv{drv}|lib{b.pencil_version()}|"
            f"{'f16' if dtype == b.PENCIL_F16 else 'f32'}|k{ks}")


def _variant(rec):
    """The variant of a cache record, or None when the record is malformed."""
    try:
        v = int(rec["variant"])
    except (KeyError, TypeError, ValueError):
        return None
    return v if 0 <= v < b.PENCIL_BATCH_VARIANTS else None


def autotune(plan, dtype: int, items, reps: int = 5, use_cache: bool = True, path: str | None = None,
             stream=None):
    """Choose and set the tile variant for every filter side in `items`
    ((in, out, k, h, w, ks) tuples, device tensors).  The search, where one
    runs, is timed on `stream` (default: the current CUDA stream).
    Returns {ks: (variant, source)}."""
    path = path or cache_path()
    cache = _load(path) if use_cache else {}
    if not isinstance(cache, dict):
        cache = {}
    chosen = {}
    todo = []
    for ks in sorted({it[5] for it in items}):
        v = _variant(cache.get(_key(dtype, ks)))
        if v is not None:
            b.pencil_batch_set_variant(plan, ks, v)
            chosen[ks] = (v, "cache")
        else:
            todo.append(ks)
    if todo:
        # the search itself runs in the library (pencil_tune: CUDA events per
        # variant and side, the fastest kept on the plan)
        if stream is None:
            import torch
            stream = torch.cuda.current_stream()
        sub = b.make_images([it for it in items if it[5] in todo])
        for ks, v in b.pencil_tune(plan, sub, reps, stream).items():
            chosen[ks] = (v, "measured")
            cache[_key(dtype, ks)] = {"variant": v, "reps": reps}
    if use_cache and any(src == "measured" for _, src in chosen.values()):
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        tmp = f"{path}.{os.getpid()}.tmp"  # one per process; the rename is atomic
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    return chosen


def cached_variants(dtype: int, path: str | None = None) -> dict:
    """{ks: variant} recorded for this GPU and dtype (sides never tuned are absent)."""
    cache = _load(path or cache_path())
    if not isinstance(cache, dict):
        return {}
    out = {}
    for ks in range(1, 16, 2):
        v = _variant(cache.get(_key(dtype, ks)))
        if v is not None:
            out[ks] = v
    return out
