"""Autotuner for the tensor-core render kernels.

The kernels' tile is fixed at 16x16 pixels (two 128-pixel halves, one TMEM
lane per pixel) and their Gaussian batch at 64 (the K of one tcgen05.mma,
two groups of 32 = one per warp lane).  What varies with the workload is the
D split: how many feature columns one CTA owns (DN = 64..512 forward,
64..256 backward).  A wider slice repeats the per-(pixel, Gaussian) alpha
work fewer times; a narrower one gives more CTAs and smaller shared-memory
stages.  The tuner times each candidate on the caller's own prepared scene
with CUDA events and keeps the fastest per workload key, in memory and in a
JSON file (FHGS_AUTOTUNE_CACHE, default ~/.cache/fhgs/autotune.json).
"""
from __future__ import annotations

import json
import os

import torch

from . import api

FWD_SPLITS = (64, 128, 256, 512)
BWD_SPLITS = (64, 128, 256)

_memory: dict = {}


def cache_path() -> str:
    return os.environ.get("FHGS_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "fhgs", "autotune.json"))


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key: str, val) -> None:
    _memory[key] = val
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        d = _load()
        d[key] = val
        tmp = path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass  # an unwritable cache only costs a re-tune


def workload_key(dev: torch.device, n: int, cams, D: int, sh_degree: int) -> str:
    """Device name, Gaussians and pixels (rounded to powers of two), cameras,
    D and SH degree."""
    P = sum(int(c["width"]) * int(c["height"]) for c in cams)
    p2 = lambda v: 1 << max(0, int(v) - 1).bit_length()  # noqa: E731
    name = torch.cuda.get_device_name(dev).replace(" ", "_")
    return f"{name}|n{p2(n)}|p{p2(P)}|c{len(cams)}|d{D}|sh{sh_degree}"


def _time_ms(fn, reps: int) -> float:
    fn()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune_splits(rast: api.Rasterizer, st: dict, features: torch.Tensor, grad_rgb, grad_feat, cams,
                reps: int = 3, use_cache: bool = True) -> dict:
    """Pick the forward and backward D split for this workload, set them on
    `rast` and return {"fwd": DN, "bwd": DN, "times_ms": {...}}.  `st` is a
    prepared scene (rast.prepare) whose forward has run."""
    D = int(features.shape[1])
    key = workload_key(rast.dev, st["n"], cams, D, rast.params.sh_degree)
    if use_cache:
        hit = _memory.get(key) or _load().get(key)
        if hit:
            rast.set_splits(hit["fwd"], hit["bwd"])
            return dict(hit, cached=True)
    times = {}
    fwd_c = [dn for dn in FWD_SPLITS if D % dn == 0]
    bwd_c = [dn for dn in BWD_SPLITS if D % dn == 0]
    if not fwd_c or not bwd_c:
        raise ValueError(f"no tensor-core split divides D={D}")
    for dn in fwd_c:
        rast.set_splits(dn, bwd_c[-1])
        times[f"fwd{dn}"] = _time_ms(lambda: rast.forward(st, features), reps)
    for dn in bwd_c:
        rast.set_splits(fwd_c[-1], dn)
        times[f"bwd{dn}"] = _time_ms(lambda: rast.backward(st, grad_rgb, grad_feat), reps)
    best_f = min(fwd_c, key=lambda dn: times[f"fwd{dn}"])
    best_b = min(bwd_c, key=lambda dn: times[f"bwd{dn}"])
    rast.set_splits(best_f, best_b)
    rast.forward(st, features)  # leave st holding this split's forward outputs
    val = {"fwd": best_f, "bwd": best_b, "times_ms": {k: round(v, 4) for k, v in times.items()}}
    _store(key, val)
    return dict(val, cached=False)
