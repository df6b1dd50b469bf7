"""Autotuner of the convolution variant per window radius.

For each radius S (and precision) it times the candidate kernels of the
convolution + combine stage -- FP32 FIR with 32 x 96 or 32 x 64 tiles, and
the BF16 tensor-core kernel when the precision allows it -- on a synthetic
512 x 512 colour image with K landmarks, and keeps the fastest.  Results are
cached in a JSON file (NYF_TUNE_CACHE, default ~/.cache/nyf_tune.json) keyed
by device name, radius, K and precision.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import _lib as L
from . import nyf

CACHE = os.environ.get("NYF_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache",
                                                      "nyf_tune.json"))


def candidates(S: int, precision: str):
    c = ["wide"] + (["narrow"] if S <= 16 else [])
    if precision == "bf16" and S <= 16:
        c.append("tensor")
    return c


def _load():
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _save(d):
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE, "w") as fh:
            json.dump(d, fh, indent=1, sort_keys=True)
    except OSError:
        pass


def time_variant(S: int, K: int, precision: str, tile: str, size=512, reps=3) -> float:
    """Milliseconds of the convolution + combine stage for one variant."""
    lib = L.load()
    g = torch.Generator(device="cpu").manual_seed(S * 131 + K)
    f = (torch.rand((size, size, 3), generator=g) * 255.0).cuda()
    P = nyf.Params(sigma_s=S / 3.0, sigma_r=30.0, K=K, S=S, kmeans_iters=2, precision=precision,
                   conv_tile=tile)
    ws = nyf.make_workspace(size, size, 3, 3, P)
    out = torch.empty_like(f)
    nyf.blf(f, P, out=out, ws=ws)                      # warm-up
    lib.nyf_set_timing(1)
    import ctypes as C
    buf = (C.c_float * 7)()
    best = math.inf
    for _ in range(reps):
        nyf.blf(f, P, out=out, ws=ws)
        lib.nyf_get_timing(buf, 7)
        best = min(best, buf[3])
    lib.nyf_set_timing(0)
    return best


def best_variant(S: int, K: int, precision: str, refresh=False) -> str:
    key = f"{torch.cuda.get_device_name()}|S={S}|K={K}|{precision}"
    cache = _load()
    if not refresh and key in cache:
        return cache[key]["best"]
    times = {t: time_variant(S, K, precision, t) for t in candidates(S, precision)}
    best = min(times, key=times.get)
    cache[key] = {"best": best, "ms": times}
    _save(cache)
    return best


def tune_batch(radii, K: int, precision: str, refresh=False):
    """Best variant for every distinct radius of a batch."""
    return {S: best_variant(S, K, precision, refresh) for S in sorted(set(radii))}
