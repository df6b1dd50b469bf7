"""Autotuner of the convolution variant per window radius and image size.

For each radius S, image-size class and precision it times the candidate
kernels of the convolution + combine stage -- FP32 FIR with 32 x 96 or
32 x 64 tiles, and the BF16 tensor-core kernel when the precision allows it --
on a synthetic square colour image of the class's side (256, 512 or 1024
pixels: the tile shapes trade halo work against the last wave's idle SMs, which
depends on the image size) with K landmarks, and keeps the fastest.  Results
are cached in a JSON file (NYF_TUNE_CACHE, default ~/.cache/nyf_tune.json)
keyed by device name, radius, size class, K and precision.
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


SIZE_CLASSES = (256, 512, 1024)


def size_class(H: int, W: int) -> int:
    """The tuning side for an H x W image: the class nearest to sqrt(H W) on a log scale."""
    side = math.sqrt(max(1, H * W))
    return min(SIZE_CLASSES, key=lambda c: abs(math.log(side / c)))


def best_variant(S: int, K: int, precision: str, size: int = 512, refresh=False) -> str:
    cands = candidates(S, precision)
    if len(cands) == 1:
        return cands[0]
    key = f"{torch.cuda.get_device_name()}|S={S}|size={size}|K={K}|{precision}"
    cache = _load()
    if not refresh and key in cache:
        return cache[key]["best"]
    times = {t: time_variant(S, K, precision, t, size=size) for t in cands}
    best = min(times, key=times.get)
    cache[key] = {"best": best, "ms": times}
    _save(cache)
    return best


def tune_batch(radii, K: int, precision: str, refresh=False):
    """Best variant for every distinct radius of a batch (512-pixel class)."""
    return {S: best_variant(S, K, precision, 512, refresh) for S in sorted(set(radii))}


def tune_images(shapes, radii, K: int, precision: str, refresh=False):
    """Best variant for every image of a batch: by its radius and size class."""
    return [best_variant(S, K, precision, size_class(H, W), refresh)
            for (H, W), S in zip(shapes, radii)]
