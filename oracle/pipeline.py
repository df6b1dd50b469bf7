"""The whole method as one call: guide, k-means landmarks, Algorithm 1.

BLF: the guide is the image (or a given joint guide); k-means runs on every
pixel.  NLM: the guide is the patch image (``oracle.guide``); k-means runs on
a seeded subsample of round(frac * N) pixels (``rng.stratified_sample``) and
the spatial kernel is a box.  The initial centroids are the rows picked by
``rng.distinct_indices(seed, m0, m)`` of the clustered list.

``landmark_dtype=np.float32`` rounds the k-means centroids to float32 before
Algorithm 1, which is how they are exchanged with the CUDA path.
"""
from __future__ import annotations

import numpy as np

from . import guide as _guide
from . import kernels as _k
from . import kmeans as _km
from . import nystrom as _ny
from . import rng as _rng


def landmarks(X: np.ndarray, K: int, iters: int, seed: int):
    """k-means landmarks of the rows of X from the seeded initial rows."""
    init_idx = _rng.distinct_indices(seed, K, X.shape[0])
    mu, c, e, hist = _km.kmeans(X, np.asarray(X, np.float64)[init_idx], iters)
    return mu, dict(init_idx=init_idx, labels=c, e=e, e_hist=hist)


def taps_for(spatial: str, sigma_s: float, S: int) -> np.ndarray:
    if spatial == "box":
        return _k.box_taps(S)
    return _k.gaussian_taps(sigma_s, S)


def blf(f, sigma_s, sigma_r, K, iters=10, seed=0, tau=1e-7, S=0, guide=None,
        landmark_dtype=np.float64, mu=None):
    """Nystrom bilateral filter of f (joint when `guide` is given)."""
    f = np.asarray(f, np.float64)
    p = f if guide is None else np.asarray(guide, np.float64)
    S = S if S > 0 else _k.window_radius(sigma_s)
    info = {}
    if mu is None:
        mu, info = landmarks(p.reshape(-1, p.shape[2]), K, iters, seed)
    mu = np.asarray(mu, landmark_dtype).astype(np.float64)
    taps = _k.gaussian_taps(sigma_s, S)
    g = _ny.nystrom_filter(f, p, mu, sigma_r, taps, tau)
    return g, mu, info


def nlm_sample_rows(f, patch_radius, frac, seed):
    """Patch vectors of the seeded k-means subsample (rows of the patch guide)."""
    p = _guide.patch_guide(f, patch_radius)
    H, W = p.shape[:2]
    Ns = _rng.subsample_size(H * W, frac)
    idx = _rng.stratified_sample(seed, Ns, H * W)
    return p.reshape(H * W, -1)[idx], idx, p


def nlm(f, sigma_r, K, S=10, patch_radius=2, frac=0.01, iters=10, seed=0, tau=1e-7,
        landmark_dtype=np.float64, mu=None):
    """Nystrom nonlocal means: patch guide, box window of radius S."""
    f = np.asarray(f, np.float64)
    X, idx, p = nlm_sample_rows(f, patch_radius, frac, seed)
    info = dict(sample_idx=idx)
    if mu is None:
        mu, kinfo = landmarks(X, K, iters, seed)
        info.update(kinfo)
    mu = np.asarray(mu, landmark_dtype).astype(np.float64)
    g = _ny.nystrom_filter(f, p, mu, sigma_r, _k.box_taps(S), tau)
    return g, mu, info
