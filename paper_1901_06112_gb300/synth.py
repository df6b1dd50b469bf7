"""Seeded synthetic workloads shaped like the paper's experiments.

The paper evaluates on colour photographs (Kodak) and hyperspectral cubes
(Section IV).  Neither dataset is available here, so these generators produce
images with the same shapes, value ranges and structure: piecewise-constant or
piecewise-smooth colour regions (Voronoi cells) with noise for the colour
bilateral / nonlocal-means workloads, and linear mixtures of smooth spectra for
the hyperspectral one.

This module holds none of the filter's arithmetic: it only draws inputs.  It
is the one module shared by the CUDA path's tests/benchmark and the CPU oracle.
Every generator draws from ``numpy.random.default_rng(seed)`` (PCG64) in float64
and casts to float32 at the end.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 1901_06112


@dataclasses.dataclass
class Workload:
    """One filtering problem: image, guide kind and filter parameters."""

    name: str
    f: np.ndarray                # H x W x n float32, values in [0, R]
    R: float                     # range bound of the image (Section II: f maps to [0, R]^n)
    sigma_s: float               # spatial Gaussian std (paper's sigma); ignored for a box
    sigma_r: float               # range Gaussian std (paper's theta)
    K: int                       # number of landmarks m0
    spatial: str = "gaussian"    # "gaussian" or "box"
    S: int = 0                   # window radius; 0 -> ceil(3 sigma_s)
    patch_radius: int = 0        # >0: nonlocal means with (2r+1)^2 x n patches as guide
    sample_frac: float = 1.0     # fraction of pixels k-means clusters (NLM: 0.01)
    kmeans_iters: int = 10
    seed: int = 0
    pca_dim: int = 0             # >0: PCA-NLM, the patch guide projected on q principal directions

    @property
    def H(self) -> int:
        return self.f.shape[0]

    @property
    def W(self) -> int:
        return self.f.shape[1]

    @property
    def n(self) -> int:
        return self.f.shape[2]

    @property
    def radius(self) -> int:
        return self.S if self.S > 0 else int(math.ceil(3.0 * self.sigma_s))


def _voronoi_labels(rng, H, W, cells):
    """Nearest-seed labels of every pixel for `cells` seeds drawn uniformly in the image."""
    from scipy.spatial import cKDTree

    seeds = np.stack([rng.uniform(0, H, cells), rng.uniform(0, W, cells)], axis=1)
    yy, xx = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    _, lab = cKDTree(seeds).query(np.stack([yy.ravel(), xx.ravel()], axis=1))
    return lab.reshape(H, W), seeds, yy, xx


def voronoi_colour(H, W, cells, noise, seed, shading=0.0, ramp=0.0):
    """Colour image of `cells` Voronoi regions with U[0,255] RGB per cell.

    shading > 0 adds amplitude * sin(2 pi x / lx + a) * sin(2 pi y / ly + b) with
    lx, ly ~ U[200, 600] px to every channel; ramp > 0 adds a per-cell, per-channel
    linear ramp of slope U[-ramp, ramp] per pixel about the cell's seed.  Gaussian
    noise of std `noise` is added last and the result clipped to [0, 255].
    """
    rng = np.random.default_rng(seed)
    lab, seeds, yy, xx = _voronoi_labels(rng, H, W, cells)
    colours = rng.uniform(0.0, 255.0, size=(cells, 3))
    img = colours[lab].astype(np.float64)
    if ramp > 0:
        g = rng.uniform(-ramp, ramp, size=(cells, 2, 3))
        dy = (yy - seeds[lab, 0])[..., None]
        dx = (xx - seeds[lab, 1])[..., None]
        img += g[lab, 0, :] * dy + g[lab, 1, :] * dx
    if shading > 0:
        lx, ly = rng.uniform(200.0, 600.0, size=2)
        a, b = rng.uniform(0.0, 2 * np.pi, size=2)
        sh = shading * np.sin(2 * np.pi * xx / lx + a) * np.sin(2 * np.pi * yy / ly + b)
        img += sh[..., None]
    img += rng.normal(0.0, noise, size=img.shape)
    return np.clip(img, 0.0, 255.0).astype(np.float32)


def hyperspectral(H, W, bands, endmembers, length_scale, noise, seed):
    """Linear mixture of smooth random spectra with Dirichlet(1) abundances.

    Each endmember spectrum is a sum of three Gaussian bumps over the band index,
    rescaled to [0.05, 0.95].  Abundances come from `endmembers` Gaussian random
    fields (white noise blurred with a Gaussian of std `length_scale` px, scaled to
    unit variance): U = Phi(z) is uniform, E = -log U is Exp(1), and E / sum(E) is
    Dirichlet(1) at every pixel.  Values are clipped to [0, 1].
    """
    from scipy.ndimage import gaussian_filter
    from scipy.special import ndtr

    rng = np.random.default_rng(seed)
    t = np.arange(bands, dtype=np.float64)
    spectra = np.zeros((endmembers, bands))
    for j in range(endmembers):
        for _ in range(3):
            c = rng.uniform(0, bands - 1)
            w = rng.uniform(0.1, 0.4) * bands
            h = rng.uniform(0.2, 1.0)
            spectra[j] += h * np.exp(-0.5 * ((t - c) / w) ** 2)
        lo, hi = spectra[j].min(), spectra[j].max()
        spectra[j] = 0.05 + 0.9 * (spectra[j] - lo) / max(hi - lo, 1e-12)
    E = np.empty((H, W, endmembers))
    for j in range(endmembers):
        z = gaussian_filter(rng.normal(size=(H, W)), length_scale, mode="wrap")
        z = (z - z.mean()) / z.std()
        u = np.clip(ndtr(z), 1e-12, 1.0)
        E[..., j] = -np.log(u)
    a = E / E.sum(axis=2, keepdims=True)
    img = a @ spectra + rng.normal(0.0, noise, size=(H, W, bands))
    return np.clip(img, 0.0, 1.0).astype(np.float32)


# ---------------------------------------------------------------------------
# The five workloads.  Sizes are (H, W); the prose sizes "W x H" are converted.
# ---------------------------------------------------------------------------

def colour_blf_small(seed=SEED_BASE + 1) -> Workload:
    """256 x 256 x 3, 40 cells, noise 10; sigma_s 3 (19 x 19), sigma_r 30, K 8."""
    f = voronoi_colour(256, 256, 40, 10.0, seed)
    return Workload("colour_blf_256x256_K8", f, 255.0, 3.0, 30.0, 8, seed=seed)


def colour_blf_hd(seed=SEED_BASE + 2) -> Workload:
    """1920 x 1080 x 3 (W x H), 400 cells, shading 20, noise 15; sigma_s 5 (31 x 31), sigma_r 40, K 32."""
    f = voronoi_colour(1080, 1920, 400, 15.0, seed, shading=20.0)
    return Workload("colour_blf_1920x1080_K32", f, 255.0, 5.0, 40.0, 32, seed=seed)


def hyperspectral_blf(seed=SEED_BASE + 3) -> Workload:
    """512 x 512 x 31 in [0, 1], 6 endmembers, noise 0.02; sigma_s 4 (25 x 25), sigma_r 0.15, K 64."""
    f = hyperspectral(512, 512, 31, 6, 40.0, 0.02, seed)
    return Workload("hyperspectral_blf_512x512x31_K64", f, 1.0, 4.0, 0.15, 64, seed=seed)


def colour_nlm(seed=SEED_BASE + 4) -> Workload:
    """768 x 512 x 3 (W x H), 200 piecewise-smooth cells, noise 20; 5x5x3 patches, 21 x 21 box, K 32."""
    f = voronoi_colour(512, 768, 200, 20.0, seed, ramp=0.1)
    return Workload("colour_nlm_768x512_K32", f, 255.0, 0.0, 20.0 * math.sqrt(75.0), 32,
                    spatial="box", S=10, patch_radius=2, sample_frac=0.01, seed=seed)


def colour_pca_nlm(seed=SEED_BASE + 4) -> Workload:
    """PCA-NLM at the paper's parameters (Sec. IV): the 768 x 512 colour NLM image (noise 20),
    7x7x3 patches (rho 147) projected on q = 25 principal directions, 21 x 21 box (S = 10),
    K = 31 landmarks from k-means on a 1 % subsample, theta = 3 x the noise level of the
    distance between two patches' PCA coordinates: 3 sigma sqrt(2 q) = 424.3."""
    f = voronoi_colour(512, 768, 200, 20.0, seed, ramp=0.1)
    return Workload("colour_pca_nlm_768x512_q25_K31", f, 255.0, 0.0, 3.0 * 20.0 * math.sqrt(50.0),
                    31, spatial="box", S=10, patch_radius=3, sample_frac=0.01, seed=seed, pca_dim=25)


def batched_blf(count=64, seed=SEED_BASE + 5, side_lo=128, side_hi=1024):
    """`count` colour images generated like the 256 x 256 case with sides U{side_lo..side_hi}.

    Per image: sigma_s ~ U[2, 8], sigma_r ~ U[10, 60], K 16.  Image b uses seed
    ``seed + 1000 + b``; the sizes and parameters come from ``seed``.
    """
    rng = np.random.default_rng(seed)
    Hs = rng.integers(side_lo, side_hi + 1, size=count)
    Ws = rng.integers(side_lo, side_hi + 1, size=count)
    ss = rng.uniform(2.0, 8.0, size=count)
    sr = rng.uniform(10.0, 60.0, size=count)
    out = []
    for b in range(count):
        f = voronoi_colour(int(Hs[b]), int(Ws[b]), 40, 10.0, seed + 1000 + b)
        out.append(Workload(f"batched_{b}", f, 255.0, float(ss[b]), float(sr[b]), 16,
                            seed=seed + 1000 + b))
    return out


def few_colour(H, W, colours, seed):
    """Image whose pixels take only the given colours (rows of `colours`), in random blocks."""
    rng = np.random.default_rng(seed)
    k = colours.shape[0]
    lab = rng.integers(0, k, size=(max(1, H // 4) + 1, max(1, W // 4) + 1))
    lab = np.kron(lab, np.ones((4, 4), dtype=np.int64))[:H, :W]
    lab.ravel()[:k] = np.arange(k)        # every colour occurs at least once
    return colours[lab].astype(np.float32)


def random_image(H, W, n, seed, R=255.0):
    """I.i.d. uniform [0, R] pixels (no structure): the hardest case for low rank."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, R, size=(H, W, n)).astype(np.float32)


def sample_indices(N, count, seed):
    """Seeded distinct pixel indices (used to pick parity sample positions)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(N, size=min(count, N), replace=False)).astype(np.int64)
