"""Guide images p: Omega -> R^rho.

For bilateral filtering the guide is the image itself (Sec. II: f and p are
identical for standard BLF, differ for joint BLF).  For nonlocal means the
guide at x is the colour patch of radius r around x, so rho = n (2r+1)^2
(Sec. II; "Color NLM" in Sec. IV gives rho = 3(2r+1)^2).

The paper does not say how patches are completed at the image border; the
oracle mirrors the image about its edge pixels without repeating them
("reflect-101": index -1 -> 1, H -> H-2).  Components are ordered (dy, dx, c)
with dy, dx running from -r to r; distances do not depend on the order.

Pinned by: tests/test_oracle_guide.py (a pure-Python per-pixel patch loop on
tiny images, and the patch of an interior pixel equal to the image block).
"""
from __future__ import annotations

import numpy as np


def reflect101(i: np.ndarray, n: int) -> np.ndarray:
    """Mirror integer indices into [0, n) without repeating the edge (n >= 2)."""
    i = np.asarray(i)
    period = 2 * (n - 1)
    j = np.mod(i, period)
    return np.where(j < n, j, period - j)


def patch_guide(f: np.ndarray, r: int) -> np.ndarray:
    """H x W x n image -> H x W x (n (2r+1)^2) patch vectors, reflect-101 border."""
    f = np.asarray(f, np.float64)
    H, W, n = f.shape
    ys = np.arange(H)
    xs = np.arange(W)
    parts = []
    for dy in range(-r, r + 1):
        iy = reflect101(ys + dy, H)
        for dx in range(-r, r + 1):
            ix = reflect101(xs + dx, W)
            parts.append(f[iy][:, ix, :])
    return np.concatenate(parts, axis=2)
