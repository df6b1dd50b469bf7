"""The exact kernel filter, Eq. (1) (Sec. II).

    g(x) = sum_{y in W_x} omega(x - y) kappa(p(x), p(y)) f(y)
           / sum_{y in W_x} omega(x - y) kappa(p(x), p(y))

W_x is the (2S+1) x (2S+1) window around x.  The paper does not define f
outside Omega; the oracle clips the window to Omega (pixels outside the image
take no part), which is what a zero-padded convolution of the numerator and
denominator planes gives in Eq. (7) and Eqs. (14)-(15).

Pinned by: tests/test_oracle_bruteforce.py -- a pure-Python per-pixel loop on
tiny images; a constant image is returned unchanged; with kappa == 1 the filter
is the normalised spatial blur (omega * f) / (omega * 1_Omega).
"""
from __future__ import annotations

import numpy as np

from .kernels import kappa


def kernel_filter(f: np.ndarray, p: np.ndarray, taps: np.ndarray, sigma_r: float) -> np.ndarray:
    """Eq. (1) at every pixel.  f: H x W x n, p: H x W x rho, taps: 1-D factor of omega.

    sigma_r = inf means kappa == 1.  The sum over y in W_x is taken offset by
    offset z = y - x, vectorised over x.
    """
    f = np.asarray(f, np.float64)
    p = np.asarray(p, np.float64)
    H, W, n = f.shape
    S = (len(taps) - 1) // 2
    num = np.zeros((H, W, n))
    den = np.zeros((H, W))
    for zy in range(-S, S + 1):
        y0, y1 = max(0, -zy), min(H, H - zy)        # x rows with x+zy inside
        if y0 >= y1:
            continue
        for zx in range(-S, S + 1):
            x0, x1 = max(0, -zx), min(W, W - zx)
            if x0 >= x1:
                continue
            px = p[y0:y1, x0:x1]
            py = p[y0 + zy:y1 + zy, x0 + zx:x1 + zx]
            k = np.ones(px.shape[:2]) if np.isinf(sigma_r) else kappa(px, py, sigma_r)
            w = taps[zy + S] * taps[zx + S] * k
            num[y0:y1, x0:x1] += w[..., None] * f[y0 + zy:y1 + zy, x0 + zx:x1 + zx]
            den[y0:y1, x0:x1] += w
    return num / den[..., None]


def kernel_filter_at(f: np.ndarray, p: np.ndarray, taps: np.ndarray, sigma_r: float,
                     ys: np.ndarray, xs: np.ndarray) -> np.ndarray:
    """Eq. (1) at the listed pixels only (direct window sum per pixel)."""
    f = np.asarray(f, np.float64)
    p = np.asarray(p, np.float64)
    H, W, n = f.shape
    S = (len(taps) - 1) // 2
    out = np.empty((len(ys), n))
    for i, (y, x) in enumerate(zip(ys, xs)):
        a0, a1 = max(0, y - S), min(H, y + S + 1)
        b0, b1 = max(0, x - S), min(W, x + S + 1)
        om = np.outer(taps[a0 - y + S:a1 - y + S], taps[b0 - x + S:b1 - x + S])
        k = np.ones(om.shape) if np.isinf(sigma_r) else kappa(p[a0:a1, b0:b1], p[y, x], sigma_r)
        w = om * k
        out[i] = np.tensordot(w, f[a0:a1, b0:b1], axes=([0, 1], [0, 1])) / w.sum()
    return out
