"""Range kernel kappa and spatial kernel omega.

* kappa(t, s) = exp(-||t - s||^2 / (2 theta^2)).  Sec. II writes the Gaussian
  range kernel as exp(-theta ||s - t||^2) with theta a precision, while the
  experimental setup (Sec. IV) states "covariance theta^2 I", i.e. theta is a
  standard deviation.  The oracle follows the setup: sigma_r = theta.
* omega(z) = exp(-||z||^2 / (2 sigma^2)) on the square window ||z||_inf <= S with
  S = ceil(3 sigma) (Sec. IV setup: "covariance sigma^2 I and S = 3 sigma"),
  left unnormalised because the constant cancels in Eq. (1) and Eq. (14)/(15).
  The nonlocal-means window is a box: omega = 1 on (2S+1)^2 pixels.
  Both kernels are separable: omega(z) = g(z_y) g(z_x).

Pinned by: tests/test_oracle_kernels.py (closed forms of the 1-D taps, a delta
image reproducing omega through the separable convolution).
"""
from __future__ import annotations

import math

import numpy as np


def window_radius(sigma_s: float) -> int:
    """S = ceil(3 sigma) (Sec. IV setup)."""
    return int(math.ceil(3.0 * sigma_s))


def gaussian_taps(sigma_s: float, S: int) -> np.ndarray:
    """1-D factor g(t) = exp(-t^2 / (2 sigma^2)), t = -S..S, of the Gaussian omega."""
    t = np.arange(-S, S + 1, dtype=np.float64)
    return np.exp(-(t * t) / (2.0 * sigma_s * sigma_s))


def gaussian_taps_dsigma(sigma_s: float, S: int) -> np.ndarray:
    """d g(t) / d sigma = g(t) t^2 / sigma^3 (window radius S held fixed)."""
    t = np.arange(-S, S + 1, dtype=np.float64)
    return gaussian_taps(sigma_s, S) * (t * t) / sigma_s ** 3


def box_taps(S: int) -> np.ndarray:
    """1-D factor of the box omega: ones on -S..S (Sec. IV: box window for NLM)."""
    return np.ones(2 * S + 1, dtype=np.float64)


def omega_2d(taps: np.ndarray) -> np.ndarray:
    """omega(z) = g(z_y) g(z_x) on the (2S+1) x (2S+1) window."""
    return np.outer(taps, taps)


def kappa(t: np.ndarray, s: np.ndarray, sigma_r: float) -> np.ndarray:
    """Gaussian range kernel exp(-||t - s||^2 / (2 sigma_r^2)) over the last axis."""
    d = np.asarray(t, np.float64) - np.asarray(s, np.float64)
    return np.exp(-np.sum(d * d, axis=-1) / (2.0 * sigma_r * sigma_r))
