"""Recursive O(1) Gaussian filter (Young & van Vliet 1995): the spatial filter
the paper's experiments run for a Gaussian omega (Sec. IV), and one of the
O(1)-per-pixel convolution methods Sec. III names for the (n+1) K convolutions
of Eqs. (14)-(15).

Test infrastructure only: imported by tests/, never by the package.

A line x[0..L) is filtered by a third-order causal pass followed by the same
recursion run backwards,
    w[i] = B x[i] + (b1 w[i-1] + b2 w[i-2] + b3 w[i-3]) / b0      (i = 0, 1, ...)
    y[i] = B w[i] + (b1 y[i+1] + b2 y[i+2] + b3 y[i+3]) / b0      (i = L-1, ...)
with the published coefficients
    q  = 0.98711 s - 0.96330                      (s >= 2.5)
    q  = 3.97156 - 4.14554 sqrt(1 - 0.26891 s)    (0.5 <= s < 2.5)
    b0 = 1.57825 + 2.44413 q + 1.4281 q^2 + 0.422205 q^3
    b1 = 2.44413 q + 2.85619 q^2 + 1.26661 q^3
    b2 = -(1.4281 q^2 + 1.26661 q^3)
    b3 = 0.422205 q^3
    B  = 1 - (b1 + b2 + b3) / b0.
Boundary reading (the paper does not state one): the window clipping of
Eq. (1) is zero padding, as for the FIR filter, so the recursive filter is
applied to the line extended by zeros on both sides and the result cropped.
On the left the zero initial state is exactly that; on the right the causal
pass runs on into the zero padding until its state has decayed below 1e-20
(|largest pole|^P < 1e-20) and the anticausal pass starts there from zero.
The result is the convolution of the zero-padded line with the filter's
two-sided impulse response h, the same operator whichever end is processed
first.  The 2-D filter runs along axis 0 (columns) and then axis 1 (rows).
It approximates the normalised Gaussian of standard deviation s (unit DC
gain); the Nystrom filter's ratio zeta / eta does not depend on the
normalisation.

Pinned by tests/test_oracle_iir.py: the roots of the recursion are the poles of
Young & van Vliet's Gaussian approximation; unit DC gain; the variance of the
impulse response equals the closed form from the poles; the filter is the
convolution of the zero-padded line with h at both ends; h is within the
method's accuracy of the sampled Gaussian; the Nystrom filter built on it
returns a constant image unchanged, gives the normalised IIR blur for
sigma_r -> infinity and, on a few-colour image with its colours as
landmarks, equals the brute-force filter of Eq. (1) with omega = h (x) h.
"""
from __future__ import annotations

import numpy as np


def yvv_coefficients(s: float):
    """(B, b1 / b0, b2 / b0, b3 / b0) for standard deviation s >= 0.5."""
    if s < 0.5:
        raise ValueError("the recursive Gaussian needs sigma >= 0.5")
    q = 0.98711 * s - 0.96330 if s >= 2.5 else 3.97156 - 4.14554 * np.sqrt(1.0 - 0.26891 * s)
    b0 = 1.57825 + 2.44413 * q + 1.4281 * q * q + 0.422205 * q ** 3
    b1 = 2.44413 * q + 2.85619 * q * q + 1.26661 * q ** 3
    b2 = -(1.4281 * q * q + 1.26661 * q ** 3)
    b3 = 0.422205 * q ** 3
    B = 1.0 - (b1 + b2 + b3) / b0
    return B, b1 / b0, b2 / b0, b3 / b0


def causal_poles(s: float) -> np.ndarray:
    """Roots of z^3 - (b1 z^2 + b2 z + b3) / b0: the poles of the causal pass."""
    _, c1, c2, c3 = yvv_coefficients(s)
    return np.roots([1.0, -c1, -c2, -c3])


def pad_length(s: float) -> int:
    """Zeros appended on the right so that the causal state decays below 1e-20."""
    rho = float(np.max(np.abs(causal_poles(s))))
    return int(np.ceil(np.log(1e-20) / np.log(rho))) + 3


def iir_1d(x: np.ndarray, s: float, axis: int = 0) -> np.ndarray:
    """Causal then anticausal pass along `axis` on the zero-padded line, cropped."""
    B, c1, c2, c3 = yvv_coefficients(s)
    a = np.moveaxis(np.asarray(x, np.float64), axis, 0)
    L = a.shape[0]
    a = np.concatenate([a, np.zeros((pad_length(s),) + a.shape[1:])], axis=0)
    n = a.shape[0]
    w = np.empty_like(a)
    zero = np.zeros(a.shape[1:])
    w1 = w2 = w3 = zero
    for i in range(n):
        wi = B * a[i] + c1 * w1 + c2 * w2 + c3 * w3
        w[i] = wi
        w3, w2, w1 = w2, w1, wi
    y = np.empty_like(a)
    y1 = y2 = y3 = zero
    for i in range(n - 1, -1, -1):
        yi = B * w[i] + c1 * y1 + c2 * y2 + c3 * y3
        y[i] = yi
        y3, y2, y1 = y2, y1, yi
    return np.moveaxis(y[:L], 0, axis)


def iir_2d(a: np.ndarray, s: float) -> np.ndarray:
    """The 2-D recursive Gaussian on an H x W (or H x W x c) array: columns, then rows."""
    return iir_1d(iir_1d(a, s, axis=0), s, axis=1)


def nystrom_filter_iir(f: np.ndarray, p: np.ndarray, mu: np.ndarray, sigma_r: float,
                       sigma_s: float, tau: float, return_parts: bool = False):
    """Algorithm 1 with every spatial convolution of Eqs. (14)-(15) done by iir_2d."""
    from .nystrom import nystrom_filter
    return nystrom_filter(f, p, mu, sigma_r, None, tau, return_parts=return_parts,
                          conv=lambda a: iir_2d(a, sigma_s))
