"""Pins for oracle.iir: the recursive Gaussian of Young & van Vliet (1995) that the
paper uses for a Gaussian omega (Sec. IV), and Algorithm 1 built on it.

The independent facts used here:
* YvV place the three causal poles at q / (m0 + q) and q / (m1 + q +- i m2) with
  m0 = 1.16680, m1 = 1.10783, m2 = 1.40586 (their Gaussian approximation); the
  expanded coefficients b0..b3 must have exactly these roots;
* a causal pass with poles p_i and gain B has the impulse response
  B sum_i A_i p_i^n, A_i = p_i^2 / prod_{j != i} (p_i - p_j) (partial fractions),
  so the causal-then-anticausal filter has the two-sided response
  h(m) = B^2 sum_{i,j} A_i A_j p_j^|m| / (1 - p_i p_j), whose variance is
  2 sum_i p_i / (1 - p_i)^2 (cumulants of the geometric factors add);
* on the zero-padded line the filter is the convolution with h at either end;
* h approximates the sampled Gaussian within a few per cent (the method's
  accuracy), which fixes q(sigma).
"""
import math

import numpy as np
import pytest

from oracle import bruteforce as bf
from oracle import iir
from oracle import kernels as K
from oracle import nystrom as ny
from paper_1901_06112_gb300 import synth

M0, M1, M2 = 1.16680, 1.10783, 1.40586
SIGMAS = [0.5, 0.8, 1.3, 2.4, 2.5, 3.0, 5.0, 8.0, 20.0]


def _q(s):
    return 0.98711 * s - 0.96330 if s >= 2.5 else 3.97156 - 4.14554 * math.sqrt(1.0 - 0.26891 * s)


def _poles(s):
    q = _q(s)
    return np.array([q / (M0 + q), q / (M1 + q + 1j * M2), q / (M1 + q - 1j * M2)])


def _h_closed(s, m):
    # the exact roots of the recursion (pinned to the published poles above)
    B = iir.yvv_coefficients(s)[0]
    p = iir.causal_poles(s)
    A = np.array([p[i] ** 2 / np.prod([p[i] - p[j] for j in range(3) if j != i]) for i in range(3)])
    m = np.abs(np.asarray(m))[..., None, None]
    h = B * B * np.sum(A[:, None] * A[None, :] * p[None, :] ** m / (1.0 - p[:, None] * p[None, :]),
                       axis=(-2, -1))
    return h.real


@pytest.mark.parametrize("s", SIGMAS)
def test_recursion_roots_are_the_published_poles(s):
    got = np.sort_complex(iir.causal_poles(s))
    want = np.sort_complex(_poles(s))
    assert np.allclose(got, want, rtol=1e-4, atol=0)   # coefficients printed to 5-6 digits


@pytest.mark.parametrize("s", [0.5, 3.0, 12.0])
def test_unit_dc_gain(s):
    L = 40 * int(s) + 400
    y = iir.iir_1d(np.ones(L), s)
    mid = y[L // 2 - 50:L // 2 + 50]
    assert np.allclose(mid, 1.0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("s", [0.7, 2.0, 3.0, 8.0])
def test_impulse_response_is_the_closed_form_at_both_ends(s):
    L = 301
    for j in (0, 1, 150, 299, 300):
        e = np.zeros(L)
        e[j] = 1.0
        y = iir.iir_1d(e, s)
        want = _h_closed(s, np.arange(L) - j)
        assert np.abs(y - want).max() <= 1e-13 * want.max(), (s, j)


@pytest.mark.parametrize("s", [1.0, 4.0, 10.0])
def test_variance_from_the_poles(s):
    L = int(60 * s) + 200
    e = np.zeros(2 * L + 1)
    e[L] = 1.0
    h = iir.iir_1d(e, s)
    m = np.arange(-L, L + 1)
    assert abs(h.sum() - 1.0) < 1e-12
    assert abs((m * h).sum()) < 1e-10 * s
    p = iir.causal_poles(s)
    want = (2.0 * np.sum(p / (1.0 - p) ** 2)).real
    assert abs((m * m * h).sum() - want) <= 1e-9 * want


def test_reversal_equivariance_random_line():
    x = np.random.default_rng(3).normal(size=(157, 4))
    y = iir.iir_1d(x, 3.3)
    yr = iir.iir_1d(x[::-1], 3.3)
    assert np.allclose(yr[::-1], y, rtol=0, atol=1e-13)


@pytest.mark.parametrize("s", [2.0, 3.0, 5.0, 8.0, 12.0, 20.0])
def test_close_to_the_sampled_gaussian(s):
    # YvV approximate the Gaussian to a few per cent in shape; a wrong q(sigma)
    # or a wrong coefficient moves the best-fitting width by far more
    L = int(30 * s)
    e = np.zeros(2 * L + 1)
    e[L] = 1.0
    h = iir.iir_1d(e, s)
    m = np.arange(-L, L + 1)

    def gauss(t):
        g = np.exp(-m * m / (2.0 * t * t))
        return g / g.sum()

    ts = s * np.linspace(0.85, 1.15, 601)
    best = ts[np.argmin([np.sum((h - gauss(t)) ** 2) for t in ts])]
    g = gauss(s)
    assert abs(best / s - 1.0) < 0.03
    assert abs(h[L] / g[L] - 1.0) < 0.03
    assert np.sqrt(np.sum((h - g) ** 2) / np.sum(g * g)) < 0.07


def test_2d_is_separable_outer_product():
    a = np.zeros((9, 11))
    a[3, 8] = 1.0
    y = iir.iir_2d(a, 1.6)
    want = np.outer(_h_closed(1.6, np.arange(9) - 3), _h_closed(1.6, np.arange(11) - 8))
    assert np.allclose(y, want, rtol=0, atol=1e-14)


def test_nystrom_iir_constant_image_unchanged():
    f = np.full((10, 9, 3), 77.0)
    guide = synth.random_image(10, 9, 3, 5)
    mu = np.random.default_rng(6).uniform(0, 255, size=(4, 3))
    g = iir.nystrom_filter_iir(f, guide, mu, 50.0, 2.0, 1e-9)
    assert np.allclose(g, 77.0, rtol=1e-12)


def test_nystrom_iir_infinite_sigma_r_is_the_normalised_iir_blur():
    f = synth.random_image(11, 12, 3, 7)
    mu = np.random.default_rng(8).uniform(0, 255, size=(5, 3))
    g = iir.nystrom_filter_iir(f, f, mu, 1e6 * 255, 1.8, 1e-7)
    want = iir.iir_2d(f, 1.8) / iir.iir_2d(np.ones((11, 12)), 1.8)[..., None]
    assert np.allclose(g, want, rtol=1e-7)


def test_nystrom_iir_few_colour_exactness_against_eq1():
    # with the colours as landmarks the Nystrom filter is exact, so Algorithm 1 on
    # the recursive filter equals Eq. (1) with omega(z) = h(z_y) h(z_x)
    cols = np.array([[0, 0, 0], [255, 0, 0], [0, 255, 0], [0, 0, 255], [255, 255, 255]], float)
    f = synth.few_colour(12, 13, cols, 16).astype(np.float64)
    R = 13
    taps = _h_closed(2.2, np.arange(-R, R + 1))
    g = iir.nystrom_filter_iir(f, f, cols, 60.0, 2.2, 1e-12)
    assert np.allclose(g, bf.kernel_filter(f, f, taps, 60.0), rtol=1e-10, atol=1e-9)


def test_iir_against_fir_nystrom_is_within_the_method_accuracy():
    # the recursive and the truncated FIR Gaussian give nearly the same Nystrom filter
    w = synth.colour_blf_small()
    f = w.f[:64, :64].astype(np.float64)
    mu = f.reshape(-1, 3)[np.random.default_rng(9).choice(64 * 64, 8, replace=False)]
    sr = float(w.sigma_r)
    fir = ny.nystrom_filter(f, f, mu, sr, K.gaussian_taps(w.sigma_s, w.radius), 1e-7)
    rec = iir.nystrom_filter_iir(f, f, mu, sr, w.sigma_s, 1e-7)
    rel = np.sqrt(np.mean((rec - fir) ** 2) / np.mean(fir ** 2))
    assert rel < 0.02
