"""Pins for oracle.kernels and the separable convolution (Sec. II, Sec. IV setup, Eq. (7))."""
import math

import numpy as np
import pytest

from oracle import kernels as K
from oracle import nystrom as ny


@pytest.mark.parametrize("sigma,S", [(3.0, 9), (5.0, 15), (4.0, 12), (2.5, 8), (8.0, 24)])
def test_window_radius_is_ceil_3sigma(sigma, S):
    assert K.window_radius(sigma) == S


def test_gaussian_taps_closed_form():
    g = K.gaussian_taps(2.0, 6)
    assert g.shape == (13,)
    assert g[6] == 1.0                                   # omega(0) = 1
    assert math.isclose(g[6 + 2], math.exp(-0.5), rel_tol=1e-15)   # t = sigma
    assert math.isclose(g[6 - 4], math.exp(-2.0), rel_tol=1e-15)   # t = -2 sigma
    assert np.array_equal(g, g[::-1])


def test_gaussian_dsigma_matches_finite_difference():
    s, S, h = 3.3, 10, 1e-6
    fd = (K.gaussian_taps(s + h, S) - K.gaussian_taps(s - h, S)) / (2 * h)
    assert np.allclose(K.gaussian_taps_dsigma(s, S), fd, rtol=1e-7, atol=1e-12)


def test_kappa_closed_form():
    t = np.array([1.0, 2.0, 3.0])
    assert K.kappa(t, t, 7.0) == 1.0
    s = t + np.array([0.0, 3.0, 4.0])                    # distance 5
    assert math.isclose(K.kappa(t, s, 5.0), math.exp(-0.5), rel_tol=1e-15)
    assert math.isclose(K.kappa(t, s, 2.5), math.exp(-2.0), rel_tol=1e-15)


def test_delta_image_reproduces_omega():
    S = 3
    taps = K.gaussian_taps(1.3, S)
    a = np.zeros((11, 12))
    a[5, 6] = 1.0
    out = ny.conv_same(a, taps)
    want = np.zeros_like(a)
    want[2:9, 3:10] = np.outer(taps, taps)
    assert np.allclose(out, want, atol=1e-15)


def test_constant_plane_gives_clipped_window_mass():
    S = 4
    taps = K.gaussian_taps(1.7, S)
    H, W = 7, 9
    out = ny.conv_same(np.ones((H, W)), taps)
    for y in range(H):
        for x in range(W):
            m = sum(taps[dy + S] * taps[dx + S]
                    for dy in range(-S, S + 1) for dx in range(-S, S + 1)
                    if 0 <= y + dy < H and 0 <= x + dx < W)
            assert math.isclose(out[y, x], m, rel_tol=1e-13)


@pytest.mark.parametrize("shape,S", [((9, 13, 2), 3), ((2, 5, 1), 3), ((6, 4, 3), 5)])
def test_separable_equals_direct(shape, S):
    rng = np.random.default_rng(1)
    a = rng.normal(size=shape)
    taps = K.gaussian_taps(1.9, S)
    assert np.allclose(ny.conv_same(a, taps), ny.conv_direct(a, taps), rtol=1e-13, atol=1e-13)
    box = K.box_taps(S)
    assert np.allclose(ny.conv_same(a, box), ny.conv_direct(a, box), rtol=1e-13, atol=1e-13)
