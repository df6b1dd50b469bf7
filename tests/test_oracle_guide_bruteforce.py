"""Pins for oracle.guide (NLM patch guide) and oracle.bruteforce (Eq. (1))."""
import math

import numpy as np
import pytest

from oracle import bruteforce as bf
from oracle import guide as gd
from oracle import kernels as K


def _mirror(i, n):
    # reflect-101 written out case by case
    while i < 0 or i >= n:
        if i < 0:
            i = -i
        if i >= n:
            i = 2 * (n - 1) - i
    return i


def test_patch_guide_matches_loop():
    rng = np.random.default_rng(2)
    f = rng.uniform(0, 255, size=(5, 6, 2))
    r = 2
    p = gd.patch_guide(f, r)
    assert p.shape == (5, 6, 2 * 25)
    for y in range(5):
        for x in range(6):
            v = []
            for dy in range(-r, r + 1):
                for dx in range(-r, r + 1):
                    for c in range(2):
                        v.append(f[_mirror(y + dy, 5), _mirror(x + dx, 6), c])
            assert np.array_equal(p[y, x], np.array(v))


def test_interior_patch_is_the_block():
    rng = np.random.default_rng(3)
    f = rng.uniform(0, 1, size=(9, 9, 3))
    p = gd.patch_guide(f, 1)
    assert np.array_equal(p[4, 5], f[3:6, 4:7, :].reshape(-1))


def _loop_filter(f, p, taps, sigma_r):
    H, W, n = f.shape
    S = (len(taps) - 1) // 2
    out = np.zeros_like(f, dtype=np.float64)
    for y in range(H):
        for x in range(W):
            num = np.zeros(n)
            den = 0.0
            for v in range(max(0, y - S), min(H, y + S + 1)):
                for u in range(max(0, x - S), min(W, x + S + 1)):
                    d2 = sum((p[y, x, c] - p[v, u, c]) ** 2 for c in range(p.shape[2]))
                    k = 1.0 if math.isinf(sigma_r) else math.exp(-d2 / (2 * sigma_r ** 2))
                    w = taps[v - y + S] * taps[u - x + S] * k
                    num += w * f[v, u]
                    den += w
            out[y, x] = num / den
    return out


@pytest.mark.parametrize("sigma_r", [20.0, 60.0, math.inf])
def test_bruteforce_matches_per_pixel_loop(sigma_r):
    rng = np.random.default_rng(4)
    f = rng.uniform(0, 255, size=(6, 7, 3))
    taps = K.gaussian_taps(1.2, 2)
    assert np.allclose(bf.kernel_filter(f, f, taps, sigma_r), _loop_filter(f, f, taps, sigma_r),
                       rtol=1e-12, atol=1e-10)


def test_bruteforce_joint_and_patch_guides():
    rng = np.random.default_rng(5)
    f = rng.uniform(0, 255, size=(6, 5, 3))
    g = rng.uniform(0, 255, size=(6, 5, 2))
    taps = K.box_taps(2)
    assert np.allclose(bf.kernel_filter(f, g, taps, 40.0), _loop_filter(f, g, taps, 40.0), rtol=1e-12)
    p = gd.patch_guide(f, 1)
    assert np.allclose(bf.kernel_filter(f, p, taps, 90.0), _loop_filter(f, p, taps, 90.0), rtol=1e-12)


def test_bruteforce_at_equals_full():
    rng = np.random.default_rng(6)
    f = rng.uniform(0, 255, size=(10, 11, 3))
    taps = K.gaussian_taps(1.5, 5)
    full = bf.kernel_filter(f, f, taps, 30.0)
    ys = np.array([0, 3, 9, 5])
    xs = np.array([0, 10, 4, 5])
    assert np.allclose(bf.kernel_filter_at(f, f, taps, 30.0, ys, xs), full[ys, xs], rtol=1e-13)


def test_constant_image_is_fixed():
    f = np.full((8, 9, 3), 77.0)
    out = bf.kernel_filter(f, f, K.gaussian_taps(2.0, 6), 10.0)
    assert np.allclose(out, 77.0, rtol=1e-14)


def test_infinite_sigma_r_is_normalised_blur():
    rng = np.random.default_rng(7)
    f = rng.uniform(0, 255, size=(8, 6, 2))
    taps = K.gaussian_taps(1.4, 3)
    S = 3
    H, W, _ = f.shape
    want = np.zeros_like(f)
    for y in range(H):
        for x in range(W):
            num = 0.0
            den = 0.0
            for v in range(max(0, y - S), min(H, y + S + 1)):
                for u in range(max(0, x - S), min(W, x + S + 1)):
                    w = taps[v - y + S] * taps[u - x + S]
                    num = num + w * f[v, u]
                    den += w
            want[y, x] = num / den
    assert np.allclose(bf.kernel_filter(f, f, taps, math.inf), want, rtol=1e-13)
