"""Pins for oracle.nystrom (Eqs. (9)-(12), (14)-(15), Algorithm 1)."""
import math

import numpy as np
import pytest

from oracle import bound as bd
from oracle import bruteforce as bf
from oracle import guide as gd
from oracle import kernels as K
from oracle import nystrom as ny
from paper_1901_06112_gb300 import synth


def test_eig_two_landmarks_closed_form():
    # A = [[1, a], [a, 1]] has eigenpairs (1 + a, (1, 1)/sqrt 2) and (1 - a, (1, -1)/sqrt 2)
    mu = np.array([[0.0, 0.0, 0.0], [3.0, 0.0, 4.0]])
    a = math.exp(-25.0 / (2 * 5.0 ** 2))
    A = ny.landmark_kernel(mu, 5.0)
    assert np.allclose(A, [[1, a], [a, 1]], rtol=1e-15)
    alpha, W = ny.eig_desc(A)
    assert np.allclose(alpha, [1 + a, 1 - a], rtol=1e-14)
    assert np.allclose(np.abs(W), 1 / math.sqrt(2), rtol=1e-14)
    assert W[0, 0] * W[1, 0] > 0 and W[0, 1] * W[1, 1] < 0


def test_eig_reconstruction_and_truncation():
    rng = np.random.default_rng(11)
    mu = rng.uniform(0, 255, size=(12, 3))
    mu[5] = mu[2]                                            # duplicate -> singular A
    A = ny.landmark_kernel(mu, 60.0)
    alpha, W = ny.eig_desc(A)
    assert np.all(np.diff(alpha) <= 0)
    assert np.linalg.norm(A - (W * alpha) @ W.T) <= 1e-12 * np.linalg.norm(A)
    assert np.allclose(W.T @ W, np.eye(12), atol=1e-13)
    keep = ny.kept_modes(alpha, 1e-7)
    assert keep.size < 12 and np.all(alpha[keep] > 1e-7 * alpha[0])


def _tiny(seed, H=9, W=10, n=3):
    return synth.random_image(H, W, n, seed)


@pytest.mark.parametrize("K_", [1, 3, 6])
def test_constant_image_returned_unchanged(K_):
    rng = np.random.default_rng(12)
    f = np.full((8, 9, 3), 123.0)
    guide = _tiny(13, 8, 9, 3)                              # joint guide: any guide works
    mu = rng.uniform(0, 255, size=(K_, 3))
    if K_ > 1:
        mu[-1] = mu[0]                                       # duplicated landmark
    g = ny.nystrom_filter(f, guide, mu, 50.0, K.gaussian_taps(1.5, 4), 1e-9)
    assert np.allclose(g, 123.0, rtol=1e-12)


def test_infinite_sigma_r_gives_normalised_blur():
    f = _tiny(14)
    mu = np.random.default_rng(15).uniform(0, 255, size=(5, 3))
    taps = K.gaussian_taps(1.3, 3)
    g = ny.nystrom_filter(f, f, mu, 1e6 * 255, taps, 1e-7)
    blur = bf.kernel_filter(f, f, taps, math.inf)
    assert np.allclose(g, blur, rtol=1e-7)


def test_few_colour_exactness():
    cols = np.array([[0, 0, 0], [255, 0, 0], [0, 255, 0], [0, 0, 255], [255, 255, 255]], float)
    f = synth.few_colour(12, 13, cols, 16).astype(np.float64)
    sigma_r = 60.0
    taps = K.gaussian_taps(1.7, 5)
    g = ny.nystrom_filter(f, f, cols, sigma_r, taps, 1e-12)
    assert np.allclose(g, bf.kernel_filter(f, f, taps, sigma_r), rtol=1e-10, atol=1e-9)


def test_all_pixels_as_landmarks_is_exact_blf_and_nlm():
    f = _tiny(17, 12, 12, 3).astype(np.float64)
    taps = K.gaussian_taps(1.5, 4)
    g = ny.nystrom_filter(f, f, f.reshape(-1, 3), 6.0, taps, 1e-13)
    assert np.allclose(g, bf.kernel_filter(f, f, taps, 6.0), rtol=1e-8, atol=1e-7)
    p = gd.patch_guide(f, 1)
    box = K.box_taps(3)
    g2 = ny.nystrom_filter(f, p, p.reshape(-1, p.shape[2]), 40.0, box, 1e-13)
    assert np.allclose(g2, bf.kernel_filter(f, p, box, 40.0), rtol=1e-8, atol=1e-7)


def test_single_landmark_closed_form():
    f = _tiny(18)
    mu = np.array([[100.0, 120.0, 90.0]])
    taps = K.gaussian_taps(1.1, 3)
    e = K.kappa(f, mu[0], 45.0)[..., None]
    want = ny.conv_direct(e * f, taps) / ny.conv_direct(e, taps)
    assert np.allclose(ny.nystrom_filter(f, f, mu, 45.0, taps, 1e-7), want, rtol=1e-12)


def test_convolution_form_equals_explicit_khat():
    f = _tiny(19, 7, 8, 3).astype(np.float64)
    mu = np.random.default_rng(20).uniform(0, 255, size=(6, 3))
    taps = K.gaussian_taps(1.2, 3)
    Kh = bd.nystrom_matrix(f.reshape(-1, 3), mu, 70.0, 1e-9)
    want = bd.filter_with_matrix(f, Kh, taps)
    assert np.allclose(ny.nystrom_filter(f, f, mu, 70.0, taps, 1e-9), want, rtol=1e-10)


def test_filter_at_equals_full_and_features_factor_khat():
    f = _tiny(21, 11, 9, 3).astype(np.float64)
    mu = np.random.default_rng(22).uniform(0, 255, size=(7, 3))
    taps = K.gaussian_taps(1.4, 4)
    full = ny.nystrom_filter(f, f, mu, 50.0, taps, 1e-8)
    ys = np.array([0, 10, 5, 3])
    xs = np.array([0, 8, 4, 7])
    assert np.allclose(ny.nystrom_filter_at(f, f, mu, 50.0, taps, 1e-8, ys, xs), full[ys, xs], rtol=1e-11)
    phi, alpha, keep = ny.features(f, mu, 50.0, 1e-8)
    Kh = bd.nystrom_matrix(f.reshape(-1, 3), mu, 50.0, 1e-8)
    assert np.allclose(phi @ phi.T, Kh, rtol=1e-9, atol=1e-11)
    ps, _, _ = ny.features_symmetric(f, mu, 50.0, 1e-8)
    assert ps.shape[1] == 7
    assert np.allclose(ps @ ps.T, Kh, rtol=1e-9, atol=1e-11)
    mu[3] = mu[1]                                   # rank deficient: still factors K-hat
    ps, _, keep = ny.features_symmetric(f, mu, 50.0, 1e-8)
    Kh = bd.nystrom_matrix(f.reshape(-1, 3), mu, 50.0, 1e-8)
    assert keep.size < 7 and np.allclose(ps @ ps.T, Kh, rtol=1e-9, atol=1e-11)


def test_no_mode_kept_raises():
    f = _tiny(23)
    with pytest.raises(FloatingPointError):
        ny.nystrom_filter(f, f, np.zeros((2, 3)), 30.0, K.gaussian_taps(1.0, 3), 2.0)
