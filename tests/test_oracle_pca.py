"""Pins for oracle.pca (PCA-NLM of the Sec. IV experiments)."""
import numpy as np
import pytest

from oracle import guide as gd
from oracle import kernels as Kr
from oracle import nystrom as ny
from oracle import pca
from oracle import pipeline as pl
from paper_1901_06112_gb300 import synth


def test_covariance_is_the_patch_loop():
    f = synth.random_image(5, 6, 2, 21).astype(np.float64)
    r = 1
    H, W, n = f.shape
    vecs = []
    for y in range(H):
        for x in range(W):
            v = []
            for dy in range(-r, r + 1):
                for dx in range(-r, r + 1):
                    yy, xx = y + dy, x + dx
                    yy = -yy if yy < 0 else (2 * (H - 1) - yy if yy >= H else yy)
                    xx = -xx if xx < 0 else (2 * (W - 1) - xx if xx >= W else xx)
                    v.extend(f[yy, xx, c] for c in range(n))
            vecs.append(v)
    P = np.array(vecs)
    m_want = sum(P) / len(P)
    C_want = sum(np.outer(p - m_want, p - m_want) for p in P) / len(P)
    m, C = pca.patch_moments(f, r)
    assert np.allclose(m, m_want, rtol=1e-13)
    assert np.allclose(C, C_want, rtol=1e-12, atol=1e-9)


def test_basis_diagonalises_the_covariance():
    f = synth.voronoi_colour(20, 24, 6, 10.0, 3).astype(np.float64)
    m, C = pca.patch_moments(f, 1)
    lam, U = pca.pca_basis(C, C.shape[0])
    assert np.all(np.diff(lam) <= 1e-9 * lam[0])
    assert np.allclose(U.T @ U, np.eye(C.shape[0]), atol=1e-12)
    assert np.allclose(U.T @ C @ U, np.diag(lam), atol=1e-9 * lam[0])
    assert abs(lam.sum() - np.trace(C)) <= 1e-10 * np.trace(C)


@pytest.mark.parametrize("r", [1, 2])
def test_full_dimension_pca_nlm_equals_nlm(r):
    # q = rho: p~ = U^T (p - m) is an isometry, so kappa and the filter are unchanged
    f = synth.voronoi_colour(14, 16, 5, 12.0, 7).astype(np.float64)
    p = gd.patch_guide(f, r)
    rho = p.shape[2]
    mu = p.reshape(-1, rho)[np.random.default_rng(4).choice(14 * 16, 6, replace=False)]
    g_pca, m, U = pca.pca_guide(f, r, rho)
    taps = Kr.box_taps(3)
    sr = 20.0 * np.sqrt(rho)                 # range scale grows with the patch dimension
    want = ny.nystrom_filter(f, p, mu, sr, taps, 1e-9)
    got = ny.nystrom_filter(f, g_pca, (mu - m) @ U, sr, taps, 1e-9)
    assert np.allclose(got, want, rtol=1e-9, atol=1e-7)
    # and through k-means, which commutes with the isometry
    g1, _, _ = pca.pca_nlm(f, sr, 5, rho, S=3, patch_radius=r, frac=0.5, iters=4, seed=2)
    g2, _, _ = pl.nlm(f, sr, 5, S=3, patch_radius=r, frac=0.5, iters=4, seed=2)
    assert np.allclose(g1, g2, rtol=1e-8, atol=1e-6)


def test_patches_of_rows_only_keep_h_minus_1_directions():
    # f varies along y only: the centred patches span at most H - 1 directions,
    # so the PCA guide with q = H - 1 preserves every distance and PCA-NLM = NLM
    H, W, n, r = 4, 11, 2, 1
    rows = np.random.default_rng(5).uniform(0, 255, size=(H, 1, n))
    f = np.repeat(rows, W, axis=1)
    m, C = pca.patch_moments(f, r)
    lam, U = pca.pca_basis(C, H - 1)
    assert np.all(lam[H - 1:] <= 1e-10 * lam[0])
    p = gd.patch_guide(f, r)
    D = p.reshape(-1, p.shape[2]) - m
    assert np.allclose(D @ U @ U.T, D, atol=1e-9)         # the projector keeps every patch
    mu = p.reshape(-1, p.shape[2])[[0, W + 3, 3 * W + 1]]
    taps = Kr.box_taps(2)
    want = ny.nystrom_filter(f, p, mu, 80.0, taps, 1e-9)
    g_pca, _, _ = pca.pca_guide(f, r, H - 1, m, U)
    got = ny.nystrom_filter(f, g_pca, (mu - m) @ U, 80.0, taps, 1e-9)
    assert np.allclose(got, want, rtol=1e-9, atol=1e-7)


def test_truncated_pca_drops_only_the_trailing_variance():
    # the projected patches keep sum(lam[:q]) of the total variance
    f = synth.voronoi_colour(24, 28, 8, 15.0, 9).astype(np.float64)
    m, C = pca.patch_moments(f, 2)
    lam, U = pca.pca_basis(C, 6)
    g, _, _ = pca.pca_guide(f, 2, 6, m, U)
    var = np.mean(np.sum(g.reshape(-1, 6) ** 2, axis=1))
    assert abs(var - lam[:6].sum()) <= 1e-9 * lam[:6].sum()
