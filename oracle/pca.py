"""PCA-NLM (Sec. IV, following Tasdizen's principal-neighbourhood NLM, which the
paper cites for its NLM experiments): the NLM guide p(x), the colour patch of
radius r around x (``oracle.guide``), is replaced by its coordinates in the
leading q principal directions of the collection of patches, reducing the
guide dimension rho = n (2r+1)^2 (147 for 7 x 7 colour patches) to q (25 or 6
in the paper's experiments).

Test infrastructure only: imported by tests/, never by the package.

Steps, in order:
1. the patch vector p(x) of every pixel x (reflect-101 border);
2. the mean patch m = (1/N) sum_x p(x) and the covariance
   C = (1/N) sum_x (p(x) - m)(p(x) - m)^T;
3. the eigendecomposition C = U diag(lambda) U^T, lambda descending (LAPACK);
4. the guide p~(x) = U_q^T (p(x) - m), U_q the q leading eigenvectors;
5. Algorithm 1 with the guide p~: k-means landmarks on the seeded subsample
   used for NLM, box window.

Readings (the paper gives the method's name and q only): the covariance is
over every pixel's patch with the 1/N normalisation (the scale does not change
U); patches are centred by the mean patch before the projection (a shift:
every distance ||p~(x) - p~(y)||, and so kappa, is unchanged by it); the
leading eigenvectors are unique only up to sign and up to rotations inside a
group of equal eigenvalues, and the filter depends on U_q only through the
subspace it spans.

Pinned by tests/test_oracle_pca.py: the covariance equals a pure-Python loop
over the patches; U diagonalises C and the eigenvalues sum to the total
variance; with q = rho the projection is orthogonal, so PCA-NLM equals NLM
exactly (same landmarks mapped into the new coordinates, and also through
k-means, which commutes with the map); patches that vary along one image axis
only span at most H - 1 centred directions, which q = H - 1 keeps, so PCA-NLM
with that q equals NLM.
"""
from __future__ import annotations

import numpy as np

from . import guide as _guide
from . import kernels as _k
from . import nystrom as _ny
from . import pipeline as _pl


def patch_moments(f: np.ndarray, r: int):
    """Mean patch m and covariance C (1/N normalisation) of every pixel's patch."""
    p = _guide.patch_guide(f, r)
    P = p.reshape(-1, p.shape[2])
    m = P.mean(axis=0)
    D = P - m
    return m, (D.T @ D) / P.shape[0]


def pca_basis(C: np.ndarray, q: int):
    """All eigenvalues of C (descending) and the q leading eigenvectors (columns)."""
    lam, U = np.linalg.eigh(np.asarray(C, np.float64))
    order = np.argsort(lam, kind="stable")[::-1]
    return lam[order], U[:, order[:q]]


def project(p: np.ndarray, m: np.ndarray, Uq: np.ndarray) -> np.ndarray:
    """p~(x) = U_q^T (p(x) - m) for an H x W x rho patch image."""
    return (np.asarray(p, np.float64) - m) @ Uq


def pca_guide(f: np.ndarray, r: int, q: int, m=None, Uq=None):
    """The H x W x q PCA guide, from the image's own moments unless (m, Uq) are given."""
    p = _guide.patch_guide(f, r)
    if Uq is None:
        m, C = patch_moments(f, r)
        _, Uq = pca_basis(C, q)
    return project(p, m, Uq), m, Uq


def pca_nlm(f, sigma_r, K, q, S=10, patch_radius=3, frac=0.01, iters=10, seed=0, tau=1e-7,
            m=None, Uq=None, mu=None, landmark_dtype=np.float64):
    """PCA-NLM through Algorithm 1: PCA guide, k-means on the NLM subsample, box window."""
    f = np.asarray(f, np.float64)
    g_pca, m, Uq = pca_guide(f, patch_radius, q, m, Uq)
    H, W = f.shape[:2]
    info = dict(m=m, Uq=Uq)
    if mu is None:
        from . import rng as _rng
        Ns = _rng.subsample_size(H * W, frac)
        idx = _rng.stratified_sample(seed, Ns, H * W)
        X = g_pca.reshape(H * W, -1)[idx]
        mu, kinfo = _pl.landmarks(X, K, iters, seed)
        info.update(kinfo, sample_idx=idx)
    mu = np.asarray(mu, landmark_dtype).astype(np.float64)
    g = _ny.nystrom_filter(f, g_pca, mu, sigma_r, _k.box_taps(S), tau)
    return g, mu, info
