"""Explicit kernel matrices and the Theorem 1 error bound (tiny images only).

* K(i, j) = kappa(r_i, r_j) (Eq. (4)) and its Nystrom approximation
  K-hat = sum_k alpha_k v_k v_k^T (Eq. (8) with Eq. (12)) over the kept modes.
* ``filter_with_matrix`` evaluates Eq. (5) (Eq. (1) rewritten with K) for any
  m x m matrix; with K it is Eq. (1), with K-hat it is Eqs. (14)-(15).
* Theorem 1 (proof in the supplement).  With Delta = K-hat - K and
  eta(x) = sum_y omega(x-y) K(iota(x), iota(y)):
    ||g_hat(x) - g(x)|| <= ( ||g_hat(x)|| |eta - eta_hat| + ||zeta_hat - zeta|| ) / eta(x)
  and each difference is at most (sum_{y in W_x} omega(x-y)) max|Delta| times
  1 or max ||f||.  ``theorem1_pointwise`` returns this certified per-pixel
  bound.  The supplement's final form uses eta(x) >= omega(0) kappa(0,0) and
  bounds ||f(y)|| and ||g_hat(x)|| by sqrt(nR); for f in [0, R]^n the bound on
  ||f(y)|| is R sqrt(n), which ``theorem1_final`` uses (it needs
  ||g_hat(x)|| <= R sqrt(n), checked by the caller).

Pinned by: tests/test_oracle_bound.py (Delta = 0 gives zero error; the
explicit K-hat filter equals Algorithm 1; the bounds hold on random cases).
"""
from __future__ import annotations

import numpy as np

from .kernels import kappa
from .nystrom import cross_kernel, spectral_step


def kernel_matrix(R: np.ndarray, sigma_r: float) -> np.ndarray:
    """K(i, j) = kappa(r_i, r_j), Eq. (4)."""
    R = np.asarray(R, np.float64)
    return kappa(R[:, None, :], R[None, :, :], sigma_r)


def nystrom_matrix(R: np.ndarray, mu: np.ndarray, sigma_r: float, tau: float) -> np.ndarray:
    """K-hat = sum over kept k of alpha_k v_k v_k^T, Eq. (8) with Eq. (12)."""
    _, alpha, W, keep = spectral_step(mu, sigma_r, tau)
    B = cross_kernel(mu, R, sigma_r)
    Kh = np.zeros((B.shape[1], B.shape[1]))
    for k in keep:
        v = (B.T @ W[:, k]) / alpha[k]
        Kh += alpha[k] * np.outer(v, v)
    return Kh


def filter_with_matrix(f: np.ndarray, Kmat: np.ndarray, taps: np.ndarray, return_parts=False):
    """Eq. (5): sum_y omega(x-y) K(iota(x), iota(y)) f(y) / sum_y omega(x-y) K(...)."""
    f = np.asarray(f, np.float64)
    H, W, n = f.shape
    S = (len(taps) - 1) // 2
    F = f.reshape(H * W, n)
    zeta = np.zeros((H * W, n))
    eta = np.zeros(H * W)
    wsum = np.zeros(H * W)
    for y in range(H):
        for x in range(W):
            i = y * W + x
            a0, a1 = max(0, y - S), min(H, y + S + 1)
            b0, b1 = max(0, x - S), min(W, x + S + 1)
            om = np.outer(taps[a0 - y + S:a1 - y + S], taps[b0 - x + S:b1 - x + S])
            idx = (np.arange(a0, a1)[:, None] * W + np.arange(b0, b1)[None, :]).ravel()
            w = om.ravel() * Kmat[i, idx]
            zeta[i] = w @ F[idx]
            eta[i] = w.sum()
            wsum[i] = om.sum()
    g = (zeta / eta[:, None]).reshape(H, W, n)
    if return_parts:
        return g, dict(zeta=zeta.reshape(H, W, n), eta=eta.reshape(H, W), wsum=wsum.reshape(H, W))
    return g


def theorem1_pointwise(f, p, mu, sigma_r, taps, tau):
    """Per-pixel error ||g_hat - g|| and its certified bound (the proof's main inequality)."""
    f = np.asarray(f, np.float64)
    H, W, n = f.shape
    R = np.asarray(p, np.float64).reshape(H * W, -1)
    K = kernel_matrix(R, sigma_r)
    Kh = nystrom_matrix(R, mu, sigma_r, tau)
    g, pg = filter_with_matrix(f, K, taps, return_parts=True)
    gh, _ = filter_with_matrix(f, Kh, taps, return_parts=True)
    dmax = np.max(np.abs(Kh - K))
    fmax = np.max(np.linalg.norm(f.reshape(-1, n), axis=1))
    err = np.linalg.norm(gh - g, axis=2)
    bound = pg["wsum"] * dmax * (np.linalg.norm(gh, axis=2) + fmax) / pg["eta"]
    return err, bound, dict(K=K, Kh=Kh, g=g, g_hat=gh, eta=pg["eta"])


def theorem1_final(f_range_R: float, n: int, S: int, d: int, Kmat, Khat, kappa00=1.0) -> float:
    """(2 / kappa(0,0)) (2S+1)^d R sqrt(n) ||K-hat - K||_F (omega(0) cancels)."""
    return (2.0 / kappa00) * (2 * S + 1) ** d * f_range_R * np.sqrt(n) * \
        np.linalg.norm(Khat - Kmat, "fro")
