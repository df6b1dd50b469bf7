"""The Nystrom kernel filter, step by step in the paper's notation (Sec. III).

Algorithm 1 (Fast Kernel Filtering):

1. form the range list R = {p(x)} (Eq. (2)); the index map iota (Eq. (3)) is the
   row-major pixel index, because R is a list with repetitions, one entry per
   pixel;
2. landmarks mu_1..mu_m0 (k-means, ``oracle.kmeans``; given here as input);
3. A(i, j) = kappa(mu_i, mu_j) (Eq. (9)) and B(i, j) = kappa(mu_i, r_j) (Eq. (11));
4. eigendecomposition A = sum_k alpha_k w_k w_k^T (Eq. (10)), by LAPACK;
5. zeta = 0, eta = 0;
6. for each k: v_k = B^T w_k / alpha_k (Eq. (12)), d_k(x) = v_k(iota(x)),
   h_k(x) = d_k(x) f(x); zeta += alpha_k d_k (omega * h_k);
   eta += alpha_k d_k (omega * d_k);
7. g_hat = zeta / eta, which is Eqs. (14)-(15).

Reading of a point the paper leaves open: Eq. (12) divides by alpha_k, and A is
only positive semi-definite (duplicate landmarks, or sigma_r large, make it
singular).  Only modes with alpha_k > tau * alpha_max are used; tau is an
input shared with the CUDA path.  No clamping of eta is done.

The spatial convolution omega * h (Eq. (7)) is zero padded, i.e. the window is
clipped to Omega, and computed separably (omega(z) = g(z_y) g(z_x)); the
separable sum equals the direct 2-D sum (tests/test_oracle_nystrom.py).

Pinned by: tests/test_oracle_nystrom.py -- constant image returned unchanged
for any landmarks; sigma_r -> infinity gives the normalised blur; few-colour
images with the colours as landmarks and K = N landmarks reproduce Eq. (1)
exactly; the K = 1 closed form; the convolution form equals the explicit
K-hat form (``oracle.bound``); tests/test_oracle_bound.py checks Theorem 1.
"""
from __future__ import annotations

import numpy as np

from .kernels import kappa


# -- Eq. (9), (10), (11), (12) ------------------------------------------------

def landmark_kernel(mu: np.ndarray, sigma_r: float) -> np.ndarray:
    """A(i, j) = kappa(mu_i, mu_j), Eq. (9)."""
    mu = np.asarray(mu, np.float64)
    return kappa(mu[:, None, :], mu[None, :, :], sigma_r)


def eig_desc(A: np.ndarray):
    """Eq. (10): eigenvalues alpha (descending) and eigenvectors w_k (columns)."""
    alpha, W = np.linalg.eigh(np.asarray(A, np.float64))
    order = np.argsort(alpha, kind="stable")[::-1]
    return alpha[order], W[:, order]


def kept_modes(alpha: np.ndarray, tau: float) -> np.ndarray:
    """Indices k with alpha_k > tau * alpha_max (the modes Eq. (12) can divide by)."""
    amax = alpha[0] if alpha.size else 0.0
    if not amax > 0:
        return np.zeros(0, dtype=np.int64)
    return np.nonzero(alpha > tau * amax)[0]


def cross_kernel(mu: np.ndarray, R: np.ndarray, sigma_r: float) -> np.ndarray:
    """B(i, j) = kappa(mu_i, r_j), Eq. (11): m0 x m."""
    mu = np.asarray(mu, np.float64)
    R = np.asarray(R, np.float64)
    B = np.empty((mu.shape[0], R.shape[0]))
    for i in range(mu.shape[0]):
        B[i] = kappa(R, mu[i], sigma_r)
    return B


def extrapolate(B: np.ndarray, w: np.ndarray, alpha_k: float) -> np.ndarray:
    """v_k = (1 / alpha_k) B^T w_k, Eq. (12)."""
    return (B.T @ w) / alpha_k


# -- Eq. (7): the spatial convolution ----------------------------------------

def conv_same(a: np.ndarray, taps: np.ndarray) -> np.ndarray:
    """(omega * a)(x) = sum_z omega(z) a(x - z), zero outside Omega, omega = g (x) g.

    `a` is H x W or H x W x c; the 2-D window is applied along axes 0 and 1.
    """
    a = np.asarray(a, np.float64)
    S = (len(taps) - 1) // 2
    H, W = a.shape[:2]
    t1 = np.zeros_like(a)
    for z in range(-S, S + 1):                      # along y: t1[y] += g(z) a[y - z]
        y0, y1 = max(0, z), min(H, H + z)
        if y0 < y1:
            t1[y0:y1] += taps[z + S] * a[y0 - z:y1 - z]
    out = np.zeros_like(a)
    for z in range(-S, S + 1):                      # along x
        x0, x1 = max(0, z), min(W, W + z)
        if x0 < x1:
            out[:, x0:x1] += taps[z + S] * t1[:, x0 - z:x1 - z]
    return out


def conv_direct(a: np.ndarray, taps: np.ndarray) -> np.ndarray:
    """The same convolution as a direct 2-D window sum (used to pin conv_same)."""
    a = np.asarray(a, np.float64)
    S = (len(taps) - 1) // 2
    H, W = a.shape[:2]
    om = np.outer(taps, taps)
    out = np.zeros_like(a)
    for zy in range(-S, S + 1):
        for zx in range(-S, S + 1):
            y0, y1 = max(0, zy), min(H, H + zy)
            x0, x1 = max(0, zx), min(W, W + zx)
            if y0 < y1 and x0 < x1:
                out[y0:y1, x0:x1] += om[zy + S, zx + S] * a[y0 - zy:y1 - zy, x0 - zx:x1 - zx]
    return out


# -- Algorithm 1 --------------------------------------------------------------

def spectral_step(mu: np.ndarray, sigma_r: float, tau: float):
    """Steps 3-4 on the landmark side: A, its eigenpairs and the kept modes."""
    A = landmark_kernel(mu, sigma_r)
    alpha, W = eig_desc(A)
    keep = kept_modes(alpha, tau)
    return A, alpha, W, keep


def nystrom_filter(f: np.ndarray, p: np.ndarray, mu: np.ndarray, sigma_r: float,
                   taps: np.ndarray, tau: float, return_parts: bool = False, conv=None):
    """Algorithm 1 on the whole image.  f: H x W x n, p: H x W x rho, mu: m0 x rho.

    `conv`, if given, is the spatial filter omega * (.) on H x W (x c) arrays
    (any linear operator, e.g. the recursive Gaussian of ``oracle.iir``); by
    default it is ``conv_same`` with `taps`.
    """
    if conv is None:
        conv = lambda a: conv_same(a, taps)
    f = np.asarray(f, np.float64)
    p = np.asarray(p, np.float64)
    H, W, n = f.shape
    R = p.reshape(H * W, -1)                         # Eq. (2); iota(x) = y * W + x
    _, alpha, Wv, keep = spectral_step(mu, sigma_r, tau)
    if keep.size == 0:
        raise FloatingPointError("no eigenvalue of A above the truncation threshold")
    B = cross_kernel(mu, R, sigma_r)                 # Eq. (11)
    zeta = np.zeros((H, W, n))
    eta = np.zeros((H, W))
    for k in keep:
        v = extrapolate(B, Wv[:, k], alpha[k])       # Eq. (12)
        d = v.reshape(H, W)                          # d_k(x) = v_k(iota(x))
        h = d[..., None] * f                         # h_k(x) = d_k(x) f(x)
        zeta += alpha[k] * d[..., None] * conv(h)
        eta += alpha[k] * d * conv(d)
    g_hat = zeta / eta[..., None]
    if return_parts:
        return g_hat, dict(zeta=zeta, eta=eta, alpha=alpha, W=Wv, keep=keep)
    return g_hat


def nystrom_filter_at(f: np.ndarray, p: np.ndarray, mu: np.ndarray, sigma_r: float,
                      taps: np.ndarray, tau: float, ys: np.ndarray, xs: np.ndarray,
                      return_eta: bool = False):
    """Eqs. (14)-(15) at the listed pixels, each by a direct 2-D window sum.

    Independent of ``conv_same``: for every listed x the sums over y in W_x are
    taken explicitly with v_k evaluated on the window (Eq. (12)).
    """
    f = np.asarray(f, np.float64)
    p = np.asarray(p, np.float64)
    H, W, n = f.shape
    S = (len(taps) - 1) // 2
    _, alpha, Wv, keep = spectral_step(mu, sigma_r, tau)
    if keep.size == 0:
        raise FloatingPointError("no eigenvalue of A above the truncation threshold")
    out = np.empty((len(ys), n))
    etas = np.empty(len(ys))
    for i, (y, x) in enumerate(zip(ys, xs)):
        a0, a1 = max(0, y - S), min(H, y + S + 1)
        b0, b1 = max(0, x - S), min(W, x + S + 1)
        win = p[a0:a1, b0:b1].reshape(-1, p.shape[2])
        om = np.outer(taps[a0 - y + S:a1 - y + S], taps[b0 - x + S:b1 - x + S]).ravel()
        fw = f[a0:a1, b0:b1].reshape(-1, n)
        Bw = cross_kernel(mu, win, sigma_r)          # B restricted to the window
        bx = cross_kernel(mu, p[y, x][None, :], sigma_r)[:, 0]
        zeta = np.zeros(n)
        eta = 0.0
        for k in keep:
            vy = (Bw.T @ Wv[:, k]) / alpha[k]
            vx = (bx @ Wv[:, k]) / alpha[k]
            zeta += alpha[k] * vx * ((om * vy) @ fw)
            eta += alpha[k] * vx * np.sum(om * vy)
        out[i] = zeta / eta
        etas[i] = eta
    if return_eta:
        return out, etas
    return out


def features(p: np.ndarray, mu: np.ndarray, sigma_r: float, tau: float):
    """Per-pixel features phi_k(x) = sqrt(alpha_k) v_k(iota(x)) for the kept modes.

    K-hat = sum_k alpha_k v_k v_k^T = sum_k phi_k phi_k^T (Eq. (8) with Eq. (12)),
    so these are the only per-pixel quantities Eqs. (14)-(15) need.  Returns
    (phi: N x r, alpha: all m0 eigenvalues descending, keep).
    """
    p = np.asarray(p, np.float64)
    R = p.reshape(-1, p.shape[-1])
    _, alpha, Wv, keep = spectral_step(mu, sigma_r, tau)
    B = cross_kernel(mu, R, sigma_r)
    phi = np.stack([np.sqrt(alpha[k]) * extrapolate(B, Wv[:, k], alpha[k]) for k in keep], axis=1) \
        if keep.size else np.zeros((R.shape[0], 0))
    return phi, alpha, keep


def features_symmetric(p: np.ndarray, mu: np.ndarray, sigma_r: float, tau: float):
    """Features for the symmetric factor of the truncated inverse of A.

    phi_j(x) = sum_m B(m, x) W[m, j] with W = W_r Lambda_r^{-1/2} W_r^T, so that
    Phi Phi^T = B^T W_r Lambda_r^{-1} W_r^T B = sum_k alpha_k v_k v_k^T = K-hat
    (Eq. (8) with Eq. (12)).  Unlike ``features`` this factor is unique.
    Returns (phi: N x m0, alpha, keep).
    """
    p = np.asarray(p, np.float64)
    R = p.reshape(-1, p.shape[-1])
    _, alpha, Wv, keep = spectral_step(mu, sigma_r, tau)
    Wr = Wv[:, keep]
    Wsym = (Wr / np.sqrt(alpha[keep])) @ Wr.T
    return cross_kernel(mu, R, sigma_r).T @ Wsym, alpha, keep
