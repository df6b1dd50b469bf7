"""FP64 gradients of the Nystrom filter (the paper gives no gradients).

The forward below is Algorithm 1 again -- Eqs. (9)-(12), (14)-(15) -- written
with PyTorch CPU float64 tensor operations so that autograd yields the exact
derivative of g_hat with respect to the image f, the guide p, sigma_r and
sigma_s.  Readings for what the paper does not cover:

* the landmarks mu are held fixed (k-means is not differentiated);
* the window radius S is held at its forward value when sigma_s varies;
* the set of kept modes (alpha_k > tau alpha_max) is held fixed;
* omega is the unnormalised Gaussian, so d omega / d sigma_s includes the
  change of its mass (the scale cancels in g_hat anyway).

``vjp`` returns the gradient of sum(G * g_hat) for a given cotangent G.

Pinned by: tests/test_oracle_grad.py (forward equals ``nystrom.nystrom_filter``
to 1e-12; every gradient equals central finite differences of the NumPy
oracle to 1e-6 relative).
"""
from __future__ import annotations

import numpy as np
import torch


def _conv_same(a: torch.Tensor, taps: torch.Tensor) -> torch.Tensor:
    """Zero-padded separable convolution of an H x W x c tensor (Eq. (7))."""
    S = (taps.shape[0] - 1) // 2
    H, W = a.shape[0], a.shape[1]
    ap = torch.nn.functional.pad(a, (0, 0, 0, 0, S, S))          # pad along y
    t1 = sum(taps[z + S] * ap[S - z:S - z + H] for z in range(-S, S + 1))
    tp = torch.nn.functional.pad(t1, (0, 0, S, S))               # pad along x
    return sum(taps[z + S] * tp[:, S - z:S - z + W] for z in range(-S, S + 1))


def nystrom_filter_t(f, p, mu, sigma_r, sigma_s, S, tau, spatial="gaussian", keep=None):
    """Algorithm 1 in torch float64.  Returns (g_hat, keep)."""
    H, W, n = f.shape
    t = torch.arange(-S, S + 1, dtype=torch.float64)
    if spatial == "box":
        taps = torch.ones(2 * S + 1, dtype=torch.float64)
    else:
        taps = torch.exp(-(t * t) / (2.0 * sigma_s * sigma_s))
    dmu = mu[:, None, :] - mu[None, :, :]
    A = torch.exp(-(dmu * dmu).sum(-1) / (2.0 * sigma_r * sigma_r))          # Eq. (9)
    alpha, Wv = torch.linalg.eigh(A)                                         # Eq. (10)
    alpha = torch.flip(alpha, [0])
    Wv = torch.flip(Wv, [1])
    if keep is None:
        a = alpha.detach()
        keep = [k for k in range(a.shape[0]) if a[k] > tau * a[0]]
    R = p.reshape(H * W, -1)
    dr = mu[:, None, :] - R[None, :, :]
    B = torch.exp(-(dr * dr).sum(-1) / (2.0 * sigma_r * sigma_r))           # Eq. (11)
    zeta = torch.zeros((H, W, n), dtype=torch.float64)
    eta = torch.zeros((H, W, 1), dtype=torch.float64)
    for k in keep:
        v = (B.T @ Wv[:, k]) / alpha[k]                                      # Eq. (12)
        d = v.reshape(H, W, 1)
        zeta = zeta + alpha[k] * d * _conv_same(d * f, taps)
        eta = eta + alpha[k] * d * _conv_same(d, taps)
    return zeta / eta, keep


def vjp(f, p, mu, sigma_r, sigma_s, S, tau, G, spatial="gaussian", guide_is_image=False):
    """Gradients of sum(G * g_hat) w.r.t. f, p, sigma_r, sigma_s (float64 NumPy out).

    guide_is_image=True ties p to f (standard BLF): the returned df is then the
    total derivative and dp is None.
    """
    ft = torch.tensor(np.asarray(f, np.float64), requires_grad=True)
    pt = ft if guide_is_image else torch.tensor(np.asarray(p, np.float64), requires_grad=True)
    sr = torch.tensor(float(sigma_r), dtype=torch.float64, requires_grad=True)
    ss = torch.tensor(float(sigma_s), dtype=torch.float64, requires_grad=True)
    mut = torch.tensor(np.asarray(mu, np.float64))
    g, _ = nystrom_filter_t(ft, pt, mut, sr, ss, S, tau, spatial)
    (g * torch.tensor(np.asarray(G, np.float64))).sum().backward()
    df = ft.grad.numpy().copy()
    dp = None if guide_is_image else pt.grad.numpy().copy()
    dss = float(ss.grad) if (spatial != "box" and ss.grad is not None) else 0.0
    return dict(df=df, dp=dp, dsigma_r=float(sr.grad), dsigma_s=dss, g=g.detach().numpy())
