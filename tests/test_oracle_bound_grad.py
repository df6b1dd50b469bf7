"""Pins for oracle.bound (Theorem 1, Proposition 1 trend) and oracle.grad (FP64 gradients)."""
import numpy as np
import pytest

from oracle import bound as bd
from oracle import grad as gr
from oracle import kernels as K
from oracle import kmeans as km
from oracle import nystrom as ny
from oracle import rng
from paper_1901_06112_gb300 import synth


@pytest.mark.parametrize("K_,seed", [(2, 30), (4, 31), (8, 32)])
def test_theorem1_pointwise_bound_holds(K_, seed):
    f = synth.random_image(8, 8, 3, seed).astype(np.float64)
    X = f.reshape(-1, 3)
    mu, _, _, _ = km.kmeans(X, X[rng.distinct_indices(seed, K_, 64)], 5)
    taps = K.gaussian_taps(1.0, 3)
    err, bound, parts = bd.theorem1_pointwise(f, f, mu, 80.0, taps, 1e-10)
    assert np.all(err <= bound * (1 + 1e-9) + 1e-12)
    # the explicit-matrix g-hat is Algorithm 1's output
    assert np.allclose(parts["g_hat"], ny.nystrom_filter(f, f, mu, 80.0, taps, 1e-10), rtol=1e-9)
    if np.all(np.linalg.norm(parts["g_hat"], axis=2) <= 255.0 * np.sqrt(3)):
        fin = bd.theorem1_final(255.0, 3, 3, 2, parts["K"], parts["Kh"])
        assert err.max() <= fin


def test_exact_landmarks_give_zero_error():
    f = synth.random_image(6, 6, 3, 33).astype(np.float64)
    err, bound, _ = bd.theorem1_pointwise(f, f, f.reshape(-1, 3), 5.0, K.gaussian_taps(1.0, 2), 1e-14)
    assert err.max() < 1e-8 and bound.max() < 1e-6


def test_proposition1_trend_with_more_landmarks():
    # parity unpinned: c1, c2 are not given; only the trend (error falls as m0 grows) is checked
    errs, qs = [], []
    for K_ in (2, 4, 8, 16):
        e_sum, k_sum = 0.0, 0.0
        for s in range(5):
            f = synth.voronoi_colour(16, 16, 12, 8.0, 40 + s).astype(np.float64)
            X = f.reshape(-1, 3)
            mu, _, e, _ = km.kmeans(X, X[rng.distinct_indices(s, K_, X.shape[0])], 10)
            Kh = bd.nystrom_matrix(X, mu, 50.0, 1e-10)
            k_sum += np.linalg.norm(Kh - bd.kernel_matrix(X, 50.0))
            e_sum += e
        qs.append(e_sum)
        errs.append(k_sum)
    assert all(b < a for a, b in zip(qs, qs[1:]))
    assert all(b < a for a, b in zip(errs, errs[1:]))


def _setup(seed, H=7, W=6):
    f = synth.voronoi_colour(H, W, 4, 20.0, seed).astype(np.float64)
    g = synth.random_image(H, W, 2, seed + 1).astype(np.float64)
    mu = np.random.default_rng(seed).uniform(0, 255, size=(4, 2))
    G = np.random.default_rng(seed + 2).normal(size=(H, W, 3))
    return f, g, mu, G


def test_torch_forward_equals_numpy():
    import torch
    f, g, mu, _ = _setup(50)
    out, _ = gr.nystrom_filter_t(torch.tensor(f), torch.tensor(g), torch.tensor(mu),
                                 torch.tensor(70.0, dtype=torch.float64),
                                 torch.tensor(1.3, dtype=torch.float64), 3, 1e-10)
    want = ny.nystrom_filter(f, g, mu, 70.0, K.gaussian_taps(1.3, 3), 1e-10)
    assert np.allclose(out.numpy(), want, rtol=1e-12)


def _loss(f, g, mu, sr, ss, G, S=3):
    return float(np.sum(G * ny.nystrom_filter(f, g, mu, sr, K.gaussian_taps(ss, S), 1e-10)))


def test_gradients_match_central_differences():
    f, g, mu, G = _setup(51)
    sr, ss = 70.0, 1.3
    out = gr.vjp(f, g, mu, sr, ss, 3, 1e-10, G)
    h = 1e-4
    rel = lambda a, b: abs(a - b) / max(abs(b), 1e-8)
    for (y, x, c) in [(0, 0, 0), (3, 2, 1), (6, 5, 2), (2, 4, 0)]:
        fp, fm = f.copy(), f.copy()
        fp[y, x, c] += h
        fm[y, x, c] -= h
        fd = (_loss(fp, g, mu, sr, ss, G) - _loss(fm, g, mu, sr, ss, G)) / (2 * h)
        assert rel(out["df"][y, x, c], fd) < 1e-6
    for (y, x, c) in [(1, 1, 0), (5, 3, 1)]:
        gp, gm = g.copy(), g.copy()
        gp[y, x, c] += h
        gm[y, x, c] -= h
        fd = (_loss(f, gp, mu, sr, ss, G) - _loss(f, gm, mu, sr, ss, G)) / (2 * h)
        assert rel(out["dp"][y, x, c], fd) < 1e-6
    fd = (_loss(f, g, mu, sr + h, ss, G) - _loss(f, g, mu, sr - h, ss, G)) / (2 * h)
    assert rel(out["dsigma_r"], fd) < 1e-6
    hs = 1e-5
    fd = (_loss(f, g, mu, sr, ss + hs, G) - _loss(f, g, mu, sr, ss - hs, G)) / (2 * hs)
    assert rel(out["dsigma_s"], fd) < 1e-6


def test_blf_total_derivative_when_guide_is_image():
    f, _, _, G = _setup(52)
    mu = np.random.default_rng(53).uniform(0, 255, size=(4, 3))
    out = gr.vjp(f, f, mu, 80.0, 1.2, 3, 1e-10, G, guide_is_image=True)
    h = 1e-4
    y, x, c = 3, 3, 1
    fp, fm = f.copy(), f.copy()
    fp[y, x, c] += h
    fm[y, x, c] -= h
    fd = (_loss(fp, fp, mu, 80.0, 1.2, G) - _loss(fm, fm, mu, 80.0, 1.2, G)) / (2 * h)
    assert abs(out["df"][y, x, c] - fd) <= 1e-6 * abs(fd) + 1e-10
