"""Parity of the recursive-Gaussian path (spatial = "gaussian_iir": Young & van
Vliet's O(1) filter for omega, Sec. IV) with the FP64 oracle (oracle.iir),
through the C ABI; and its distance from the truncated FIR Gaussian."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import guide as gd
from oracle import iir
from oracle import kernels as Kr
from oracle import nystrom as ny
from oracle import pipeline as pl
from paper_1901_06112_gb300 import synth
from tests._util import FP32_REL_RMSE, report

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nyf():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1901_06112_gb300 import build
    build.build()
    from paper_1901_06112_gb300 import nyf as N
    return N


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _landmarks(X, K, seed=3):
    # k-means landmarks (5 Lloyd steps of the oracle): they cover the image's
    # colours, so eta-hat (Eq. (15)) stays away from zero and the FP32 ratio is
    # well conditioned; uniform draws of few landmarks can leave pixels with
    # eta-hat ~ 0, where the oracle's own g-hat is meaningless
    K = min(K, X.shape[0])
    mu, _ = pl.landmarks(np.asarray(X, np.float64), K, 5, seed)
    return mu.astype(np.float32)


def _oracle(f, p, mu, sigma_r, sigma_s):
    g, parts = iir.nystrom_filter_iir(f, p, mu.astype(np.float64), sigma_r, sigma_s, 1e-7,
                                      return_parts=True)
    assert parts["eta"].min() > 0.0        # the premise of an FP32 comparison
    return g


def test_blf_colour_256(nyf):
    w = synth.colour_blf_small()
    mu, _ = pl.landmarks(w.f.reshape(-1, 3).astype(np.float64), w.K, 10, w.seed)
    mu = mu.astype(np.float32)
    want = iir.nystrom_filter_iir(w.f, w.f, mu.astype(np.float64), w.sigma_r, w.sigma_s, 1e-7)
    P = nyf.Params(sigma_s=w.sigma_s, sigma_r=w.sigma_r, K=w.K, spatial="gaussian_iir")
    ws = nyf.make_workspace(w.H, w.W, 3, 3, P)
    out = nyf.blf(cuda(w.f), P, landmarks=cuda(mu), ws=ws)
    st = nyf.stats(ws)
    assert st["status"] == 0 and st["eta_small"] == 0
    r, m = report("iir blf 256x256 K=8", out.cpu().numpy(), want)
    assert r < FP32_REL_RMSE and m < 0.05
    # the recursive filter is within the method's accuracy of the FIR Gaussian
    fir = ny.nystrom_filter(w.f, w.f, mu.astype(np.float64), w.sigma_r,
                            Kr.gaussian_taps(w.sigma_s, w.radius), 1e-7)
    d = np.sqrt(np.mean((want - fir) ** 2) / np.mean(fir ** 2))
    print(f"[iir] 256x256 sigma_s {w.sigma_s}: recursive vs FIR Gaussian rel RMSE {d:.3e}")
    assert d < 0.02


@pytest.mark.parametrize("H,W,sigma_s,K", [(1, 1, 1.0, 1), (1, 57, 2.0, 3), (43, 1, 1.5, 2),
                                           (37, 53, 0.5, 5), (5, 7, 4.0, 4), (97, 131, 5.6, 6),
                                           (70, 66, 8.0, 8), (40, 45, 20.0, 3), (33, 2016, 3.0, 4),
                                           (2016, 21, 2.5, 4), (64, 1920, 5.0, 6)])
def test_blf_ragged_and_edge_sizes(nyf, H, W, sigma_s, K):
    f = synth.voronoi_colour(H, W, 12, 8.0, H * 1000 + W)
    mu = _landmarks(f.reshape(-1, 3), K)
    want = _oracle(f, f, mu, 45.0, sigma_s)
    P = nyf.Params(sigma_s=sigma_s, sigma_r=45.0, K=mu.shape[0], spatial="gaussian_iir")
    out = nyf.blf(cuda(f), P, landmarks=cuda(mu))
    r, _ = report(f"iir blf {H}x{W} sigma_s={sigma_s} K={mu.shape[0]}", out.cpu().numpy(), want)
    assert r < FP32_REL_RMSE


@pytest.mark.parametrize("H,W,n", [(24, 1900, 9), (40, 200, 31), (30, 90, 17)])
def test_many_channels_split_combine(nyf, H, W, n):
    # more quantities than one CTA's warps: zeta goes through the workspace
    r_ = np.random.default_rng(H + W + n)
    f = (r_.uniform(0, 255, size=(H, W, n))).astype(np.float32)
    g = synth.voronoi_colour(H, W, 9, 6.0, 77 + n)
    mu = _landmarks(g.reshape(-1, 3), 6)
    want = _oracle(f, g, mu, 50.0, 3.0)
    P = nyf.Params(sigma_s=3.0, sigma_r=50.0, K=6, spatial="gaussian_iir")
    out = nyf.blf(cuda(f), P, guide=cuda(g), landmarks=cuda(mu))
    r, _ = report(f"iir joint blf {H}x{W} n={n}", out.cpu().numpy(), want)
    assert r < FP32_REL_RMSE


def test_nlm_patch_guide(nyf):
    f = synth.voronoi_colour(48, 52, 10, 12.0, 5)
    p = gd.patch_guide(f.astype(np.float64), 1)
    mu = _landmarks(p.reshape(-1, p.shape[2]), 7, seed=9)
    want = _oracle(f, p, mu, 80.0, 2.0)
    P = nyf.Params(sigma_s=2.0, sigma_r=80.0, K=7, spatial="gaussian_iir", patch_radius=1)
    out = nyf.nlm(cuda(f), P, landmarks=cuda(mu))
    r, _ = report("iir nlm 48x52 r=1 K=7", out.cpu().numpy(), want)
    assert r < FP32_REL_RMSE


def test_constant_image_and_infinite_sigma_r(nyf):
    f = np.full((50, 61, 3), 91.0, np.float32)
    mu = np.random.default_rng(2).uniform(0, 255, size=(4, 3)).astype(np.float32)
    out = nyf.blf(cuda(f), nyf.Params(sigma_s=3.0, sigma_r=40.0, K=4, spatial="gaussian_iir"),
                  guide=cuda(synth.random_image(50, 61, 3, 4)), landmarks=cuda(mu))
    assert np.allclose(out.cpu().numpy(), 91.0, rtol=2e-6)
    f = synth.random_image(45, 70, 3, 8).astype(np.float32)
    out = nyf.blf(cuda(f), nyf.Params(sigma_s=2.5, sigma_r=1e6 * 255, K=4, spatial="gaussian_iir"),
                  landmarks=cuda(mu[:4]))
    want = iir.iir_2d(f, 2.5) / iir.iir_2d(np.ones((45, 70)), 2.5)[..., None]
    r, _ = report("iir sigma_r -> inf blur", out.cpu().numpy(), want)
    assert r < FP32_REL_RMSE


def test_full_size_1920x1080_k32(nyf):
    # the 1920 x 1080 colour workload (sigma_s 5, sigma_r 40, K 32) at full size,
    # every pixel compared with the FP64 oracle on the oracle's landmarks
    w = synth.colour_blf_hd()
    mu, _ = pl.landmarks(w.f.reshape(-1, 3).astype(np.float64), w.K, w.kmeans_iters, w.seed)
    mu = mu.astype(np.float32)
    P = nyf.Params(sigma_s=w.sigma_s, sigma_r=w.sigma_r, K=w.K, seed=w.seed, spatial="gaussian_iir")
    ws = nyf.make_workspace(w.H, w.W, 3, 3, P)
    out = nyf.blf(cuda(w.f), P, landmarks=cuda(mu), ws=ws).cpu().numpy()
    st = nyf.stats(ws)
    assert st["status"] == 0 and st["rank"] == w.K and st["eta_small"] == 0
    want = iir.nystrom_filter_iir(w.f, w.f, mu.astype(np.float64), w.sigma_r, w.sigma_s, 1e-7)
    r, _ = report("iir blf 1920x1080 K=32 (all pixels)", out, want)
    assert r < FP32_REL_RMSE


def test_pca_nlm_with_the_recursive_gaussian(nyf):
    # PCA guide (Sec. IV PCA-NLM) with the recursive Gaussian as omega
    from oracle import pca
    w = synth.colour_pca_nlm()
    f = w.f[:64, :80].copy()
    g, m, U = pca.pca_guide(f.astype(np.float64), 2, 10)
    mf, Uf = m.astype(np.float32), U.astype(np.float32)
    g, _, _ = pca.pca_guide(f.astype(np.float64), 2, 10, mf.astype(np.float64), Uf.astype(np.float64))
    mu = _landmarks(g.reshape(-1, 10), 8)
    want = _oracle(f, g, mu, w.sigma_r, 2.0)
    P = nyf.Params(sigma_s=2.0, sigma_r=w.sigma_r, K=8, spatial="gaussian_iir", patch_radius=2)
    out = nyf.pca_nlm(cuda(f), 10, P, mean=cuda(mf), basis=cuda(Uf), landmarks=cuda(mu))
    r, _ = report("pca-nlm 64x80 q=10 with the recursive Gaussian", out.cpu().numpy(), want)
    assert r < FP32_REL_RMSE


def test_batched_recursive_gaussian_equals_single_image_calls(nyf):
    # uneven images with their own sigma_s, sigma_r through the batched entry point
    shapes = [(40, 56), (33, 20), (64, 64)]
    ss, sr = [1.5, 3.0, 5.0], [30.0, 45.0, 25.0]
    imgs = [synth.voronoi_colour(h, w_, 12, 8.0, h * 100 + w_) for h, w_ in shapes]
    P = nyf.Params(K=6, kmeans_iters=5, spatial="gaussian_iir")
    bt = nyf.Batched(shapes, ss, sr, P, backward=False)
    got = bt.unpack(bt.forward(bt.pack(imgs)))
    for b, im in enumerate(imgs):
        Pb = nyf.Params(sigma_s=ss[b], sigma_r=sr[b], K=6, kmeans_iters=5, spatial="gaussian_iir")
        one = nyf.blf(cuda(im), Pb).cpu().numpy()
        r, _ = report(f"batched recursive image {b} vs single call", got[b].cpu().numpy(), one)
        assert r < 1e-6
