"""Parity at the full workload sizes, in the launch configuration the benchmark
times: the CUDA path on the whole image, the FP64 oracle at sampled pixels
(direct window sums, Eqs. (14)-(15)), both with the oracle's own k-means
landmarks.  Backward at full size: with dL/dg_hat supported on a window, the
gradient equals the oracle's on the window grown by S (exact); over the whole
image, a directional derivative is checked against central differences of
the CUDA forward (FP32 forward: h and tolerance sized for its rounding)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def sample_pixels(H, W, count, seed):
    """Seeded interior samples plus the four corners and edge midpoints."""
    idx = synth.sample_indices(H * W, count, seed)
    ys, xs = list(idx // W), list(idx % W)
    for y, x in [(0, 0), (0, W - 1), (H - 1, 0), (H - 1, W - 1), (0, W // 2), (H // 2, 0),
                 (H - 1, W // 2), (H // 2, W - 1)]:
        ys.append(y)
        xs.append(x)
    return np.array(ys), np.array(xs)


def _params(nyf, w, **kw):
    P = nyf.Params(sigma_s=w.sigma_s, sigma_r=float(np.float32(w.sigma_r)), K=w.K,
                   kmeans_iters=w.kmeans_iters, seed=w.seed, spatial=w.spatial, S=w.S,
                   patch_radius=w.patch_radius, sample_frac=w.sample_frac)
    for k, v in kw.items():
        setattr(P, k, v)
    return P


@pytest.fixture(scope="module")
def hd():
    w = synth.colour_blf_hd()
    mu, info = pl.landmarks(w.f.reshape(-1, 3).astype(np.float64), w.K, w.kmeans_iters, w.seed)
    return w, mu.astype(np.float32), info


def test_colour_1920x1080_sampled_parity(nyf, hd):
    w, mu, _ = hd
    P = _params(nyf, w)
    out = nyf.blf(cuda(w.f), P, landmarks=cuda(mu)).cpu().numpy()
    ys, xs = sample_pixels(w.H, w.W, 300, 11)
    want = ny.nystrom_filter_at(w.f, w.f, mu.astype(np.float64), P.sigma_r,
                                Kr.gaussian_taps(w.sigma_s, w.radius), 1e-7, ys, xs)
    r, _ = report("colour 1920x1080 K=32 (300 samples)", out[ys, xs], want)
    assert r < FP32_REL_RMSE


def test_colour_1920x1080_device_kmeans(nyf, hd):
    w, mu_o, info = hd
    P = _params(nyf, w)
    ws = nyf.make_workspace(w.H, w.W, 3, 3, P)
    nyf.blf(cuda(w.f), P, ws=ws)
    st = nyf.stats(ws)
    print(f"[parity] 1920x1080 k-means e: gpu={st['qerr']:.6e} oracle={info['e']:.6e}")
    assert st["status"] == 0 and st["rank"] == w.K and st["eta_small"] == 0
    assert abs(st["qerr"] - info["e"]) <= 1e-3 * info["e"]


def test_hyperspectral_512x512x31_sampled_parity(nyf):
    w = synth.hyperspectral_blf()
    X = w.f.reshape(-1, 31).astype(np.float64)
    mu, info = pl.landmarks(X, w.K, w.kmeans_iters, w.seed)
    mu = mu.astype(np.float32)
    P = _params(nyf, w)
    ws = nyf.make_workspace(w.H, w.W, 31, 31, P)
    out = nyf.blf(cuda(w.f), P, landmarks=cuda(mu), ws=ws).cpu().numpy()
    st = nyf.stats(ws)
    ys, xs = sample_pixels(w.H, w.W, 120, 12)
    want = ny.nystrom_filter_at(w.f, w.f, mu.astype(np.float64), P.sigma_r,
                                Kr.gaussian_taps(w.sigma_s, w.radius), 1e-7, ys, xs)
    print(f"[parity] hyperspectral rank={st['rank']} alpha_min_kept/max="
          f"{st['alpha_min_kept'] / st['alpha_max']:.3e} eta_small={st['eta_small']}")
    r, _ = report("hyperspectral 512x512x31 K=64 (120 samples)", out[ys, xs], want)
    assert r < FP32_REL_RMSE


def test_nlm_768x512_sampled_parity(nyf):
    w = synth.colour_nlm()
    X, idx, p = pl.nlm_sample_rows(w.f.astype(np.float64), w.patch_radius, w.sample_frac, w.seed)
    mu, _ = pl.landmarks(X, w.K, w.kmeans_iters, w.seed)
    mu = mu.astype(np.float32)
    P = _params(nyf, w)
    out = nyf.nlm(cuda(w.f), P, landmarks=cuda(mu)).cpu().numpy()
    ys, xs = sample_pixels(w.H, w.W, 150, 13)
    want = ny.nystrom_filter_at(w.f, p, mu.astype(np.float64), P.sigma_r, Kr.box_taps(w.S), 1e-7,
                                ys, xs)
    r, _ = report("nlm 768x512 K=32 (150 samples)", out[ys, xs], want)
    assert r < FP32_REL_RMSE
    # device k-means on the same subsample reaches the same objective
    ws = nyf.make_workspace(w.H, w.W, 3, 75, P)
    nyf.nlm(cuda(w.f), P, ws=ws)
    st = nyf.stats(ws)
    _, info = pl.landmarks(X, w.K, w.kmeans_iters, w.seed)
    print(f"[parity] nlm k-means e: gpu={st['qerr']:.6e} oracle={info['e']:.6e}")
    assert st["status"] == 0 and abs(st["qerr"] - info["e"]) <= 1e-3 * info["e"]


@pytest.mark.parametrize("mode", ["planes", "recompute"])
def test_colour_1920x1080_backward_vs_oracle_on_a_window(nyf, hd, mode):
    # G = dL/d g_hat is nonzero only on a window R; g_hat on R depends only on the
    # image inside R grown by S, so the oracle gradient on that crop is exact.
    # mode "recompute": the low-memory backward (C_kq convolved again, 4 modes at a time).
    from oracle import grad as gr
    w, mu, _ = hd
    S = w.radius
    y0, x0, h = 520, 911, 40
    G = np.zeros(w.f.shape, np.float32)
    G[y0:y0 + h, x0:x0 + h] = np.random.default_rng(7).normal(size=(h, h, 3))
    sr = float(np.float32(w.sigma_r))
    res = nyf.blf_vjp(cuda(w.f), nyf.Params(sigma_s=w.sigma_s, sigma_r=sr, K=w.K, backward_mode=mode),
                      cuda(G), landmarks=cuda(mu))
    c0, c1 = (y0 - S, y0 + h + S), (x0 - S, x0 + h + S)
    crop = w.f[c0[0]:c0[1], c1[0]:c1[1]]
    ref = gr.vjp(crop, crop, mu, sr, w.sigma_s, S, 1e-7, G[c0[0]:c0[1], c1[0]:c1[1]],
                 guide_is_image=True)
    df = res["df"].cpu().numpy()
    r, _ = report("full-size grad f on the window crop", df[c0[0]:c0[1], c1[0]:c1[1]], ref["df"])
    assert r < 1e-3
    outside = np.abs(df).copy()
    outside[c0[0]:c0[1], c1[0]:c1[1]] = 0
    assert outside.max() == 0.0                       # no gradient leaks outside the crop
    for nm in ("dsigma_r", "dsigma_s"):
        rel = abs(res[nm] - ref[nm]) / abs(ref[nm])
        print(f"[parity] full-size {nm}: gpu={res[nm]:.6e} oracle={ref[nm]:.6e} rel={rel:.2e}")
        assert rel < 1e-3


def test_colour_1920x1080_backward_directional_derivative(nyf, hd):
    w, mu, _ = hd
    ft, mut = cuda(w.f), cuda(mu)
    G = torch.randn(ft.shape, generator=torch.Generator().manual_seed(5)).cuda()
    sr, ss = float(np.float32(w.sigma_r)), w.sigma_s
    P = nyf.Params(sigma_s=ss, sigma_r=sr, K=w.K)

    def loss(f_):
        return float((nyf.blf(f_, P, landmarks=mut).double() * G.double()).sum())

    res = nyf.blf_vjp(ft, P, G, landmarks=mut)
    v = torch.randn(ft.shape, generator=torch.Generator().manual_seed(6)).cuda()
    h = 0.5
    fd_v = (loss(ft + h * v) - loss(ft - h * v)) / (2 * h)
    dv = float((res["df"].double() * v.double()).sum())
    print(f"[parity] full-size <df, v>: gpu={dv:.6e} fd={fd_v:.6e}")
    assert abs(dv - fd_v) <= 2e-3 * abs(fd_v)
