"""Parity of the CUDA forward path (k-means, eigendecomposition, features,
convolution + combine, BLF and NLM) with the FP64 oracle, through the C ABI."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import bruteforce as bf
from oracle import guide as gd
from oracle import kernels as Kr
from oracle import kmeans as km
from oracle import nystrom as ny
from oracle import pipeline as pl
from oracle import rng
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


def oracle_landmarks(X, K, iters, seed):
    mu, info = pl.landmarks(np.asarray(X, np.float64), K, iters, seed)
    return mu.astype(np.float32), info


# ---------------------------------------------------------------- k-means

def test_device_init_draw_matches_splitmix64(nyf):
    X = synth.random_image(37, 29, 3, 1).reshape(-1, 3)
    for seed, K in [(0, 8), (12345, 33), (2 ** 63 + 7, 64)]:
        cent, _, _ = nyf.kmeans(cuda(X), K, iters=0, seed=seed)
        want = X[rng.distinct_indices(seed, K, X.shape[0])]
        assert np.array_equal(cent.cpu().numpy(), want)


def test_kmeans_separated_clusters_exact(nyf):
    cols = np.array([[10, 10, 10], [200, 30, 30], [30, 200, 30], [30, 30, 200], [220, 220, 220],
                     [120, 120, 40]], float)
    r = np.random.default_rng(3)
    X = (cols[r.integers(0, 6, size=50_000)] + r.normal(0, 4, size=(50_000, 3))).astype(np.float32)
    init = rng.distinct_indices(5, 6, X.shape[0])
    mu_o, c_o, e_o, _ = km.kmeans(X.astype(np.float64), X[init].astype(np.float64), 8)
    cent, labels, qerr = nyf.kmeans(cuda(X), 6, iters=8, init_idx=torch.from_numpy(init))
    assert np.array_equal(labels.cpu().numpy(), c_o)
    report("kmeans centroids (separated)", cent.cpu().numpy(), mu_o)
    assert np.allclose(cent.cpu().numpy(), mu_o, rtol=2e-6, atol=1e-4)
    assert abs(float(qerr.cpu()) - e_o) <= 1e-4 * e_o


def test_kmeans_one_step_unique_labels_match(nyf):
    w = synth.colour_blf_small()
    X = w.f.reshape(-1, 3)
    init = rng.distinct_indices(w.seed, 8, X.shape[0])
    cent, labels, qerr = nyf.kmeans(cuda(X), 8, iters=1, init_idx=torch.from_numpy(init))
    mu_o, _, _, _ = km.kmeans(X.astype(np.float64), X[init].astype(np.float64), 1)
    report("kmeans 1 step", cent.cpu().numpy(), mu_o)
    assert np.allclose(cent.cpu().numpy(), mu_o, rtol=1e-5, atol=1e-3)
    # labels are unique wherever the oracle's best and second-best distances differ clearly
    D = km.sq_dists(X, mu_o)
    part = np.sort(D, axis=1)
    unique = (part[:, 1] - part[:, 0]) > 1e-2 * (1.0 + part[:, 0])
    lab_o = np.argmin(D, axis=1)
    got = labels.cpu().numpy()
    assert np.array_equal(got[unique], lab_o[unique])
    # the rest are valid: within rounding of the best
    rest = ~unique
    assert np.all(D[rest, got[rest]] <= part[rest, 0] * (1 + 1e-2) + 1e-2)


def test_kmeans_ten_iterations_objective(nyf):
    w = synth.colour_blf_small()
    X = w.f.reshape(-1, 3)
    init = rng.distinct_indices(w.seed, 8, X.shape[0])
    cent, labels, qerr = nyf.kmeans(cuda(X), 8, iters=10, init_idx=torch.from_numpy(init))
    _, _, e_o, _ = km.kmeans(X.astype(np.float64), X[init].astype(np.float64), 10)
    print(f"[parity] kmeans e: gpu={float(qerr.cpu()):.6e} oracle={e_o:.6e}")
    assert abs(float(qerr.cpu()) - e_o) <= 1e-3 * e_o


@pytest.mark.parametrize("rho,K,N", [(31, 16, 1000), (75, 32, 3932), (25, 31, 777), (80, 64, 4200)])
def test_kmeans_tensor_cores_match_oracle(nyf, rho, K, N):
    # 16 <= rho <= 80: distances and per-cluster sums on the tensor cores (N not a
    # multiple of the 128-row tile)
    r = np.random.default_rng(rho + K)
    C = r.uniform(0, 1, size=(K + 3, rho))
    X = (C[r.integers(0, K + 3, size=N)] + r.normal(0, 0.08, size=(N, rho))).astype(np.float32)
    init = rng.distinct_indices(7, K, N)
    # one step: centroids equal the oracle's where the labels are unique
    cent1, labels1, _ = nyf.kmeans(cuda(X), K, iters=1, init_idx=torch.from_numpy(init))
    mu1, _, _, _ = km.kmeans(X.astype(np.float64), X[init].astype(np.float64), 1)
    rr, _ = report(f"tensor-core kmeans 1 step rho={rho} K={K}", cent1.cpu().numpy(), mu1)
    assert rr < 1e-6
    # labels of the final centroids: the oracle's wherever its best distance is unique,
    # within rounding of the best elsewhere
    D = km.sq_dists(X.astype(np.float64), cent1.cpu().numpy().astype(np.float64))
    srt = np.sort(D, axis=1)
    unique = (srt[:, 1] - srt[:, 0]) > 1e-5 * (1.0 + srt[:, 0])
    got = labels1.cpu().numpy()
    assert np.array_equal(got[unique], np.argmin(D, axis=1)[unique])
    assert np.all(D[~unique, got[~unique]] <= srt[~unique, 0] * (1 + 1e-5) + 1e-5)
    # ten iterations: the objective
    _, _, qerr = nyf.kmeans(cuda(X), K, iters=10, init_idx=torch.from_numpy(init))
    _, _, e_o, _ = km.kmeans(X.astype(np.float64), X[init].astype(np.float64), 10)
    print(f"[parity] tensor-core kmeans e: gpu={float(qerr.cpu()):.6e} oracle={e_o:.6e}")
    assert abs(float(qerr.cpu()) - e_o) <= 1e-4 * e_o


# ---------------------------------------------------------------- eig + features

@pytest.mark.parametrize("K,sigma_r,rho", [(8, 30.0, 3), (32, 40.0, 3), (64, 0.15, 31), (1, 50.0, 3)])
def test_features_match_oracle(nyf, K, sigma_r, rho):
    if rho == 31:
        f = synth.hyperspectral(48, 40, 31, 6, 10.0, 0.02, 7)
    else:
        f = synth.voronoi_colour(48, 40, 60, 10.0, 8)
    X = f.reshape(-1, rho)
    mu, _ = oracle_landmarks(X, K, 5, 11)
    sigma_r = float(np.float32(sigma_r))       # the C ABI takes sigma_r as float32
    phi, rank, alphas = nyf.features(cuda(X), cuda(mu), sigma_r, 1e-7)
    _, alpha_o, W_o, keep = ny.spectral_step(mu.astype(np.float64), sigma_r, 1e-7)
    r = int(rank.cpu())
    assert r == keep.size
    a = alphas.cpu().numpy()
    assert np.allclose(a, alpha_o, rtol=0, atol=1e-12 * alpha_o[0])
    phi_o, _, _ = ny.features_symmetric(X.astype(np.float64), mu.astype(np.float64), sigma_r, 1e-7)
    got = phi.cpu().numpy().T
    rr, _ = report(f"features K={K} rho={rho}", got, phi_o)
    assert rr < 1e-5


def _tc_guide(kind, seed):
    """Guides of dimension >= 16 (the tensor-core features path) and their sigma_r."""
    from oracle import guide as gd
    from oracle import pca as pc
    if kind == "patch75":             # 5x5x3 NLM patches, 37 x 41 (N = 1517: ragged last tile)
        g = synth.voronoi_colour(37, 41, 20, 20.0, seed, ramp=0.1)
        return gd.patch_guide(g.astype(np.float64), 2).reshape(-1, 75), 20.0 * np.sqrt(75.0)
    if kind == "pca25":               # 7x7x3 patches projected on 25 principal directions
        g = synth.voronoi_colour(40, 36, 20, 20.0, seed, ramp=0.1)
        return pc.pca_guide(g.astype(np.float64), 3, 25)[0].reshape(-1, 25), 424.0
    if kind == "rho16":               # N = 117 < one 128-pixel tile
        return synth.random_image(9, 13, 16, seed, R=1.0).reshape(-1, 16), 0.9
    if kind == "rho47":
        return synth.hyperspectral(25, 40, 47, 5, 8.0, 0.02, seed).reshape(-1, 47), 0.2
    if kind == "rho160":              # the largest guide dimension
        return synth.hyperspectral(20, 15, 160, 4, 6.0, 0.02, seed).reshape(-1, 160), 0.4
    raise ValueError(kind)


@pytest.mark.parametrize("kind,K", [("patch75", 32), ("pca25", 31), ("rho16", 5), ("rho47", 17),
                                    ("rho160", 64), ("rho160", 1)])
def test_features_tensor_cores_match_oracle(nyf, kind, K):
    # rho >= 16: distances and E W_hat on the tensor cores (three-term bf16 split)
    X, sigma_r = _tc_guide(kind, 40 + K)
    X = np.ascontiguousarray(X, np.float32)
    mu, _ = oracle_landmarks(X, K, 5, 13)
    sigma_r = float(np.float32(sigma_r))
    phi, rank, alphas = nyf.features(cuda(X), cuda(mu), sigma_r, 1e-7)
    _, alpha_o, _, keep = ny.spectral_step(mu.astype(np.float64), sigma_r, 1e-7)
    assert int(rank.cpu()) == keep.size
    phi_o, _, _ = ny.features_symmetric(X.astype(np.float64), mu.astype(np.float64), sigma_r, 1e-7)
    rr, _ = report(f"tensor-core features {kind} K={K} N={X.shape[0]}", phi.cpu().numpy().T, phi_o)
    assert rr < 1e-5
    # bfloat16 storage of the same features: each value rounded by at most 2^-8
    pb, _, _ = nyf.features(cuda(X), cuda(mu), sigma_r, 1e-7, precision="bf16")
    rb, _ = report(f"tensor-core features {kind} K={K} bf16", pb.float().cpu().numpy().T, phi_o)
    assert rb < 2.0 ** -8


# ---------------------------------------------------------------- filters

def _params(nyf, w, **kw):
    P = nyf.Params(sigma_s=w.sigma_s, sigma_r=w.sigma_r, K=w.K, kmeans_iters=w.kmeans_iters,
                   seed=w.seed, spatial=w.spatial, S=w.S, patch_radius=w.patch_radius,
                   sample_frac=w.sample_frac)
    for k, v in kw.items():
        setattr(P, k, v)
    return P


def test_blf_colour_256_full_image(nyf):
    w = synth.colour_blf_small()
    mu, _ = oracle_landmarks(w.f.reshape(-1, 3), w.K, 10, w.seed)
    taps = Kr.gaussian_taps(w.sigma_s, w.radius)
    want = ny.nystrom_filter(w.f, w.f, mu.astype(np.float64), w.sigma_r, taps, 1e-7)
    out = nyf.blf(cuda(w.f), _params(nyf, w), landmarks=cuda(mu))
    r, m = report("blf 256x256 K=8 (oracle landmarks)", out.cpu().numpy(), want)
    assert r < FP32_REL_RMSE and m < 0.05


def test_blf_colour_256_with_device_kmeans(nyf):
    w = synth.colour_blf_small()
    mu_o, info = oracle_landmarks(w.f.reshape(-1, 3), w.K, 10, w.seed)
    P = _params(nyf, w)
    ws = nyf.make_workspace(w.H, w.W, 3, 3, P)
    out = nyf.blf(cuda(w.f), P, ws=ws)
    st = nyf.stats(ws)
    assert st["status"] == 0 and st["rank"] == w.K and st["eta_small"] == 0
    print(f"[parity] device kmeans e={st['qerr']:.6e} oracle e={info['e']:.6e}")
    assert abs(st["qerr"] - info["e"]) <= 1e-3 * info["e"]
    taps = Kr.gaussian_taps(w.sigma_s, w.radius)
    want = ny.nystrom_filter(w.f, w.f, mu_o.astype(np.float64), w.sigma_r, taps, 1e-7)
    r, _ = report("blf 256x256 K=8 (device k-means vs oracle pipeline)", out.cpu().numpy(), want)
    assert r < 1e-3


@pytest.mark.parametrize("H,W,sigma_s,K", [(1, 1, 1.0, 1), (1, 57, 2.0, 3), (43, 1, 1.5, 2),
                                           (37, 53, 3.0, 5), (5, 7, 4.0, 4), (97, 131, 5.6, 6),
                                           (70, 66, 8.0, 8), (40, 45, 10.5, 3)])
def test_blf_ragged_and_edge_sizes(nyf, H, W, sigma_s, K):
    f = synth.voronoi_colour(H, W, 12, 8.0, H * 1000 + W)
    X = f.reshape(-1, 3)
    K = min(K, X.shape[0])
    mu = X[rng.distinct_indices(3, K, X.shape[0])].astype(np.float32)
    S = int(math.ceil(3 * sigma_s))
    want = ny.nystrom_filter(f, f, mu.astype(np.float64), 45.0, Kr.gaussian_taps(sigma_s, S), 1e-7)
    P = nyf.Params(sigma_s=sigma_s, sigma_r=45.0, K=K)
    out = nyf.blf(cuda(f), P, landmarks=cuda(mu))
    r, _ = report(f"blf {H}x{W} S={S} K={K}", out.cpu().numpy(), want)
    assert r < FP32_REL_RMSE


def test_blf_joint_guide_and_many_channels(nyf):
    # n = 31 channels: the n + 1 quantities are split over several CTAs
    f = synth.hyperspectral(40, 52, 31, 6, 8.0, 0.02, 21)
    g = synth.voronoi_colour(40, 52, 10, 5.0, 22)[..., :2].copy()
    mu = g.reshape(-1, 2)[rng.distinct_indices(9, 6, 40 * 52)].astype(np.float32)
    taps = Kr.gaussian_taps(2.0, 6)
    want = ny.nystrom_filter(f, g, mu.astype(np.float64), 35.0, taps, 1e-7)
    out = nyf.blf(cuda(f), nyf.Params(sigma_s=2.0, sigma_r=35.0, K=6), guide=cuda(g),
                  landmarks=cuda(mu))
    r, _ = report("joint blf n=31 rho=2", out.cpu().numpy(), want)
    assert r < FP32_REL_RMSE


def test_blf_box_window(nyf):
    f = synth.voronoi_colour(45, 61, 15, 10.0, 23)
    mu = f.reshape(-1, 3)[rng.distinct_indices(4, 7, 45 * 61)].astype(np.float32)
    want = ny.nystrom_filter(f, f, mu.astype(np.float64), 30.0, Kr.box_taps(6), 1e-7)
    out = nyf.blf(cuda(f), nyf.Params(sigma_r=30.0, K=7, spatial="box", S=6), landmarks=cuda(mu))
    r, _ = report("blf box S=6", out.cpu().numpy(), want)
    assert r < FP32_REL_RMSE


# ---------------------------------------------------------------- invariants on the GPU

def test_constant_image_returned(nyf):
    f = np.full((33, 47, 3), 91.0, np.float32)
    mu = np.array([[10, 20, 30], [91, 91, 91], [91, 91, 91], [200, 0, 5]], np.float32)
    out = nyf.blf(cuda(f), nyf.Params(sigma_s=3.0, sigma_r=40.0, K=4), landmarks=cuda(mu))
    assert np.allclose(out.cpu().numpy(), 91.0, rtol=1e-6)


def test_large_sigma_r_is_spatial_blur(nyf):
    f = synth.voronoi_colour(40, 36, 10, 10.0, 24)
    mu = f.reshape(-1, 3)[rng.distinct_indices(1, 5, 40 * 36)].astype(np.float32)
    taps = Kr.gaussian_taps(2.0, 6)
    blur = bf.kernel_filter(f, f, taps, math.inf)
    out = nyf.blf(cuda(f), nyf.Params(sigma_s=2.0, sigma_r=1e6 * 255, K=5), landmarks=cuda(mu))
    r, _ = report("sigma_r -> inf vs blur", out.cpu().numpy(), blur)
    assert r < 1e-5


def test_few_colour_exactness(nyf):
    cols = np.array([[0, 0, 0], [255, 0, 0], [0, 255, 0], [0, 0, 255], [255, 255, 255]], np.float32)
    f = synth.few_colour(40, 44, cols, 25)
    taps = Kr.gaussian_taps(2.5, 8)
    want = bf.kernel_filter(f, f, taps, 60.0)
    out = nyf.blf(cuda(f), nyf.Params(sigma_s=2.5, sigma_r=60.0, K=5, eig_rel_tol=1e-12),
                  landmarks=cuda(cols))
    r, _ = report("few-colour exactness vs brute force", out.cpu().numpy(), want)
    assert r < 1e-5


# ---------------------------------------------------------------- NLM

def test_nlm_subsample_and_parity(nyf):
    f = synth.voronoi_colour(60, 72, 20, 20.0, 26, ramp=0.1)
    P = nyf.Params(sigma_r=20.0 * math.sqrt(75.0), K=6, spatial="box", S=4, patch_radius=2,
                   sample_frac=0.05, seed=77, kmeans_iters=6)
    X, idx, p = pl.nlm_sample_rows(f.astype(np.float64), 2, 0.05, 77)
    mu_o, _ = oracle_landmarks(X, 6, 6, 77)
    want = ny.nystrom_filter(f, p, mu_o.astype(np.float64), P.sigma_r, Kr.box_taps(4), 1e-7)
    out = nyf.nlm(cuda(f), P, landmarks=cuda(mu_o))
    r, _ = report("nlm 60x72 K=6 (oracle landmarks)", out.cpu().numpy(), want)
    assert r < FP32_REL_RMSE
    ws = nyf.make_workspace(60, 72, 3, 75, P)
    out2 = nyf.nlm(cuda(f), P, ws=ws)
    st = nyf.stats(ws)
    assert st["status"] == 0
    r2, _ = report("nlm 60x72 K=6 (device k-means)", out2.cpu().numpy(), want)
    assert r2 < 1e-3


@pytest.mark.parametrize("case", ["few_colour", "duplicate", "random"])
def test_features_gram_matches_oracle(nyf, case):
    # K-hat = Phi Phi^T is unique even when eigenvalues are (nearly) degenerate
    if case == "few_colour":
        mu = np.array([[0, 0, 0], [255, 0, 0], [0, 255, 0], [0, 0, 255], [255, 255, 255]], np.float32)
        sr, tau = 60.0, 1e-12
    elif case == "duplicate":
        mu = np.random.default_rng(5).uniform(0, 255, size=(7, 3)).astype(np.float32)
        mu[4] = mu[1]
        sr, tau = 50.0, 1e-7
    else:
        mu = np.random.default_rng(6).uniform(0, 255, size=(13, 3)).astype(np.float32)
        sr, tau = 45.0, 1e-7
    X = synth.random_image(20, 21, 3, 40).reshape(-1, 3)
    phi, rank, alphas = nyf.features(cuda(X), cuda(mu), sr, tau)
    _, alpha_o, _, keep = ny.spectral_step(mu.astype(np.float64), sr, tau)
    print(f"[parity] eig {case}: gpu={alphas.cpu().numpy()} oracle={alpha_o}")
    assert int(rank.cpu()) == keep.size
    assert np.allclose(alphas.cpu().numpy(), alpha_o, rtol=0, atol=1e-12 * alpha_o[0])
    P = phi.cpu().numpy().T.astype(np.float64)
    from oracle import bound as bd
    Kh = bd.nystrom_matrix(X.astype(np.float64), mu.astype(np.float64), sr, tau)
    r, _ = report(f"K-hat {case}", P @ P.T, Kh)
    assert r < 1e-5
