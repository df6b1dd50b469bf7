"""Parity of the PCA-NLM path (Sec. IV: PCA of the patches, the projected
guide, Algorithm 1 on it) with the FP64 oracle (oracle.pca), through the C ABI.

The leading eigenvectors are unique only up to sign and up to rotations inside
groups of (nearly) equal eigenvalues, so the tests compare what is unique (the
eigenvalues, the mean, eigenvectors whose eigenvalue is well separated, the
projection for a given basis, the filter for a given basis and landmarks) and
check that the rest is valid (orthonormal columns that satisfy C u = lambda u)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import guide as gd
from oracle import kernels as Kr
from oracle import nystrom as ny
from oracle import pca
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


def _crop(H=96, W=120):
    w = synth.colour_pca_nlm()
    return w, w.f[:H, :W].copy()


@pytest.mark.parametrize("r,n", [(1, 3), (2, 3), (3, 3), (2, 1), (1, 7)])
def test_moments_and_eigenpairs(nyf, r, n):
    w, f3 = _crop()
    f = f3 if n == 3 else np.concatenate([f3] * 3, axis=2)[..., :n]
    rho = n * (2 * r + 1) ** 2
    q = min(rho, 25)
    m_o, C_o = pca.patch_moments(f.astype(np.float64), r)
    lam_o, U_o = pca.pca_basis(C_o, q)
    m, U, lam, ws = nyf.patch_pca(cuda(f), r, q)
    st = nyf.stats(ws)
    assert st["status"] == 0
    m, U, lam = (t.cpu().numpy().astype(np.float64) for t in (m, U, lam))
    assert np.allclose(m, m_o, rtol=2e-6, atol=1e-4)
    assert np.abs(lam - lam_o).max() <= 2e-5 * lam_o[0]
    # valid basis: orthonormal columns with C u = lambda u
    assert np.allclose(U.T @ U, np.eye(q), atol=2e-5)
    res = np.linalg.norm(C_o @ U - U * lam[:q], axis=0)
    assert res.max() <= 2e-4 * lam_o[0]
    # unique where the eigenvalue is well separated: equal to the oracle's up to sign
    ext = np.r_[np.inf, lam_o[:q], lam_o[q] if q < rho else -np.inf]
    gap = np.minimum(ext[:-2] - ext[1:-1], ext[1:-1] - ext[2:])       # to both neighbours
    sep = gap > 1e-2 * lam_o[0]
    cos = np.abs(np.sum(U * U_o, axis=0))
    print(f"[pca] r={r} n={n} rho={rho}: {sep.sum()} separated of {q}, min |cos| {cos[sep].min():.8f}")
    assert np.all(cos[sep] >= 1 - 1e-4)


def test_projection_with_a_given_basis(nyf):
    w, f = _crop()
    m_o, C_o = pca.patch_moments(f.astype(np.float64), 3)
    _, U_o = pca.pca_basis(C_o, 25)
    mf, Uf = m_o.astype(np.float32), U_o.astype(np.float32)
    g = nyf.pca_project(cuda(f), 3, cuda(mf), cuda(Uf)).cpu().numpy()
    want = pca.project(gd.patch_guide(f.astype(np.float64), 3), mf.astype(np.float64),
                       Uf.astype(np.float64))
    r, _ = report("pca projection 96x120 r=3 q=25", g, want)
    assert r < 1e-6


@pytest.mark.parametrize("H,W,r,q,K", [(96, 120, 3, 25, 31), (41, 57, 2, 6, 9), (33, 29, 1, 8, 5)])
def test_pca_nlm_with_oracle_basis_and_landmarks(nyf, H, W, r, q, K):
    w, f = _crop(H, W)
    g_pca, m, U = pca.pca_guide(f.astype(np.float64), r, q)
    mf, Uf = m.astype(np.float32), U.astype(np.float32)
    g_pca, _, _ = pca.pca_guide(f.astype(np.float64), r, q, mf.astype(np.float64), Uf.astype(np.float64))
    mu, _ = pl.landmarks(g_pca.reshape(-1, q), K, 5, 3)
    mu = mu.astype(np.float32)
    want = ny.nystrom_filter(f, g_pca, mu.astype(np.float64), w.sigma_r, Kr.box_taps(w.S), 1e-7)
    P = nyf.Params(sigma_r=w.sigma_r, K=K, spatial="box", S=w.S, patch_radius=r)
    out = nyf.pca_nlm(cuda(f), q, P, mean=cuda(mf), basis=cuda(Uf), landmarks=cuda(mu))
    rr, _ = report(f"pca-nlm {H}x{W} r={r} q={q} K={K} (oracle basis, landmarks)",
                   out.cpu().numpy(), want)
    assert rr < FP32_REL_RMSE


def test_full_dimension_pca_nlm_equals_nlm_on_gpu(nyf):
    # q = rho = 27: the projection is an isometry, so with the landmarks mapped by it
    # the GPU's PCA-NLM (its own basis) equals the GPU's NLM
    w, f = _crop(64, 80)
    r, rho = 1, 27
    X = gd.patch_guide(f.astype(np.float64), r).reshape(-1, rho)
    mu, _ = pl.landmarks(X, 7, 5, 2)
    mu = mu.astype(np.float32)
    sr = 40.0 * np.sqrt(rho)                # eta-hat well away from zero on this crop
    P = nyf.Params(sigma_r=sr, K=7, spatial="box", S=4, patch_radius=r)
    ft = cuda(f)
    g_nlm = nyf.nlm(ft, P, landmarks=cuda(mu)).cpu().numpy()
    m, U, _, _ = nyf.patch_pca(ft, r, rho)
    mu_p = ((mu.astype(np.float64) - m.cpu().numpy()) @ U.cpu().numpy()).astype(np.float32)
    g_pca = nyf.pca_nlm(ft, rho, P, landmarks=cuda(mu_p)).cpu().numpy()
    rr, _ = report("pca-nlm q=rho vs nlm (GPU)", g_pca, g_nlm)
    assert rr < FP32_REL_RMSE


def test_full_workload_768x512(nyf):
    # the PCA-NLM workload at full size (7x7x3 patches, q 25, K 31, S 10): the GPU's
    # moments and eigenvalues against the oracle's, and the filter on the oracle's
    # basis and landmarks against the oracle on every pixel
    w = synth.colour_pca_nlm()
    f = w.f
    m_o, C_o = pca.patch_moments(f.astype(np.float64), w.patch_radius)
    lam_o, U_o = pca.pca_basis(C_o, w.pca_dim)
    ft = cuda(f)
    m, U, lam, ws = nyf.patch_pca(ft, w.patch_radius, w.pca_dim)
    assert nyf.stats(ws)["status"] == 0
    assert np.allclose(m.cpu().numpy(), m_o, rtol=2e-6, atol=1e-4)
    assert np.abs(lam.cpu().numpy() - lam_o).max() <= 2e-5 * lam_o[0]
    mf, Uf = m_o.astype(np.float32), U_o.astype(np.float32)
    g_pca, _, _ = pca.pca_guide(f.astype(np.float64), w.patch_radius, w.pca_dim,
                                mf.astype(np.float64), Uf.astype(np.float64))
    from oracle import rng
    H, W = f.shape[:2]
    idx = rng.stratified_sample(w.seed, rng.subsample_size(H * W, w.sample_frac), H * W)
    mu, _ = pl.landmarks(g_pca.reshape(H * W, -1)[idx], w.K, w.kmeans_iters, w.seed)
    mu = mu.astype(np.float32)
    want = ny.nystrom_filter(f, g_pca, mu.astype(np.float64), w.sigma_r, Kr.box_taps(w.S), 1e-7)
    P = nyf.Params(sigma_r=w.sigma_r, K=w.K, spatial="box", S=w.S, patch_radius=w.patch_radius,
                   sample_frac=w.sample_frac, seed=w.seed)
    ws2 = nyf.make_pca_workspace(H, W, 3, w.pca_dim, P)
    out = nyf.pca_nlm(ft, w.pca_dim, P, mean=cuda(mf), basis=cuda(Uf), landmarks=cuda(mu), ws=ws2)
    st = nyf.stats(ws2)
    assert st["status"] == 0 and st["rank"] >= 1
    rr, _ = report("pca-nlm 768x512 q=25 K=31 (oracle basis, landmarks)", out.cpu().numpy(), want)
    assert rr < FP32_REL_RMSE
    # the whole path on its own (basis and k-means on the GPU): valid and close
    out2 = nyf.pca_nlm(ft, w.pca_dim, P, ws=ws2)
    st2 = nyf.stats(ws2)
    assert st2["status"] == 0
    d = float(np.sqrt(np.mean((out2.cpu().numpy() - want) ** 2) / np.mean(want ** 2)))
    print(f"[pca] own basis + device k-means vs oracle pipeline: rel RMSE {d:.3e}")
    assert d < 0.05
