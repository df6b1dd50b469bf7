"""Parity of the CUDA backward pass with the FP64 oracle gradient (autograd of
Algorithm 1) and with central finite differences of the CUDA forward."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import grad as gr
from oracle import kernels as Kr
from oracle import nystrom as ny
from oracle import rng
from paper_1901_06112_gb300 import synth
from tests._util import report

pytestmark = pytest.mark.gpu
GRAD_TOL = 1e-3


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


def _case(H, W, K, seed, rho=None):
    f = synth.voronoi_colour(H, W, 8, 12.0, seed)
    g = None if rho is None else synth.random_image(H, W, rho, seed + 1)
    src = (f if g is None else g).reshape(-1, 3 if g is None else rho)
    mu = src[rng.distinct_indices(seed, K, src.shape[0])].astype(np.float32)
    G = np.random.default_rng(seed + 2).normal(size=f.shape).astype(np.float32)
    return f, g, mu, G


@pytest.mark.parametrize("mode", ["planes", "recompute"])
@pytest.mark.parametrize("H,W,K,sigma_s,sigma_r", [(40, 36, 5, 2.0, 45.0), (33, 70, 8, 3.3, 60.0),
                                                   (17, 19, 3, 1.4, 80.0), (45, 38, 9, 2.5, 50.0)])
def test_blf_backward_matches_oracle(nyf, H, W, K, sigma_s, sigma_r, mode):
    # mode "recompute": C_kq convolved again in chunks of 4 modes (K = 5, 9: a ragged last chunk)
    f, _, mu, G = _case(H, W, K, 100 + H)
    sr, ss = float(np.float32(sigma_r)), float(np.float32(sigma_s))
    S = int(math.ceil(3 * ss))
    ref = gr.vjp(f, f, mu, sr, ss, S, 1e-7, G, guide_is_image=True)
    res = nyf.blf_vjp(cuda(f), nyf.Params(sigma_s=ss, sigma_r=sr, K=K, backward_mode=mode), cuda(G),
                      landmarks=cuda(mu))
    r, _ = report(f"grad f {H}x{W} K={K} {mode}", res["df"].cpu().numpy(), ref["df"])
    assert r < GRAD_TOL
    for nm in ("dsigma_r", "dsigma_s"):
        rel = abs(res[nm] - ref[nm]) / max(abs(ref[nm]), 1e-12)
        print(f"[parity] {nm}: gpu={res[nm]:.6e} oracle={ref[nm]:.6e} rel={rel:.2e}")
        assert rel < GRAD_TOL


def test_joint_guide_backward_matches_oracle(nyf):
    f, g, mu, G = _case(30, 28, 4, 7, rho=2)
    sr, ss = float(np.float32(70.0)), float(np.float32(1.8))
    ref = gr.vjp(f, g, mu, sr, ss, 6, 1e-7, G)
    res = nyf.blf_vjp(cuda(f), nyf.Params(sigma_s=ss, sigma_r=sr, K=4), cuda(G), guide=cuda(g),
                      landmarks=cuda(mu))
    r1, _ = report("joint grad f", res["df"].cpu().numpy(), ref["df"])
    r2, _ = report("joint grad guide", res["dp"].cpu().numpy(), ref["dp"])
    assert r1 < GRAD_TOL and r2 < GRAD_TOL
    assert abs(res["dsigma_r"] - ref["dsigma_r"]) <= GRAD_TOL * abs(ref["dsigma_r"])
    assert abs(res["dsigma_s"] - ref["dsigma_s"]) <= GRAD_TOL * abs(ref["dsigma_s"])


@pytest.mark.parametrize("rho,K", [(31, 16), (40, 8), (160, 64)])
def test_deep_guide_backward_matches_oracle(nyf, rho, K):
    # dL/dp for guides of dimension 31 (row in registers), 40 (row staged in shared
    # memory) and 160 with K = 64 (row in global memory): the three paths of the
    # features backward
    f = synth.voronoi_colour(22, 27, 6, 8.0, 50 + rho)
    g = synth.hyperspectral(22, 27, rho, 4, 6.0, 0.02, 60 + rho)
    mu = g.reshape(-1, rho)[rng.distinct_indices(3, K, 22 * 27)].astype(np.float32)
    G = np.random.default_rng(rho).normal(size=f.shape).astype(np.float32)
    sr = float(np.float32(0.35 if rho < 100 else 0.8))
    ref = gr.vjp(f, g, mu, sr, 1.5, 5, 1e-7, G)
    res = nyf.blf_vjp(cuda(f), nyf.Params(sigma_s=1.5, sigma_r=sr, K=K), cuda(G), guide=cuda(g),
                      landmarks=cuda(mu))
    r1, _ = report(f"rho={rho} K={K} grad f", res["df"].cpu().numpy(), ref["df"])
    r2, _ = report(f"rho={rho} K={K} grad guide", res["dp"].cpu().numpy(), ref["dp"])
    assert r1 < GRAD_TOL and r2 < GRAD_TOL
    assert abs(res["dsigma_r"] - ref["dsigma_r"]) <= GRAD_TOL * abs(ref["dsigma_r"])


@pytest.mark.parametrize("mode", ["planes", "recompute"])
def test_many_channels_backward(nyf, mode):
    # n = 7: quantities split over CTAs (dL/dphi accumulated across them)
    f = synth.hyperspectral(24, 26, 7, 3, 6.0, 0.02, 9) * 255.0
    g = synth.voronoi_colour(24, 26, 6, 5.0, 10)
    mu = g.reshape(-1, 3)[rng.distinct_indices(2, 5, 24 * 26)].astype(np.float32)
    G = np.random.default_rng(3).normal(size=f.shape).astype(np.float32)
    ref = gr.vjp(f, g, mu, 50.0, 1.5, 5, 1e-7, G)
    res = nyf.blf_vjp(cuda(f), nyf.Params(sigma_s=1.5, sigma_r=50.0, K=5, backward_mode=mode),
                      cuda(G), guide=cuda(g), landmarks=cuda(mu))
    r1, _ = report(f"n=7 grad f {mode}", res["df"].cpu().numpy(), ref["df"])
    r2, _ = report(f"n=7 grad guide {mode}", res["dp"].cpu().numpy(), ref["dp"])
    assert r1 < GRAD_TOL and r2 < GRAD_TOL
    for nm in ("dsigma_r", "dsigma_s"):
        assert abs(res[nm] - ref[nm]) <= GRAD_TOL * abs(ref[nm])


def test_recompute_mode_workspace_and_agreement(nyf):
    # the recompute workspace holds 4 modes' planes instead of K; the gradients agree
    # with the saved-planes backward to FP32 rounding (the same arithmetic, summed in
    # chunks of modes)
    f, _, mu, G = _case(96, 130, 11, 61)
    P = nyf.Params(sigma_s=3.0, sigma_r=40.0, K=11)
    Pp, Pr = P.for_backward(), nyf.Params(**{**P.__dict__, "backward_mode": "recompute"}).for_backward()
    wp = nyf.workspace_size(96, 130, 3, 3, Pp)
    wr = nyf.workspace_size(96, 130, 3, 3, Pr)
    assert wp - wr >= (11 - 4) * 4 * 96 * 130 * 4
    a = nyf.blf_vjp(cuda(f), Pp, cuda(G), landmarks=cuda(mu))
    b = nyf.blf_vjp(cuda(f), Pr, cuda(G), landmarks=cuda(mu))
    assert torch.equal(a["out"], b["out"])
    r, _ = report("recompute vs planes grad f", b["df"].cpu().numpy(), a["df"].cpu().numpy())
    assert r < 1e-5
    for nm in ("dsigma_r", "dsigma_s"):
        assert abs(a[nm] - b[nm]) <= 1e-5 * abs(a[nm])


def test_sigma_gradients_match_finite_differences(nyf):
    f, _, mu, G = _case(48, 40, 6, 21)
    Gt, ft, mut = cuda(G), cuda(f), cuda(mu)

    def loss(sr, ss):
        out = nyf.blf(ft, nyf.Params(sigma_s=ss, sigma_r=sr, K=6, S=7), landmarks=mut)
        return float((out.double() * Gt.double()).sum())

    sr, ss = 50.0, 2.2
    res = nyf.blf_vjp(ft, nyf.Params(sigma_s=ss, sigma_r=sr, K=6, S=7), Gt, landmarks=mut)
    hr, hs = 0.25, 0.01
    fd_r = (loss(sr + hr, ss) - loss(sr - hr, ss)) / (2 * hr)
    fd_s = (loss(sr, ss + hs) - loss(sr, ss - hs)) / (2 * hs)
    print(f"[parity] FD sigma_r gpu={res['dsigma_r']:.6e} fd={fd_r:.6e}")
    print(f"[parity] FD sigma_s gpu={res['dsigma_s']:.6e} fd={fd_s:.6e}")
    assert abs(res["dsigma_r"] - fd_r) <= GRAD_TOL * abs(fd_r) + 1e-4
    assert abs(res["dsigma_s"] - fd_s) <= GRAD_TOL * abs(fd_s) + 1e-4


def test_autograd_function(nyf):
    f, _, mu, G = _case(32, 30, 4, 31)
    ft = cuda(f).requires_grad_(True)
    sr = torch.tensor(55.0, device="cuda", requires_grad=True)
    ss = torch.tensor(2.0, device="cuda", requires_grad=True)
    out = nyf.blf_autograd(ft, sr, ss, nyf.Params(K=4), landmarks=cuda(mu))
    (out * cuda(G)).sum().backward()
    ref = gr.vjp(f, f, mu, 55.0, 2.0, 6, 1e-7, G, guide_is_image=True)
    r, _ = report("autograd grad f", ft.grad.cpu().numpy(), ref["df"])
    assert r < GRAD_TOL
    assert abs(float(sr.grad) - ref["dsigma_r"]) <= GRAD_TOL * abs(ref["dsigma_r"])
    assert abs(float(ss.grad) - ref["dsigma_s"]) <= GRAD_TOL * abs(ref["dsigma_s"])
