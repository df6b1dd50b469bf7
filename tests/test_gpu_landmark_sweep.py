"""Landmark selection and the number of landmarks against the exact filter.

The Nystrom filter (Algorithm 1) with K landmarks from k-means (Sec. III) or
from a uniform draw of pixels (the seeded initial draw with no Lloyd
iteration), on the 256 x 256 colour workload, against the brute-force kernel
filter of Eq. (1).  Sec. III argues that the approximation error falls with the
k-means quantisation error e, which k-means minimises and which falls as K
grows (Proposition 1); the experiments report k-means ahead of uniform sampling
and the PSNR rising with m0.  This checks both effects on the synthetic image
(averaged over three seeds) and prints the table."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import bruteforce as bf
from oracle import kernels as Kr
from paper_1901_06112_gb300 import synth

pytestmark = pytest.mark.gpu

KS = [2, 4, 8, 16, 32]
SEEDS = [1, 2, 3]


@pytest.fixture(scope="module")
def nyf():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1901_06112_gb300 import build
    build.build()
    from paper_1901_06112_gb300 import nyf as N
    return N


def psnr(x, ref, peak=255.0):
    return 10.0 * np.log10(peak * peak / np.mean((x - ref) ** 2))


def test_kmeans_beats_uniform_and_psnr_rises_with_k(nyf):
    w = synth.colour_blf_small()
    sr = float(np.float32(w.sigma_r))
    exact = bf.kernel_filter(w.f, w.f, Kr.gaussian_taps(w.sigma_s, w.radius), sr)
    ft = torch.from_numpy(w.f).cuda()
    table = {}
    for mode, iters in (("k-means", 10), ("uniform", 0)):
        for K in KS:
            vals = []
            for seed in SEEDS:
                P = nyf.Params(sigma_s=w.sigma_s, sigma_r=sr, K=K, kmeans_iters=iters, seed=seed)
                vals.append(psnr(nyf.blf(ft, P).cpu().numpy().astype(np.float64), exact))
            table[(mode, K)] = float(np.mean(vals))
    print("\n[sweep] 256x256 colour BLF, sigma_s 3, sigma_r 30: PSNR (dB) vs the exact filter, "
          "mean of 3 seeds")
    print("[sweep]   K    k-means   uniform")
    for K in KS:
        print(f"[sweep] {K:3d}   {table[('k-means', K)]:7.2f}   {table[('uniform', K)]:7.2f}")
    km = [table[("k-means", K)] for K in KS]
    un = [table[("uniform", K)] for K in KS]
    # PSNR rises with K for k-means landmarks (each doubling helps)
    assert all(b > a for a, b in zip(km, km[1:]))
    # k-means landmarks beat uniform ones for every K >= 4
    assert all(table[("k-means", K)] > table[("uniform", K)] for K in KS if K >= 4)
