"""Strip processing (one image cut into horizontal strips with an S-row halo,
k-means over all strips by exchanging per-cluster sums): the owned rows equal
the whole-image filter with the same landmarks bitwise (FP32), the strips'
k-means reaches the whole-image k-means, and the filter matches the FP64 oracle
with the oracle's landmarks."""
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
def mods():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1901_06112_gb300 import build
    build.build()
    from paper_1901_06112_gb300 import nyf, strips
    return nyf, strips


@pytest.mark.parametrize("parts", [2, 3, 7])
def test_strips_equal_whole_image(mods, parts):
    nyf, strips = mods
    f = synth.voronoi_colour(301, 257, 30, 10.0, 40 + parts)
    P = nyf.Params(sigma_s=3.0, sigma_r=30.0, K=8, kmeans_iters=6, seed=5)
    ft = torch.from_numpy(f).cuda()
    out, cent, qerr = strips.blf_strips(ft, P, parts)
    whole = nyf.blf(ft, P, landmarks=cent)
    torch.cuda.synchronize()
    assert torch.equal(out, whole)                     # owned rows: same window sums
    c1, _, q1 = nyf.kmeans(ft.reshape(-1, 3), 8, iters=6, seed=5)
    r, _ = report(f"strip k-means ({parts} strips) vs whole-image k-means", cent.cpu().numpy(),
                  c1.cpu().numpy())
    assert r < 1e-5
    assert abs(float(qerr.cpu()) - float(q1.cpu())) <= 1e-6 * float(q1.cpu())


def test_strips_match_oracle(mods):
    nyf, strips = mods
    f = synth.voronoi_colour(120, 97, 20, 10.0, 9)
    mu, _ = pl.landmarks(f.reshape(-1, 3).astype(np.float64), 6, 5, 2)
    mu = mu.astype(np.float32)
    P = nyf.Params(sigma_s=2.0, sigma_r=35.0, K=6)
    want = ny.nystrom_filter(f, f, mu.astype(np.float64), 35.0, Kr.gaussian_taps(2.0, 6), 1e-7)

    class Fixed(strips.StripOps):                        # the oracle's landmarks for the filter
        def filter(self, f_halo, params, landmarks):
            return nyf.blf(f_halo, params, landmarks=torch.from_numpy(mu).cuda())
    out, _, _ = strips.blf_strips(torch.from_numpy(f).cuda(), P, 4, ops=Fixed())
    r, _ = report("strips (4) vs the FP64 oracle", out.cpu().numpy(), want)
    assert r < FP32_REL_RMSE
