"""The FP32 C++/OpenMP CPU baseline (timed by bench.py beside the GPU) computes
the same filter as the FP64 oracle: with the oracle's landmarks to FP32
accuracy, and its own k-means (same seeded initial rows) reaches the oracle's
k-means objective.  It is a baseline, not the oracle, so it is held to the
oracle like the GPU path is."""
import numpy as np
import pytest

from oracle import cpu_build
from oracle import kernels as Kr
from oracle import nystrom as ny
from oracle import pipeline as pl
from paper_1901_06112_gb300 import synth
from tests._util import FP32_REL_RMSE, report


@pytest.fixture(scope="module")
def lib():
    try:
        return cpu_build.load()
    except (RuntimeError, OSError) as ex:
        pytest.skip(f"no C++ toolchain: {ex}")


@pytest.mark.parametrize("threads", [1, 4])
def test_cpu_baseline_matches_oracle(lib, threads):
    f = synth.voronoi_colour(41, 57, 12, 10.0, 3)
    mu, _ = pl.landmarks(f.reshape(-1, 3).astype(np.float64), 6, 5, 2)
    mu = mu.astype(np.float32)
    want = ny.nystrom_filter(f, f, mu.astype(np.float64), 30.0, Kr.gaussian_taps(2.0, 6), 1e-7)
    got, code = cpu_build.blf(lib, f, 2.0, 30.0, 6, landmarks=mu, threads=threads)
    assert code == 0
    r, _ = report(f"cpu baseline {threads} threads", got, want)
    assert r < FP32_REL_RMSE


def test_cpu_baseline_kmeans_reaches_the_oracle_objective(lib):
    f = synth.voronoi_colour(48, 40, 20, 10.0, 5)
    X = f.reshape(-1, 3).astype(np.float64)
    mu, info = pl.landmarks(X, 8, 10, 4)
    got, code = cpu_build.blf(lib, f, 2.0, 30.0, 8, iters=10, seed=4)
    want = ny.nystrom_filter(f, f, mu.astype(np.float32).astype(np.float64), 30.0,
                             Kr.gaussian_taps(2.0, 6), 1e-7)
    assert code == 0
    r, _ = report("cpu baseline with its own k-means", got, want)
    assert r < 1e-3            # near-ties may move a few points between clusters
