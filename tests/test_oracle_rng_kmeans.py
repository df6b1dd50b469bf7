"""Pins for oracle.rng (SplitMix64 draws) and oracle.kmeans (Lloyd landmarks, Sec. III)."""
import os

import numpy as np
import pytest

from oracle import kmeans as km
from oracle import rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed0.txt")


def test_splitmix64_published_sequence():
    vals = [int(l, 16) for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert [rng.splitmix64(0, t) for t in range(1, len(vals) + 1)] == vals


def test_distinct_indices_skip_repeats_in_draw_order():
    N, seed = 5, 12345
    cands = [rng.splitmix64(seed, t) % N for t in range(1, 200)]
    want = []
    for c in cands:
        if c not in want:
            want.append(c)
        if len(want) == 4:
            break
    assert list(rng.distinct_indices(seed, 4, N)) == want
    got = rng.distinct_indices(99, 64, 1000)
    assert len(set(got.tolist())) == 64 and got.min() >= 0 and got.max() < 1000
    with pytest.raises(ValueError):
        rng.distinct_indices(1, 6, 5)


def test_stratified_sample_one_per_stratum():
    N, c = 393216, 3932
    idx = rng.stratified_sample(7, c, N)
    assert idx.shape == (c,)
    t = np.arange(c)
    assert np.all(idx >= (t * N) // c) and np.all(idx < ((t + 1) * N) // c)
    assert rng.subsample_size(N, 0.01) == 3932
    assert rng.subsample_size(10, 0.01) == 1


def test_kmeans_objective_non_increasing():
    r = np.random.default_rng(8)
    X = r.uniform(0, 255, size=(3000, 3))
    init = X[rng.distinct_indices(3, 16, 3000)]
    _, _, e, hist = km.kmeans(X, init, 12)
    assert all(b <= a * (1 + 1e-12) for a, b in zip(hist, hist[1:]))
    assert e == hist[-1]


def test_kmeans_recovers_separated_colours():
    cols = np.array([[10, 10, 10], [200, 30, 30], [30, 200, 30], [30, 30, 200], [220, 220, 220]], float)
    r = np.random.default_rng(9)
    lab = r.integers(0, 5, size=2000)
    lab[:5] = np.arange(5)
    X = cols[lab]
    init = X[[0, 1, 2, 3, 4]] + r.normal(0, 3, size=(5, 3))
    mu, c, e, _ = km.kmeans(X, init, 3)
    assert np.allclose(mu, cols, atol=1e-12)
    assert np.array_equal(c, lab) and e < 1e-18


def test_kmeans_tie_goes_to_lowest_index_and_empty_keeps():
    X = np.array([[0.0, 0.0], [2.0, 0.0]])
    mu0 = np.array([[1.0, 1.0], [1.0, -1.0], [50.0, 50.0]])   # both points tie between 0 and 1
    c, _ = km.assign(X, mu0)
    assert list(c) == [0, 0]
    mu1 = km.update(X, c, mu0)
    assert np.allclose(mu1[0], [1.0, 0.0])
    assert np.array_equal(mu1[1], mu0[1]) and np.array_equal(mu1[2], mu0[2])


def test_kmeans_agrees_with_scikit_learn_lloyd():
    sk = pytest.importorskip("sklearn.cluster")
    r = np.random.default_rng(10)
    centres = r.uniform(0, 255, size=(6, 3))
    X = centres[r.integers(0, 6, size=1500)] + r.normal(0, 6, size=(1500, 3))
    init = X[rng.distinct_indices(5, 6, 1500)]
    ours, _, _, _ = km.kmeans(X, init, 50)
    ref = sk.KMeans(n_clusters=6, init=init, n_init=1, max_iter=50, tol=0.0,
                    algorithm="lloyd").fit(X).cluster_centers_
    assert np.allclose(ours, ref, rtol=1e-10, atol=1e-9)
