"""Lloyd k-means for landmark selection (Sec. III; Algorithm 1, clustering step).

The landmarks mu_1..mu_m0 are the centroids of a k-means partition of the
range list R (Sec. III, following Zhang et al. 2008).  The paper fixes neither
initialisation nor iteration count; the reading used here (and by the CUDA
path):

* start from given centroids (normally rows of R drawn by
  ``rng.distinct_indices``);
* each iteration assigns every r_i to c(i) = argmin_j ||r_i - mu_j||^2, ties to
  the lowest j, then replaces each centroid by the mean of its members; a
  centroid with no members keeps its position;
* exactly `iters` iterations, no convergence test;
* the quantisation error e = sum_i ||r_i - mu_c(i)||^2 (Sec. III, before
  Proposition 1) is evaluated for the final centroids.

Distances are direct differences in float64.

Pinned by: tests/test_oracle_kmeans.py -- objective non-increasing; exact
recovery of well-separated colours; ties and empty clusters; agreement with
scikit-learn's Lloyd iterations on well-separated data.
"""
from __future__ import annotations

import numpy as np


def sq_dists(X: np.ndarray, mu: np.ndarray) -> np.ndarray:
    """||x_i - mu_j||^2 for all i, j (m x m0), by direct differences."""
    X = np.asarray(X, np.float64)
    mu = np.asarray(mu, np.float64)
    D = np.empty((X.shape[0], mu.shape[0]))
    for j in range(mu.shape[0]):
        d = X - mu[j]
        D[:, j] = np.sum(d * d, axis=1)
    return D


def assign(X: np.ndarray, mu: np.ndarray):
    """Nearest centroid (lowest index on ties) and the quantisation error e."""
    D = sq_dists(X, mu)
    c = np.argmin(D, axis=1)            # argmin returns the first minimum
    e = float(np.sum(D[np.arange(D.shape[0]), c]))
    return c, e


def update(X: np.ndarray, c: np.ndarray, mu: np.ndarray) -> np.ndarray:
    """Centroid = mean of its members; an empty cluster keeps its centroid."""
    X = np.asarray(X, np.float64)
    new = np.array(mu, dtype=np.float64, copy=True)
    for j in range(new.shape[0]):
        members = X[c == j]
        if members.shape[0] > 0:
            new[j] = members.mean(axis=0)
    return new


def kmeans(X: np.ndarray, init: np.ndarray, iters: int):
    """Lloyd iterations from `init`.

    Returns (mu, labels, e, e_history): the centroids after `iters` updates,
    the labels and quantisation error for those centroids, and the error seen at
    every assignment step (iters + 1 values, the last being `e`).
    """
    mu = np.array(init, dtype=np.float64, copy=True)
    hist = []
    for _ in range(iters):
        c, e = assign(X, mu)
        hist.append(e)
        mu = update(X, c, mu)
    c, e = assign(X, mu)
    hist.append(e)
    return mu, c, e, hist
