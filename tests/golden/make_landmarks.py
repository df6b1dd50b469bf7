"""Writes the FP64 oracle's k-means landmarks of the benchmark workloads.

Each file holds the landmarks that the oracle's pipeline (``oracle.pipeline``:
seeded initial rows, ``kmeans_iters`` Lloyd iterations in FP64, Sec. III and
Algorithm 1's clustering step) finds for one seeded synthetic workload, rounded
to float32 (how landmarks are handed to the CUDA path).  ``bench.py`` feeds them
to the library for the accuracy pass it reports beside each throughput, and
compares the result with the oracle's Algorithm 1 on sampled pixels.  Nothing
here calls the CUDA path.

Usage: python tests/golden/make_landmarks.py [workload ...]
  workloads: colour_256, colour_hd, hyperspectral, nlm, batched
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import pipeline as pl          # noqa: E402
from paper_1901_06112_gb300 import synth   # noqa: E402


def _landmarks(w):
    """Oracle landmarks of workload w (K x rho, float32)."""
    if w.patch_radius > 0:
        X, _, _ = pl.nlm_sample_rows(w.f.astype(np.float64), w.patch_radius, w.sample_frac, w.seed)
    else:
        X = w.f.reshape(-1, w.n).astype(np.float64)
    mu, info = pl.landmarks(X, w.K, w.kmeans_iters, w.seed)
    return mu.astype(np.float32), info["e"]


def _write(name, header, blocks):
    path = os.path.join(HERE, f"landmarks_{name}.txt")
    with open(path, "w") as fh:
        for line in header:
            fh.write(f"# {line}\n")
        for b, (mu, e) in enumerate(blocks):
            fh.write(f"# block {b} K {mu.shape[0]} rho {mu.shape[1]} e {e:.17g}\n")
            for row in mu:
                fh.write(" ".join(f"{v:.9g}" for v in row) + "\n")
    print(path)


def load(name):
    """(list of K x rho float32 landmark blocks, list of the oracle's k-means errors e)."""
    blocks, errs, cur = [], [], None
    with open(os.path.join(HERE, f"landmarks_{name}.txt")) as fh:
        for line in fh:
            if line.startswith("# block"):
                if cur is not None:
                    blocks.append(np.array(cur, np.float32))
                cur = []
                errs.append(float(line.split()[-1]))
            elif not line.startswith("#") and line.strip():
                cur.append([float(v) for v in line.split()])
    if cur is not None:
        blocks.append(np.array(cur, np.float32))
    return blocks, errs


HEADER = ["Oracle k-means landmarks (oracle.pipeline.landmarks: seeded initial rows,",
          "Lloyd iterations in FP64; Sec. III / Algorithm 1 clustering) of the seeded",
          "synthetic workload named in the file name, rounded to float32.",
          "Written by tests/golden/make_landmarks.py, which calls only oracle/ and the",
          "input generators."]

WORKLOADS = {
    "colour_256": lambda: [synth.colour_blf_small()],
    "colour_hd": lambda: [synth.colour_blf_hd()],
    "hyperspectral": lambda: [synth.hyperspectral_blf()],
    "nlm": lambda: [synth.colour_nlm()],
    "batched": lambda: synth.batched_blf(),
}


def main(names):
    for name in names or list(WORKLOADS):
        ws = WORKLOADS[name]()
        blocks = []
        for w in ws:
            if name == "batched":       # the batch's shared k-means settings (K 16, seed 0)
                w = synth.Workload(w.name, w.f, w.R, w.sigma_s, w.sigma_r, 16, seed=0)
            blocks.append(_landmarks(w))
        _write(name, HEADER + [f"workload: {ws[0].name if len(ws) == 1 else name}"
                               f"{'' if len(ws) == 1 else f' ({len(ws)} images, seed 0, K 16)'}"],
               blocks)


if __name__ == "__main__":
    main(sys.argv[1:])
