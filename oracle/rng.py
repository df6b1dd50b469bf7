"""SplitMix64 and the seeded index draws that both sides implement.

The paper does not say how k-means is initialised (Sec. III, Algorithm 1 only
says "k-means").  Both the oracle and the CUDA path draw the initial landmark
indices, and the nonlocal-means k-means subsample, from SplitMix64 (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), a
counter-based generator: output t (t = 1, 2, ...) of a stream seeded with s is
mix(s + t * 0x9E3779B97F4A7C15) with the published finaliser below.  Each side
implements it from that definition.

* ``distinct_indices`` -- candidate t is output_t mod N; a repeat of an earlier
  candidate is skipped; the first `count` distinct candidates are returned in
  draw order.
* ``stratified_sample`` -- stratum t covers [floor(tN/c), floor((t+1)N/c)) and
  contributes the index lo + output_{t+1} mod (hi - lo) of the sample stream
  (seed XOR 0xA5A5A5A5A5A5A5A5).  Distinct and sorted by construction.

Pinned by: tests/test_oracle_rng.py against the published SplitMix64 output
sequence for seed 0 (tests/golden/splitmix64_seed0.txt).
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MASK = (1 << 64) - 1
SAMPLE_STREAM = 0xA5A5A5A5A5A5A5A5


def mix64(z: int) -> int:
    """SplitMix64 output finaliser (variant 13 of Stafford's mixers)."""
    z &= MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def splitmix64(seed: int, t: int) -> int:
    """Output t (1-based) of the stream seeded with `seed`."""
    return mix64((seed + t * GAMMA) & MASK)


def distinct_indices(seed: int, count: int, N: int, max_draws: int | None = None) -> np.ndarray:
    """First `count` distinct values of output_t mod N, t = 1, 2, ... (draw order)."""
    if count > N:
        raise ValueError("cannot draw more distinct indices than there are items")
    if max_draws is None:
        max_draws = 64 * count + 4096
    seen = set()
    out = []
    t = 0
    while len(out) < count:
        t += 1
        if t > max_draws:
            raise RuntimeError("index draw did not finish within the draw limit")
        i = splitmix64(seed, t) % N
        if i not in seen:
            seen.add(i)
            out.append(i)
    return np.asarray(out, dtype=np.int64)


def stratified_sample(seed: int, count: int, N: int) -> np.ndarray:
    """One index per stratum [floor(tN/count), floor((t+1)N/count)), t < count."""
    if count > N or count <= 0:
        raise ValueError("sample size must lie in [1, N]")
    s = (seed ^ SAMPLE_STREAM) & MASK
    out = np.empty(count, dtype=np.int64)
    for t in range(count):
        lo = (t * N) // count
        hi = ((t + 1) * N) // count
        out[t] = lo + splitmix64(s, t + 1) % (hi - lo)
    return out


def subsample_size(N: int, frac: float) -> int:
    """round(frac * N) clamped to [1, N]: the number of pixels k-means sees."""
    return int(min(N, max(1, int(np.floor(frac * N + 0.5)))))
