"""Strip processing of one image: horizontal strips, each filtered with an
S-row halo, and k-means over all strips by exchanging per-cluster sums.

The paper's method (Algorithm 1) is separable into per-pixel steps (features),
window sums of radius S (the convolutions) and one global step, the k-means
clustering of Sec. III.  So an image can be cut into horizontal strips that
are processed independently -- one per GPU, or one after another on one GPU
when the image is too large for one workspace -- provided that

* each strip carries S rows of halo above and below (clipped to the image), so
  that the window sums of its own rows see the same pixels as in the whole
  image (the zero padding of Eq. (1) only at the image's true borders);
* k-means runs on the union of the strips' own rows: the initial rows are one
  draw over the whole image (each strip contributes the drawn rows it owns),
  and every Lloyd iteration adds the strips' per-cluster sums and counts (one
  all-reduce of K x (rho + 1) numbers) before the centroids move;
* every strip then filters with the same landmarks.

The owned rows of the strips' outputs equal the whole-image filter with those
landmarks, bitwise on the FP32 path (the window sums of a row do not depend on
where its tile starts).

`StripOps` holds the per-strip operations and `reduce` the collective: a sum
over a list (one process holding every strip, `local_reduce`) or
`torch.distributed.all_reduce` (one strip per rank, `dist_reduce`).  The GPU
operations are those of libnyf's C ABI.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib as L
from . import nyf


def strip_rows(H: int, parts: int, i: int):
    """Rows [y0, y1) that strip i of `parts` owns."""
    return (i * H) // parts, ((i + 1) * H) // parts


def halo_rows(H: int, y0: int, y1: int, S: int):
    """Rows [h0, h1) a strip owning [y0, y1) reads: its rows grown by S, clipped to the image."""
    return max(0, y0 - S), min(H, y1 + S)


def local_reduce(parts):
    """Sum of the strips' arrays (one process holds every strip)."""
    out = parts[0].clone()
    for p in parts[1:]:
        out += p
    return out


def dist_reduce(parts):
    """All-reduce (sum) of this rank's single array over the process group."""
    import torch.distributed as dist
    (t,) = parts
    t = t.clone()
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


class StripOps:
    """The per-strip steps on the GPU through libnyf."""

    def __init__(self):
        self.lib = L.load()

    def draw(self, seed, N, K):
        out = (C.c_int64 * K)()
        got = self.lib.nyf_draw_indices(int(seed) & ((1 << 64) - 1), int(N), int(K), out)
        if got != K:
            raise RuntimeError("initial-row draw did not finish")
        return torch.tensor(list(out), dtype=torch.int64, device="cuda")

    def gather(self, X, row0, idx):
        K = idx.shape[0]
        out = torch.empty((K, X.shape[1]), dtype=torch.float32, device=X.device)
        L.check(self.lib.nyf_gather_rows(nyf._ptr(X), X.shape[0], X.shape[1], int(row0),
                                         nyf._ptr(idx), K, nyf._ptr(out), nyf._stream()),
                "nyf_gather_rows")
        return out

    def partials(self, X, cent, ws):
        K, rho = cent.shape
        sums = torch.empty((K, rho + 1), dtype=torch.float64, device=X.device)
        qerr = torch.empty(1, dtype=torch.float64, device=X.device)
        L.check(self.lib.nyf_kmeans_partials(nyf._ptr(X), X.shape[0], rho, K, nyf._ptr(cent),
                                             nyf._ptr(sums), nyf._ptr(qerr), ws.cptr(), ws.nbytes,
                                             nyf._stream()), "nyf_kmeans_partials")
        return sums, qerr

    def apply(self, sums, cent):
        K, rho = cent.shape
        L.check(self.lib.nyf_kmeans_apply_sums(nyf._ptr(sums), K, rho, nyf._ptr(cent),
                                               nyf._stream()), "nyf_kmeans_apply_sums")

    def workspace(self, N, rho, K):
        return nyf.make_workspace(N, 1, rho, rho, nyf.Params(K=K))

    def filter(self, f_halo, params, landmarks):
        return nyf.blf(f_halo, params, landmarks=landmarks)


def kmeans_strips(Xs, row0s, N, K, iters, seed, reduce, ops):
    """k-means over the union of the strips' rows.

    Xs: this process's strips' own rows (N_i x rho each), row0s: the whole-image
    number of each strip's first row, N: rows of the whole image.  Returns the
    centroids (K x rho) and the error e of the last assignment (Sec. III).
    """
    idx = ops.draw(seed, N, K)
    cent = reduce([ops.gather(X, r0, idx) for X, r0 in zip(Xs, row0s)])
    rho = cent.shape[1]
    wss = [ops.workspace(X.shape[0], rho, K) for X in Xs]
    qerr = None
    for it in range(iters + 1):            # the last pass only measures e
        parts = [ops.partials(X, cent, ws) for X, ws in zip(Xs, wss)]
        sums = reduce([p[0] for p in parts])
        qerr = reduce([p[1] for p in parts])
        if it < iters:
            ops.apply(sums, cent)
    return cent, qerr


def blf_strips(f, params: nyf.Params, parts: int, ops=None):
    """The bilateral filter of f (H x W x n, guide = f) computed strip by strip in one
    process: k-means over all strips, then each strip with its halo.  Returns
    (g_hat, landmarks, e)."""
    ops = ops or StripOps()
    H, W, n = f.shape
    S = params.radius
    bounds = [strip_rows(H, parts, i) for i in range(parts)]
    Xs = [f[y0:y1].reshape(-1, n) for y0, y1 in bounds]
    cent, qerr = kmeans_strips(Xs, [y0 * W for y0, _ in bounds], H * W, params.K,
                               params.kmeans_iters, params.seed, local_reduce, ops)
    out = torch.empty_like(f)
    for y0, y1 in bounds:
        h0, h1 = halo_rows(H, y0, y1, S)
        g = ops.filter(f[h0:h1].contiguous(), params, cent)
        out[y0:y1] = g[y0 - h0:y1 - h0]
    return out, cent, qerr


def blf_strip_rank(f_halo, h0, y0, y1, H, W, params: nyf.Params, reduce=dist_reduce, ops=None):
    """One rank's strip: f_halo holds rows [h0, h0 + f_halo.shape[0]) of the image and the
    rank owns rows [y0, y1).  Returns (g_hat of the owned rows, landmarks, e)."""
    ops = ops or StripOps()
    n = f_halo.shape[2]
    X = f_halo[y0 - h0:y1 - h0].reshape(-1, n)
    cent, qerr = kmeans_strips([X], [y0 * W], H * W, params.K, params.kmeans_iters, params.seed,
                               reduce, ops)
    g = ops.filter(f_halo.contiguous(), params, cent)
    return g[y0 - h0:y1 - h0], cent, qerr
