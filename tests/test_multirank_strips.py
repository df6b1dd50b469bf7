"""Strip processing across ranks, on the CPU: two gloo ranks on 127.0.0.1 each
hold one horizontal strip of the image with its S-row halo and run the strip
driver (paper_1901_06112_gb300.strips) -- the initial rows gathered by their
owners and summed, per-cluster sums and counts all-reduced every Lloyd
iteration, the filter of each strip with its halo -- with the per-strip steps
done by the FP64 oracle.  The assembled result equals the oracle's k-means and
its filter of the whole image: the driver's partition, halo, reductions and
update rule are those of the single image."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
H, W, K, ITERS, SEED, SIGMA_S, SIGMA_R = 45, 38, 5, 4, 11, 2.0, 40.0


def _image():
    from paper_1901_06112_gb300 import synth
    return synth.voronoi_colour(H, W, 9, 8.0, 21).astype(np.float64)


class OracleOps:
    """The per-strip steps in FP64 with the oracle (CPU tensors)."""

    def draw(self, seed, N, k):
        import torch
        from oracle import rng
        return torch.from_numpy(rng.distinct_indices(seed, k, N))

    def gather(self, X, row0, idx):
        import torch
        out = torch.zeros((idx.shape[0], X.shape[1]), dtype=torch.float64)
        for j, i in enumerate(idx.tolist()):
            if 0 <= i - row0 < X.shape[0]:
                out[j] = X[i - row0]
        return out

    def workspace(self, N, rho, k):
        return None

    def partials(self, X, cent, ws):
        import torch
        from oracle import kmeans as km
        c, e = km.assign(X.numpy(), cent.numpy())
        sums = np.zeros((cent.shape[0], cent.shape[1] + 1))
        for j in range(cent.shape[0]):
            sums[j, :-1] = X.numpy()[c == j].sum(axis=0)
            sums[j, -1] = np.sum(c == j)
        return torch.from_numpy(sums), torch.tensor([e], dtype=torch.float64)

    def apply(self, sums, cent):
        cnt = sums[:, -1:]
        upd = cnt[:, 0] > 0
        cent[upd] = sums[upd, :-1] / cnt[upd]

    def filter(self, f_halo, params, landmarks):
        import torch
        from oracle import kernels as Kr
        from oracle import nystrom as ny
        f = f_halo.numpy()
        return torch.from_numpy(ny.nystrom_filter(f, f, landmarks.numpy(), params.sigma_r,
                                                  Kr.gaussian_taps(params.sigma_s, params.radius),
                                                  1e-7))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1901_06112_gb300 import nyf, strips
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from test_multirank_strips import OracleOps, _image
    f = torch.from_numpy(_image())
    P = nyf.Params(sigma_s=SIGMA_S, sigma_r=SIGMA_R, K=K, kmeans_iters=ITERS, seed=SEED)
    y0, y1 = strips.strip_rows(H, world, rank)
    h0, h1 = strips.halo_rows(H, y0, y1, P.radius)
    g, cent, qerr = strips.blf_strip_rank(f[h0:h1].clone(), h0, y0, y1, H, W, P,
                                          reduce=strips.dist_reduce, ops=OracleOps())
    q.put((rank, y0, y1, g.numpy(), cent.numpy(), float(qerr[0])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_filter_their_strips_like_the_whole_image():
    sys.path.insert(0, ROOT)
    from oracle import kernels as Kr
    from oracle import nystrom as ny
    from oracle import pipeline as pl
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    f = _image()
    mu, info = pl.landmarks(f.reshape(-1, 3), K, ITERS, SEED)
    want = ny.nystrom_filter(f, f, mu, SIGMA_R, Kr.gaussian_taps(SIGMA_S, 6), 1e-7)
    out = np.zeros_like(f)
    for rank, y0, y1, g, cent, qerr in res:
        assert np.allclose(cent, mu, rtol=0, atol=1e-10)          # every rank: the same landmarks
        assert abs(qerr - info["e"]) <= 1e-10 * info["e"]
        out[y0:y1] = g
    assert [r[1:3] for r in res] == [(0, 22), (22, 45)]
    assert np.max(np.abs(out - want)) <= 1e-9 * np.max(np.abs(want))
