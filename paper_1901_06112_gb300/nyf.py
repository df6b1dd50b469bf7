"""Python entry points of the GB300 Nystrom kernel filter.

Each function checks and marshals torch CUDA tensors into the C ABI of
libnyf (include/nyf.h) and enqueues the work on the current CUDA stream.
PyTorch supplies device memory and streams only; every step of the method
runs in the library's kernels.
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass

import torch

from . import _lib as L


@dataclass
class Params:
    """Filter parameters (see nyf_params in include/nyf.h)."""

    sigma_s: float = 3.0
    sigma_r: float = 30.0
    K: int = 8
    kmeans_iters: int = 10
    seed: int = 0
    eig_rel_tol: float = 1e-7
    precision: str = "fp32"        # "fp32" | "bf16": storage of the per-pixel features
    spatial: str = "gaussian"      # "gaussian" | "box" | "gaussian_iir" (recursive, Sec. IV)
    S: int = 0                     # window radius; 0 -> ceil(3 sigma_s)
    patch_radius: int = 0          # NLM patch radius
    sample_frac: float = 1.0
    conv_tile: str = "auto"        # "auto" | "wide" | "narrow" | "tensor"
    save_for_backward: bool = False  # forward keeps what blf_backward reads
    backward_mode: str = "planes"  # "planes": keep the K (n+1) convolved planes;
    #                                "recompute": the backward convolves them again (low memory)

    def c(self) -> L.NyfParams:
        return L.NyfParams(float(self.sigma_s), float(self.sigma_r), int(self.K),
                           int(self.kmeans_iters), int(self.seed) & ((1 << 64) - 1),
                           float(self.eig_rel_tol),
                           L.BF16 if self.precision == "bf16" else L.FP32,
                           {"gaussian": L.GAUSSIAN, "box": L.BOX,
                            "gaussian_iir": L.GAUSSIAN_IIR}[self.spatial], int(self.S),
                           int(self.patch_radius), float(self.sample_frac),
                           {"auto": L.TILE_AUTO, "wide": L.TILE_WIDE, "narrow": L.TILE_NARROW,
                            "tensor": L.TILE_TENSOR}[self.conv_tile],
                           0 if not self.save_for_backward else
                           {"planes": 1, "recompute": 2}[self.backward_mode])

    def for_backward(self) -> "Params":
        """A copy whose forward keeps what the backward pass reads."""
        return Params(**{**self.__dict__, "save_for_backward": True})

    @property
    def radius(self) -> int:
        return self.S if self.S > 0 else int(math.ceil(3.0 * self.sigma_s))


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check_image(t, name, channels=None):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
            and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    if channels is not None and (t.dim() != 3 or t.shape[2] != channels):
        raise ValueError(f"{name} must be H x W x {channels}")


class Workspace:
    """A 256-byte aligned device buffer of at least `nbytes` bytes."""

    def __init__(self, nbytes: int, device):
        self.buf = torch.empty(int(nbytes) + 256, dtype=torch.uint8, device=device)
        off = (-self.buf.data_ptr()) % 256
        self.ptr = self.buf.data_ptr() + off
        self.nbytes = int(nbytes)

    def cptr(self):
        return C.c_void_p(self.ptr)


def workspace_size(H, W, n, rho, params: Params) -> int:
    lib = L.load()
    p = params.c()
    s = lib.nyf_workspace_size(H, W, n, rho, C.byref(p))
    if s == 0:
        raise ValueError("invalid sizes or parameters for nyf_workspace_size")
    return int(s)


def make_workspace(H, W, n, rho, params: Params, device="cuda") -> Workspace:
    return Workspace(workspace_size(H, W, n, rho, params), device)


def blf(f, params: Params, guide=None, landmarks=None, out=None, ws: Workspace | None = None):
    """Nystrom bilateral filter (Algorithm 1): returns g_hat (H x W x n)."""
    lib = L.load()
    _check_image(f, "f")
    H, W, n = f.shape
    rho = n
    if guide is not None:
        _check_image(guide, "guide")
        if guide.shape[:2] != f.shape[:2]:
            raise ValueError("guide must have the image's H x W")
        rho = guide.shape[2]
    if landmarks is not None:
        if not (landmarks.is_cuda and landmarks.dtype == torch.float32 and landmarks.is_contiguous()
                and landmarks.shape == (params.K, rho)):
            raise ValueError("landmarks must be a contiguous float32 CUDA tensor of K x rho")
    out = torch.empty_like(f) if out is None else out
    ws = ws or make_workspace(H, W, n, rho, params, f.device)
    p = params.c()
    L.check(lib.nyf_filter_blf(_ptr(f), _ptr(guide), H, W, n, rho, C.byref(p), _ptr(landmarks),
                               _ptr(out), ws.cptr(), ws.nbytes, _stream()), "nyf_filter_blf")
    return out


def nlm(f, params: Params, landmarks=None, out=None, ws: Workspace | None = None):
    """Nystrom nonlocal means (patch guide, box window): returns g_hat."""
    lib = L.load()
    _check_image(f, "f")
    H, W, n = f.shape
    out = torch.empty_like(f) if out is None else out
    rho = n * (2 * params.patch_radius + 1) ** 2
    ws = ws or make_workspace(H, W, n, rho, params, f.device)
    p = params.c()
    L.check(lib.nyf_filter_nlm(_ptr(f), H, W, n, C.byref(p), _ptr(landmarks), _ptr(out), ws.cptr(),
                               ws.nbytes, _stream()), "nyf_filter_nlm")
    return out


def patch_pca(f, r: int, q: int):
    """PCA of the image's (2r+1)^2 n patches (PCA-NLM, Sec. IV): (mean, basis rho x q,
    eigenvalues rho, descending, ws) -- the workspace holds the device status word."""
    lib = L.load()
    _check_image(f, "f")
    H, W, n = f.shape
    rho = n * (2 * r + 1) ** 2
    mean = torch.empty(rho, dtype=torch.float32, device=f.device)
    basis = torch.empty(rho, q, dtype=torch.float32, device=f.device)
    lam = torch.empty(rho, dtype=torch.float32, device=f.device)
    nb = lib.nyf_patch_pca_workspace_size(n, r)
    if nb == 0:
        raise ValueError("patch dimension outside 1..160")
    ws = Workspace(nb, f.device)
    L.check(lib.nyf_patch_pca(_ptr(f), H, W, n, r, q, _ptr(mean), _ptr(basis), _ptr(lam), ws.cptr(),
                              ws.nbytes, _stream()), "nyf_patch_pca")
    return mean, basis, lam, ws


def pca_project(f, r: int, mean, basis):
    """The H x W x q PCA guide U_q^T (p(x) - m)."""
    lib = L.load()
    _check_image(f, "f")
    H, W, n = f.shape
    q = basis.shape[1]
    guide = torch.empty(H, W, q, dtype=torch.float32, device=f.device)
    L.check(lib.nyf_pca_project(_ptr(f), H, W, n, r, q, _ptr(mean.contiguous()),
                                _ptr(basis.contiguous()), _ptr(guide), _stream()), "nyf_pca_project")
    return guide


def make_pca_workspace(H, W, n, q, params: Params, device="cuda") -> Workspace:
    nb = L.load().nyf_pca_nlm_workspace_size(H, W, n, q, C.byref(params.c()))
    if nb == 0:
        raise ValueError("unsupported PCA-NLM configuration")
    return Workspace(nb, device)


def pca_nlm(f, q: int, params: Params, mean=None, basis=None, landmarks=None, out=None,
            ws: Workspace | None = None):
    """PCA-NLM: the patch guide (radius params.patch_radius) projected on its q leading
    principal directions (computed from f unless mean and basis are given), then the
    joint filter with that guide."""
    lib = L.load()
    _check_image(f, "f")
    H, W, n = f.shape
    out = torch.empty_like(f) if out is None else out
    ws = ws or make_pca_workspace(H, W, n, q, params, f.device)
    if landmarks is not None and landmarks.shape != (params.K, q):
        raise ValueError("landmarks must be K x q")
    p = params.c()
    L.check(lib.nyf_filter_pca_nlm(_ptr(f), H, W, n, q, C.byref(p),
                                   _ptr(None if mean is None else mean.contiguous()),
                                   _ptr(None if basis is None else basis.contiguous()),
                                   _ptr(landmarks), _ptr(out), ws.cptr(), ws.nbytes, _stream()),
            "nyf_filter_pca_nlm")
    return out


def kmeans(X, K, iters=10, seed=0, init_idx=None, ws: Workspace | None = None):
    """k-means landmarks of the rows of X (N x rho): (centroids, labels, qerr)."""
    lib = L.load()
    if not (X.is_cuda and X.dtype == torch.float32 and X.is_contiguous() and X.dim() == 2):
        raise TypeError("X must be a contiguous float32 CUDA tensor of N x rho")
    N, rho = X.shape
    cent = torch.empty((K, rho), dtype=torch.float32, device=X.device)
    labels = torch.empty(N, dtype=torch.int32, device=X.device)
    qerr = torch.empty(1, dtype=torch.float64, device=X.device)
    if init_idx is not None:
        init_idx = init_idx.to(device=X.device, dtype=torch.int64).contiguous()
    ws = ws or make_workspace(N, 1, rho, rho, Params(K=K))
    L.check(lib.nyf_kmeans(_ptr(X), N, rho, K, iters, int(seed) & ((1 << 64) - 1),
                           _ptr(init_idx), _ptr(cent), _ptr(labels), _ptr(qerr), ws.cptr(),
                           ws.nbytes, _stream()), "nyf_kmeans")
    return cent, labels, qerr


def features(guide2d, landmarks, sigma_r, eig_rel_tol=1e-7, precision="fp32",
             ws: Workspace | None = None):
    """Per-pixel Nystrom features: (phi K x N, rank, alphas)."""
    lib = L.load()
    N, rho = guide2d.shape
    K = landmarks.shape[0]
    dt = torch.bfloat16 if precision == "bf16" else torch.float32
    phi = torch.zeros((K, N), dtype=dt, device=guide2d.device)
    rank = torch.zeros(1, dtype=torch.int32, device=guide2d.device)
    alphas = torch.zeros(K, dtype=torch.float64, device=guide2d.device)
    ws = ws or make_workspace(N, 1, rho, rho, Params(K=K, precision=precision))
    L.check(lib.nyf_features(_ptr(guide2d), N, rho, _ptr(landmarks), K, float(sigma_r),
                             float(eig_rel_tol), L.BF16 if precision == "bf16" else L.FP32,
                             _ptr(phi), _ptr(rank), _ptr(alphas), ws.cptr(), ws.nbytes,
                             _stream()), "nyf_features")
    return phi, rank, alphas


def stats(ws: Workspace) -> dict:
    """Device-side results of the last call on `ws` (synchronises the stream)."""
    lib = L.load()
    s = L.NyfStats()
    L.check(lib.nyf_get_stats(ws.cptr(), C.byref(s), _stream()), "nyf_get_stats")
    return {k: getattr(s, k) for k, _ in L.NyfStats._fields_}


# ----------------------------------------------------------------------------- backward

class BackwardBuffers:
    """Output buffers of the backward pass: dL/df, dL/dguide (joint guide) and dL/dsigma."""

    def __init__(self, f, guide=None):
        self.grad_f = torch.empty_like(f)
        self.grad_guide = None if guide is None else torch.empty_like(guide)
        self.grad_sigma = torch.zeros(2, dtype=torch.float32, device=f.device)


def blf_backward_available() -> bool:
    return True


def blf_backward(f, params: Params, out, grad_out, ws: Workspace, bufs: BackwardBuffers = None,
                 guide=None) -> BackwardBuffers:
    """Adjoint of blf(): must follow the forward call that produced `out` on `ws`,
    made with params.save_for_backward set (Params.for_backward()).

    Landmarks, the window radius and the kept modes are held at their forward
    values.  Returns the buffers (grad_f is the total derivative when the guide
    is the image).
    """
    lib = L.load()
    _check_image(grad_out, "grad_out")
    H, W, n = f.shape
    rho = n if guide is None else guide.shape[2]
    bufs = bufs or BackwardBuffers(f, guide)
    p = params.c()
    L.check(lib.nyf_filter_blf_backward(_ptr(f), _ptr(guide), H, W, n, rho, C.byref(p), _ptr(out),
                                        _ptr(grad_out), _ptr(bufs.grad_f), _ptr(bufs.grad_guide),
                                        _ptr(bufs.grad_sigma), ws.cptr(), ws.nbytes, _stream()),
            "nyf_filter_blf_backward")
    return bufs


def blf_vjp(f, params: Params, grad_out, guide=None, landmarks=None) -> dict:
    """Forward + backward: gradients of sum(grad_out * g_hat)."""
    params = params.for_backward()
    H, W, n = f.shape
    rho = n if guide is None else guide.shape[2]
    ws = make_workspace(H, W, n, rho, params, f.device)
    out = blf(f, params, guide=guide, landmarks=landmarks, ws=ws)
    b = blf_backward(f, params, out, grad_out.contiguous(), ws, guide=guide)
    gs = b.grad_sigma.cpu()
    return {"out": out, "df": b.grad_f, "dp": b.grad_guide, "dsigma_r": float(gs[0]),
            "dsigma_s": float(gs[1])}


class NyfBLF(torch.autograd.Function):
    """Differentiable Nystrom bilateral filter (w.r.t. image, guide, sigma_r, sigma_s).

    Landmarks are a stop-gradient input (computed by k-means when None).
    """

    @staticmethod
    def forward(ctx, f, guide, sigma_r, sigma_s, params: Params, landmarks=None):
        P = params.for_backward()
        P.sigma_r = float(sigma_r)
        P.sigma_s = float(sigma_s)
        f = f.contiguous()
        g = None if guide is None else guide.contiguous()
        H, W, n = f.shape
        rho = n if g is None else g.shape[2]
        ws = make_workspace(H, W, n, rho, P, f.device)
        out = blf(f, P, guide=g, landmarks=landmarks, ws=ws)
        ctx.P, ctx.ws, ctx.has_guide = P, ws, g is not None
        ctx.save_for_backward(f, g if g is not None else torch.empty(0, device=f.device), out)
        ctx.sig_dev = (sigma_r.device if isinstance(sigma_r, torch.Tensor) else None,
                       sigma_s.device if isinstance(sigma_s, torch.Tensor) else None)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        f, g, out = ctx.saved_tensors
        g = g if ctx.has_guide else None
        b = blf_backward(f, ctx.P, out, grad_out.contiguous(), ctx.ws, guide=g)
        dsr = b.grad_sigma[0]
        dss = b.grad_sigma[1]
        dev_r, dev_s = ctx.sig_dev
        dsr = dsr.to(dev_r) if dev_r is not None else None
        dss = dss.to(dev_s) if dev_s is not None else None
        return b.grad_f, b.grad_guide, dsr, dss, None, None


def blf_autograd(f, sigma_r, sigma_s, params: Params, guide=None, landmarks=None):
    """g_hat with autograd support; sigma_r / sigma_s may be 0-dim tensors."""
    return NyfBLF.apply(f, guide, sigma_r, sigma_s, params, landmarks)


# ----------------------------------------------------------------------------- batched

class Batched:
    """A batch of colour images of uneven sizes filtered by one call per pass.

    The images live packed (HWC, back to back) in one device buffer; image b
    has its own sigma_s, sigma_r (and optionally a tuned convolution variant).
    forward()/backward() enqueue the whole batch; capture() records one
    forward + backward into a CUDA graph that replay() launches again.
    """

    TILES = {"auto": L.TILE_AUTO, "wide": L.TILE_WIDE, "narrow": L.TILE_NARROW,
             "tensor": L.TILE_TENSOR}

    def __init__(self, shapes, sigmas_s, sigmas_r, params: Params, n=3, device="cuda",
                 tiles=None, backward=True):
        self.lib = L.load()
        self.B = len(shapes)
        self.n = n
        params = params.for_backward() if backward else params
        self.params = params
        self.items = (L.NyfBatchItem * self.B)()
        # the library's window radius: ceil(3 sigma_s) of the float32 sigma_s
        self.radii = [params.S if params.S > 0 else math.ceil(3.0 * C.c_float(float(s)).value)
                      for s in sigmas_s]
        if tiles == "tuned":                     # the autotuner's variant per radius and size
            from . import tune
            tiles = tune.tune_images([(int(H), int(W)) for H, W in shapes], self.radii, params.K,
                                     params.precision)
        self.tiles = list(tiles) if tiles else None
        off = 0
        self.offsets = []
        for b, (H, W) in enumerate(shapes):
            t = self.TILES[tiles[b]] if tiles else L.TILE_AUTO
            self.items[b] = L.NyfBatchItem(off, int(H), int(W), float(sigmas_s[b]),
                                           float(sigmas_r[b]), t, 0)
            self.offsets.append(off)
            off += int(H) * int(W) * n
        self.total = off
        self.shapes = [(int(H), int(W)) for H, W in shapes]
        self._p = params.c()
        nbytes = self.lib.nyf_batched_workspace_size(self.items, self.B, n, C.byref(self._p))
        if nbytes == 0:
            raise ValueError("invalid batch for nyf_batched_workspace_size")
        self.ws = Workspace(nbytes, device)
        self.grad_sigma = torch.zeros((self.B, 2), dtype=torch.float32, device=device)
        self.graph = None

    def pack(self, images):
        return torch.cat([torch.as_tensor(im).reshape(-1) for im in images]).to(
            self.ws.buf.device, torch.float32).contiguous()

    def unpack(self, flat):
        out = []
        for (H, W), o in zip(self.shapes, self.offsets):
            out.append(flat[o:o + H * W * self.n].view(H, W, self.n))
        return out

    def set_tiles(self, tiles):
        """Convolution variant per image ("wide", "narrow", "tensor" or "auto")."""
        for b, t in enumerate(tiles):
            self.items[b].conv_tile = self.TILES[t]
        self.tiles = list(tiles)

    def tune_tiles(self, f, landmarks=None, reps=3, gain=0.01):
        """Tunes the convolution variants in the batch itself: starting from the
        library's defaults, each group of images with the same radius and size class
        tries the other variants, and a change is kept when the whole batch's forward
        gets faster by more than `gain` (the images share the GPU, so an image's best
        variant alone is not always the batch's).  Returns the tiles it keeps."""
        from . import tune
        n3 = self.n <= 3
        cur = ["tensor" if self.params.precision == "bf16" and S <= 16 and n3 else "wide"
               for S in self.radii]
        groups = {}
        for b, ((H, W), S) in enumerate(zip(self.shapes, self.radii)):
            groups.setdefault((S, tune.size_class(H, W)), []).append(b)
        out = torch.empty_like(f)

        def run(tiles):
            self.set_tiles(tiles)
            self.forward(f, out, landmarks)
            torch.cuda.synchronize()
            best = math.inf
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(torch.cuda.current_stream())
                self.forward(f, out, landmarks)
                e1.record(torch.cuda.current_stream())
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1))
            return best

        best_t = run(cur)
        for (S, _), idx in sorted(groups.items()):
            cands = [c for c in tune.candidates(S, self.params.precision)
                     if not (c == "tensor" and not n3)]
            for c in cands:
                if c == cur[idx[0]]:
                    continue
                trial = list(cur)
                for b in idx:
                    trial[b] = c
                t = run(trial)
                if t < best_t * (1.0 - gain):
                    best_t, cur = t, trial
        self.set_tiles(cur)
        return cur

    def forward(self, f, out=None, landmarks=None):
        """Forward of every image; landmarks: None (k-means per image) or a
        B x K x n float32 CUDA tensor."""
        out = torch.empty_like(f) if out is None else out
        if landmarks is not None and not (
                landmarks.is_cuda and landmarks.dtype == torch.float32
                and landmarks.is_contiguous() and landmarks.shape == (self.B, self.params.K, self.n)):
            raise ValueError("landmarks must be a contiguous float32 CUDA tensor of B x K x n")
        L.check(self.lib.nyf_filter_blf_batched(_ptr(f), self.items, self.B, self.n,
                                                C.byref(self._p), _ptr(landmarks), _ptr(out),
                                                self.ws.cptr(), self.ws.nbytes, _stream()),
                "nyf_filter_blf_batched")
        return out

    def backward(self, f, out, grad_out, grad_f=None):
        grad_f = torch.empty_like(f) if grad_f is None else grad_f
        L.check(self.lib.nyf_filter_blf_batched_backward(
            _ptr(f), self.items, self.B, self.n, C.byref(self._p), _ptr(out), _ptr(grad_out),
            _ptr(grad_f), _ptr(self.grad_sigma), self.ws.cptr(), self.ws.nbytes, _stream()),
            "nyf_filter_blf_batched_backward")
        return grad_f, self.grad_sigma

    def stats(self, b):
        s = L.NyfStats()
        L.check(self.lib.nyf_batched_stats(self.ws.cptr(), self.items, self.B, self.n,
                                           C.byref(self._p), b, C.byref(s), _stream()),
                "nyf_batched_stats")
        return {k: getattr(s, k) for k, _ in L.NyfStats._fields_}

    def capture(self, f, grad_out, landmarks=None):
        """Record forward + backward on static buffers into a CUDA graph (the
        warm-up call before it also creates the library's stream pool outside
        the capture)."""
        self.f_static, self.g_static, self.lm_static = f, grad_out, landmarks
        self.out_static = torch.empty_like(f)
        self.gf_static = torch.empty_like(f)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):                # warm-up outside the graph
            self.forward(f, self.out_static, landmarks)
            self.backward(f, self.out_static, grad_out, self.gf_static)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.forward(self.f_static, self.out_static, self.lm_static)
            self.backward(self.f_static, self.out_static, self.g_static, self.gf_static)
        return self.out_static, self.gf_static, self.grad_sigma

    def replay(self):
        self.graph.replay()
        return self.out_static, self.gf_static, self.grad_sigma
