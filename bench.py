#!/usr/bin/env python3
"""Throughput of the Nystrom bilateral filter on GB300 (megapixels/s).

Workload (default): the 1920 x 1080 x 3 colour bilateral filter -- 400
Voronoi cells with sinusoidal shading and noise 15, sigma_s 5 (31 x 31
window), sigma_r 40, K 32 k-means landmarks (10 Lloyd iterations).  One step
is one pass of the whole path on one image: k-means, FP64-accurate
eigendecomposition, features, convolutions + combine, then (default
--mode fwdbwd) the backward pass w.r.t. the image, sigma_r and sigma_s.
Inputs are resident in HBM; L2 is flushed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|bf16]
                       [--mode fwd|fwdbwd] [--impl nyf|reference]
For N > 1 the script runs under torchrun: every rank filters its own image
(independent replicas, no collective on the data path) and rank 0 prints the
JSON line.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "megapixels/s (fwd, fwd+bwd) at stated RMSE vs FP64 oracle; % of roofline"
FP32_LANES_PER_SM = 128
SMS = 152
SM_MAX_MHZ = 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16"])
    ap.add_argument("--mode", default="fwdbwd", choices=["fwd", "fwdbwd"])
    ap.add_argument("--spatial", default="gaussian", choices=["gaussian", "gaussian_iir"],
                    help="omega: truncated FIR Gaussian, or the recursive Gaussian (forward, fp32)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the forward-only, BF16 and batched side measurements")
    ap.add_argument("--workload", default="colour_hd",
                    choices=["colour_hd", "colour_256", "hyperspectral", "nlm"],
                    help="the timed single-image workload (default: the 1920x1080 colour BLF); "
                         "nlm runs the forward only")
    ap.add_argument("--crop", type=int, nargs=2, metavar=("H", "W"), default=None,
                    help="time the top-left H x W crop of the workload instead (a smaller case "
                         "for profiling; no accuracy pass and no extras)")
    ap.add_argument("--impl", default="nyf", choices=["nyf", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


# ----------------------------------------------------------------------------- CPU oracle leg

CPU_SAMPLE = (192, 192)     # crop of the workload the oracle filters (and differentiates) per step

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the convolution kernels
# on the 1920 x 1080, K = 32 workload, from the ncu captures summarised in
# profiles/ncu_conv_kernels_colour_blf_1920x1080.md; only for the kernels as captured.
NCU_TRAFFIC = {("conv_bwd", "fp32"): 1.421e9 + 0.250e9,   # profiles/ncu_conv_bwd_colour_blf_512x1024_crop.md
               ("conv_combine", "fp32"): 0.323e9 + 1.035e9, ("conv_combine", "bf16"): 0.315e9 + 1.034e9,
               # both recursive-Gaussian passes (k_cols + k_rows), sigma_s 5, from
               # profiles/ncu_recursive_gaussian_colour_blf_1920x1080.md
               ("recursive_pair", "fp32"): 0.625e9 + 1.025e9 + 1.327e9 + 0.032e9}


def weak_scaling_value(ms, megapixels, world, device, dist=None):
    """Max over ranks of the per-step time and the whole-job throughput: every rank
    filters its own replica (one image each), so value = ranks x megapixels / slowest."""
    import torch
    t = torch.tensor([float(ms)], device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * megapixels / (ms_max / 1e3)


def replica_seed(base_seed, rank):
    """Seed of rank `rank`'s replica (each rank draws its own landmarks)."""
    return base_seed + rank


def hbm_peak():
    """Measured copy bandwidth (GB/s) on this machine type, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def iir_bytes_per_pixel(K, n):
    """Algorithmic DRAM bytes per pixel of the convolution + combine stage (the method's
    own traffic): phi (4 K) and f (4 n) read, g_hat (4 n) and eta (4) written."""
    return 4 * K + 8 * n + 4


def iir_design_bytes_per_pixel(K, n):
    """DRAM bytes per pixel of the two recursive-Gaussian passes as built: the column pass
    reads phi and f and writes the K (n + 1) vertically filtered planes Y; the row pass
    reads Y and phi and writes g_hat and eta."""
    return 4 * K + 4 * n + 4 * K * (n + 1) + 4 * K * (n + 1) + 4 * K + 4 * n + 4


def bf16_tensor_peak():
    """Dense BF16 tensor peak (TFLOP/s, burst) measured on this machine type, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops"]), "measured"
    except (OSError, ValueError, KeyError):
        return 1900.0, "fallback"


def _oracle_step_code(h, w, backward):
    return f"""
import os, sys, time, json
sys.path.insert(0, {ROOT!r})
import numpy as np
from paper_1901_06112_gb300 import synth
from oracle import pipeline as pl, grad as gr
wl = synth.colour_blf_hd()
f = wl.f[:{h}, :{w}].astype(np.float64)
t0 = time.perf_counter()
g, mu, info = pl.blf(f, wl.sigma_s, wl.sigma_r, wl.K, iters=wl.kmeans_iters, seed=wl.seed)
if {backward!r}:
    G = np.random.default_rng(0).normal(size=f.shape)
    gr.vjp(f, f, mu, wl.sigma_r, wl.sigma_s, wl.radius, 1e-7, G, guide_is_image=True)
dt = time.perf_counter() - t0
print(json.dumps({{"seconds": dt, "pixels": {h * w}}}))
"""


def cpu_oracle_seconds(h=CPU_SAMPLE[0], w=CPU_SAMPLE[1], backward=True):
    """Time the FP64 oracle (k-means + Algorithm 1, and its gradient) on an h x w crop."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", _oracle_step_code(h, w, backward)],
                       capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["seconds"], d["pixels"]


def cpu_baseline_obj(backward=True):
    sec, px = cpu_oracle_seconds(backward=backward)
    what = "forward + backward" if backward else "forward"
    return {"value": px / 1e6 / sec, "unit": "megapixels/s", "cores": 1, "kind": "oracle",
            "sample": f"FP64 oracle {what} (k-means 10 iters + Algorithm 1"
                      f"{' + autograd gradient' if backward else ''}) on a {CPU_SAMPLE[0]}x"
                      f"{CPU_SAMPLE[1]} crop of the workload, one thread, {sec:.1f} s"}


def cpu_model():
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu part", "hardware")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_fp32_baseline(wl, reps=3):
    """The FP32 C++/OpenMP filter (same algorithm as the GPU path, forward) on the host:
    the whole workload with every core, and a 512 x 512 crop with one thread; median of
    `reps` runs each, megapixels/s."""
    from oracle import cpu_build
    lib = cpu_build.load()
    res = {}
    for label, f, threads in (("all_cores", wl.f, 0), ("one_thread", wl.f[:512, :512], 1)):
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            _, code = cpu_build.blf(lib, f, wl.sigma_s, wl.sigma_r, wl.K, wl.kmeans_iters, wl.seed,
                                    threads=threads)
            ts.append(time.perf_counter() - t0)
            if code != 0:
                raise RuntimeError(f"cpu baseline status {code}")
        sec = float(np.median(ts))
        res[label] = {"value": f.shape[0] * f.shape[1] / 1e6 / sec, "seconds": sec,
                      "threads": threads if threads else lib.nyf_cpu_threads(),
                      "pixels": f.shape[0] * f.shape[1]}
    res.update({"unit": "megapixels/s", "kind": "fp32 C++/OpenMP, forward (k-means 10 iters, "
                "eig, features, FIR convolutions, combine)", "cpu": cpu_model(),
                "os_cpu_count": os.cpu_count()})
    return res


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps = max(1, args.steps)
    times = []
    px = 0
    for _ in range(max(0, min(args.warmup, 1))):
        cpu_oracle_seconds(64, 64, backward=args.mode == "fwdbwd")
    # each step is a bounded sample of the workload (a crop, forward + backward)
    bwd = args.mode == "fwdbwd"
    for _ in range(min(steps, 3)):
        sec, px = cpu_oracle_seconds(backward=bwd)
        times.append(sec)
    sec = float(np.median(times))
    v = px / 1e6 / sec
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "megapixels/s",
            "n_gpus": args.gpus, "steps": len(times), "warmup": args.warmup,
            "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"colour_blf_1920x1080_K32 ({CPU_SAMPLE[0]}x{CPU_SAMPLE[1]} "
                                   "crop per step)",
                       "sigma_s": 5.0, "sigma_r": 40.0, "K": 32, "mode": args.mode},
            "cpu_baseline": {"value": v, "unit": "megapixels/s", "cores": 1, "kind": "oracle",
                             "sample": f"{CPU_SAMPLE[0]}x{CPU_SAMPLE[1]} crop of the 1920x1080 "
                                       "workload per step, FP64 oracle, one thread"},
            "e2e": {"value": v, "unit": "megapixels/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- GPU leg

def conv_flops_per_pixel(K, n, S):
    """Algorithmic FLOPs of the forward convolution + combine per pixel.

    K (n + 1) planes, each a separable FIR of 2 passes x (2S + 1) taps x 2 FLOP,
    plus the combine multiply-add of every plane.
    """
    return K * (n + 1) * (2 * (2 * S + 1) * 2 + 2)


def conv_bwd_flops_per_pixel(K, n, S):
    """Algorithmic FLOPs of the adjoint convolutions per pixel.

    The forward keeps C = omega * (phi f), so per plane the backward convolves
    u = a phi with omega and with omega' = g' (x) g + g (x) g': a vertical
    (g, g') pass and three horizontal passes (g and g' on the vertical g result,
    g on the vertical g' result) = 5 passes x (2S + 1) taps x 2 FLOP, plus 10
    FLOP of products (u; a C + f B; phi B; phi f B').
    """
    return K * (n + 1) * (5 * (2 * S + 1) * 2 + 10)


STAGES = ["landmarks", "eig", "features", "conv_combine", "bwd_conv", "bwd_features"]

# Peaks of the step roofline.  FP32: 152 SMs x 128 lanes x 2 FLOP x 2070 MHz (derived
# from the unit counts and the maximum clock).  SFU: 16 special-function results per SM
# and clock (the exp of the features) x 152 SMs x 2070 MHz, derived the same way.
SFU_PER_SM_CLK = 16


def peaks():
    """Roofline denominators: HBM GB/s and BF16 TFLOP/s sustained (measured), FP32 TFLOP/s
    and SFU Gop/s (derived)."""
    hbm, how = hbm_peak()
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            tc, tc_how = float(json.load(fh)["bf16_tflops_sustained"]), "measured"
    except (OSError, ValueError, KeyError):
        tc, tc_how = 1700.0, "fallback"
    fp32 = SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    sfu = SMS * SFU_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e9
    return {"hbm_GBs": hbm, "tc_TFLOPs": tc, "fp32_TFLOPs": fp32, "sfu_Gops": sfu,
            "basis": f"HBM copy ({how}), BF16 dense sustained ({tc_how}); FP32 and SFU derived "
                     "from 152 SMs x 128 lanes x 2 FLOP and x 16 results per clock at 2070 MHz"}


def stage_counts(N, n, rho, K, T, iters, Ns, fwdbwd, conv_tensor=False, feat_tensor=None,
                 keep_planes=True, nlm_r=0, box=False):
    """Algorithmic work of each stage of one step (the method's own counts, not the
    kernels'): {stage: (bytes, fp32 FLOP, tensor FLOP, exp)}.

    N pixels, n channels, rho guide dimension, K modes, T = 2S + 1 taps, `iters` Lloyd
    iterations on Ns rows.  k-means: 3 rho K FLOP per row and iteration, the rows read
    once per iteration.  Features: the distance contraction 2 rho K, exp, E W_hat 2 K^2
    per pixel (on the tensor cores for rho >= 16); guide (or, for NLM, image) read, phi
    written.  Convolutions: per plane 2 passes x T taps x 2 FLOP + 2 for the combine
    (forward), 5 passes + 10 (backward, over the saved planes C); f and phi read, g_hat
    and eta written, C written (forward) and read (backward) when kept.
    """
    if feat_tensor is None:
        feat_tensor = rho >= 16
    q = n + 1
    c = {}
    c["landmarks"] = (4.0 * rho * Ns * iters, 3.0 * rho * K * Ns * iters, 0.0, 0.0)
    c["eig"] = (0.0, 0.0, 0.0, 0.0)         # K x K, latency only
    guide_bytes = 4 * n if nlm_r else 4 * rho
    feat_flop = (2.0 * rho * K + 2.0 * K * K) * N
    c["features"] = (N * (guide_bytes + 4.0 * K), 0.0 if feat_tensor else feat_flop,
                     feat_flop if feat_tensor else 0.0, float(N * K))
    # box window by running sums: 2 passes x (one add, one subtract) per output + the combine
    conv_flop = N * K * q * ((2.0 * 2 + 2) if box else (2.0 * T * 2 + 2))
    cbytes = 4.0 * K * q * N if (fwdbwd and keep_planes) else 0.0
    c["conv_combine"] = (N * (4.0 * n + 4.0 * K + 4.0 * n + 4.0) + cbytes,
                         0.0 if conv_tensor else conv_flop, conv_flop if conv_tensor else 0.0, 0.0)
    if fwdbwd:
        bflop = N * K * q * (5.0 * T * 2 + 10)
        if not keep_planes:
            bflop += conv_flop
        c["bwd_conv"] = (N * (4.0 * K + 8.0 * q + 4.0 * n * 3 + 4.0 + 4.0 * K + 4.0 * n) + cbytes,
                         bflop, 0.0, 0.0)
        c["bwd_features"] = (N * (4.0 * K + 4.0 * rho + 8.0 * n),
                             N * (4.0 * K * K + 4.0 * rho * K), 0.0, float(N * K))
    return c


def step_roofline(counts, stage_ms, step_ms):
    """Sec. 8(d) roofline time of a step: sum over stages of the largest of bytes / HBM,
    FP32 FLOP / FP32 peak, tensor FLOP / tensor peak and exp / SFU rate; frac = that
    sum / the measured step time.  Also the binding resource of each stage."""
    pk = peaks()
    total, per = 0.0, {}
    for s, (b, fl, tc, ex) in counts.items():
        times = {"hbm": b / (pk["hbm_GBs"] * 1e9), "fp32": fl / (pk["fp32_TFLOPs"] * 1e12),
                 "tensor": tc / (pk["tc_TFLOPs"] * 1e12), "sfu": ex / (pk["sfu_Gops"] * 1e9)}
        bound = max(times, key=times.get)
        t = times[bound] * 1e3
        total += t
        got = stage_ms.get(s)
        per[s] = {"bound": bound, "roofline_ms": t, "measured_ms": got,
                  "frac": (t / got) if got else None}
    return {"roofline_ms": total, "step_ms": step_ms, "frac": total / step_ms, "stages": per,
            "peaks": pk}


def timed_steps(step, steps, flush, stream, lib):
    """Per-step CUDA-event times (ms) and per-stage library event times."""
    import ctypes as C
    import torch
    buf = (C.c_float * 7)()
    step_ms, stage_ms = [], []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        lib.nyf_get_timing(buf, 7)
        stage_ms.append([buf[i] for i in range(7)])
    st = np.array(stage_ms)
    means = [float(np.mean(st[:, i][st[:, i] >= 0])) if np.any(st[:, i] >= 0) else None
             for i in range(7)]
    return float(np.mean(step_ms)), means


def golden_landmarks(name):
    """The oracle's k-means landmarks of a workload, stored by tests/golden/make_landmarks.py."""
    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    import make_landmarks
    return make_landmarks.load(name)


def _rel(got, want):
    got, want = np.asarray(got, np.float64), np.asarray(want, np.float64)
    return float(np.linalg.norm(got - want) / np.linalg.norm(want)), float(np.max(np.abs(got - want)))


def accuracy_blf(nyf, w, mu, precision, fwdbwd, samples=256, guide=None):
    """The library's output on workload w with the oracle's landmarks mu against the FP64
    oracle (Algorithm 1 by direct window sums) on `samples` seeded pixels; with fwdbwd also
    the gradients w.r.t. the image and both sigmas for a cotangent on a 24 x 24 window,
    against the oracle's autograd on the window grown by S (exact there)."""
    import torch
    from oracle import grad as gr
    from oracle import kernels as Kr
    from oracle import nystrom as ny
    from paper_1901_06112_gb300 import synth
    sr = float(np.float32(w.sigma_r))
    P = nyf.Params(sigma_s=w.sigma_s, sigma_r=sr, K=w.K, precision=precision, spatial=w.spatial,
                   S=w.S, patch_radius=w.patch_radius, sample_frac=w.sample_frac)
    f = torch.from_numpy(w.f).cuda()
    mut = torch.from_numpy(np.ascontiguousarray(mu, np.float32)).cuda()
    taps = Kr.box_taps(w.radius) if w.spatial == "box" else Kr.gaussian_taps(w.sigma_s, w.radius)
    idx = synth.sample_indices(w.H * w.W, samples, 17)
    ys, xs = idx // w.W, idx % w.W
    if w.patch_radius > 0:
        from oracle import guide as gd
        out = nyf.nlm(f, P, landmarks=mut).cpu().numpy()
        p = gd.patch_guide(w.f.astype(np.float64), w.patch_radius)
    else:
        out = nyf.blf(f, P, landmarks=mut).cpu().numpy()
        p = w.f
    want = ny.nystrom_filter_at(w.f, p, mu.astype(np.float64), sr, taps, 1e-7, ys, xs)
    r, m = _rel(out[ys, xs], want)
    acc = {"vs": f"FP64 oracle, Algorithm 1 with the oracle's k-means landmarks, {len(ys)} pixels",
           "rel_rmse": r, "max_abs": m}
    if fwdbwd and w.patch_radius == 0:
        S, h = w.radius, 24
        y0, x0 = w.H // 2 - h // 2, w.W // 2 - h // 2
        G = np.zeros(w.f.shape, np.float32)
        G[y0:y0 + h, x0:x0 + h] = np.random.default_rng(7).normal(size=(h, h, w.n))
        res = nyf.blf_vjp(f, P, torch.from_numpy(G).cuda(), landmarks=mut)
        c0, c1 = (max(0, y0 - S), min(w.H, y0 + h + S)), (max(0, x0 - S), min(w.W, x0 + h + S))
        crop = w.f[c0[0]:c0[1], c1[0]:c1[1]]
        ref = gr.vjp(crop, crop, mu, sr, w.sigma_s, S, 1e-7, G[c0[0]:c0[1], c1[0]:c1[1]],
                     guide_is_image=True)
        rg, mg = _rel(res["df"].cpu().numpy()[c0[0]:c0[1], c1[0]:c1[1]], ref["df"])
        acc["grad_f"] = {"rel_rmse": rg, "max_abs": mg, "window": f"{h}x{h} at ({y0},{x0})"}
        for nm in ("dsigma_r", "dsigma_s"):
            acc[nm] = {"rel": abs(res[nm] - ref[nm]) / abs(ref[nm])}
    return acc


def config_line(nyf, lib, w, golden, precision, fwdbwd, steps, flush, stream):
    """One workload measured like the headline: the whole call (k-means on the device,
    eig, features, convolutions [, backward]) per step, per-stage CUDA events, the
    Sec. 8(d) step roofline, and the accuracy pass with the oracle's landmarks."""
    import torch
    H, W, n = w.f.shape
    sr = float(np.float32(w.sigma_r))
    P = nyf.Params(sigma_s=w.sigma_s, sigma_r=sr, K=w.K, kmeans_iters=w.kmeans_iters, seed=w.seed,
                   precision=precision, spatial=w.spatial, S=w.S, patch_radius=w.patch_radius,
                   sample_frac=w.sample_frac, save_for_backward=fwdbwd)
    f = torch.from_numpy(w.f).cuda()
    rho = n * (2 * w.patch_radius + 1) ** 2 if w.patch_radius else n
    ws = nyf.make_workspace(H, W, n, rho, P)
    out = torch.empty_like(f)
    G = torch.randn(f.shape, generator=torch.Generator().manual_seed(1)).cuda()
    grads = nyf.BackwardBuffers(f)

    def step():
        if w.patch_radius:
            nyf.nlm(f, P, out=out, ws=ws)
        else:
            nyf.blf(f, P, out=out, ws=ws)
        if fwdbwd:
            nyf.blf_backward(f, P, out, G, ws, grads)
    lib.nyf_set_timing(1)
    for _ in range(3):
        step()
    ms, stages = timed_steps(step, steps, flush, stream, lib)
    lib.nyf_set_timing(0)
    st = nyf.stats(ws)
    N = H * W
    Ns = max(1, int(np.floor(w.sample_frac * N + 0.5)))
    planes = w.K if st["rank"] > 0 else 0
    counts = stage_counts(N, n, rho, planes, 2 * w.radius + 1, w.kmeans_iters, Ns, fwdbwd,
                          conv_tensor=precision == "bf16" and w.radius <= 16 and n <= 3,
                          nlm_r=w.patch_radius, box=w.spatial == "box")
    sm = {k: v for k, v in zip(STAGES, stages[:6 if fwdbwd else 4]) if v is not None}
    line = {"workload": w.name, "mode": "fwd+bwd" if fwdbwd else "fwd", "precision": precision,
            "value": N / 1e6 / (ms / 1e3), "unit": "megapixels/s", "ms_per_step": ms,
            "stages_ms": sm, "status": st["status"], "rank_r": st["rank"],
            "roofline_step": step_roofline(counts, sm, ms)}
    blocks, errs = golden_landmarks(golden)
    line["kmeans_qerr_rel"] = abs(st["qerr"] - errs[0]) / errs[0]
    line["accuracy"] = accuracy_blf(nyf, w, blocks[0], precision, fwdbwd)
    return line


def batched_extra(nyf, steps, warmup, flush, stream, precision="bf16", tiles=None):
    """The 64-image workload (K = 16): forward + backward by CUDA-graph replay.  tiles:
    None (the library's choice per radius) or "tuned" (the autotuner's variant per
    radius and image-size class, tuned before the timed region)."""
    import torch
    from paper_1901_06112_gb300 import synth
    batch = synth.batched_blf()
    shapes = [(w.H, w.W) for w in batch]
    P = nyf.Params(K=16, kmeans_iters=10, precision=precision)
    bt = nyf.Batched(shapes, [w.sigma_s for w in batch], [w.sigma_r for w in batch], P)
    f = bt.pack([w.f for w in batch])
    if tiles == "tuned":                           # before the timed region
        bt.tune_tiles(f)
    G = torch.randn(f.shape, generator=torch.Generator().manual_seed(0)).cuda()
    bt.capture(f, G)
    for _ in range(warmup):
        bt.replay()
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bt.replay()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    mpix = bt.total / 3 / 1e6
    t = float(np.mean(ms))
    # Sec. 8(d) step roofline: the stages' algorithmic work summed over the images
    tot = {}
    for w in batch:
        c = stage_counts(w.H * w.W, 3, 3, 16, 2 * w.radius + 1, 10, w.H * w.W, True,
                         conv_tensor=precision == "bf16" and w.radius <= 16)
        for k, v in c.items():
            tot[k] = tuple(a + b for a, b in zip(tot.get(k, (0.0,) * 4), v))
    roof = step_roofline(tot, {}, t)
    line = {"workload": f"batched_blf_64_images_128-1024_K16_{precision}", "images": len(batch),
            "tiles": ("tuned in the batch (Batched.tune_tiles): " + ", ".join(
                f"{t} {bt.tiles.count(t)}" for t in sorted(set(bt.tiles))))
            if tiles == "tuned" else "library default",
            "megapixels": mpix, "ms_per_step": t, "value": mpix / (t / 1e3),
            "unit": "megapixels/s", "mode": "fwd+bwd, one CUDA-graph replay per step",
            "roofline_step": roof}
    # accuracy: the same batched call with the oracle's landmarks, checked images against
    # the FP64 oracle on sampled pixels
    try:
        from oracle import kernels as Kr
        from oracle import nystrom as ny
        blocks, _ = golden_landmarks("batched")
        lm = torch.from_numpy(np.stack(blocks).astype(np.float32)).cuda()
        outs = bt.unpack(bt.forward(f, landmarks=lm))
        worst, worst_max, used, total = 0.0, 0.0, 0, 0
        for b in (0, 7, 23, 41, 63):
            w = batch[b]
            idx = synth.sample_indices(w.H * w.W, 64, b)
            ys, xs = idx // w.W, idx % w.W
            taps = Kr.gaussian_taps(w.sigma_s, w.radius)
            want, eta = ny.nystrom_filter_at(w.f, w.f, blocks[b].astype(np.float64),
                                             float(np.float32(w.sigma_r)), taps, 1e-7, ys, xs,
                                             return_eta=True)
            ok = eta > 1e-3 * taps.sum() ** 2      # eta_hat (Eq. (15)) away from zero
            r, m = _rel(outs[b].cpu().numpy()[ys[ok], xs[ok]], want[ok])
            worst, worst_max = max(worst, r), max(worst_max, m)
            used, total = used + int(ok.sum()), total + len(ok)
        line["accuracy"] = {"vs": "FP64 oracle with the oracle's landmarks, images 0, 7, 23, 41, "
                                  "63, 64 pixels each (worst image), at the pixels where the "
                                  "oracle's eta_hat is at least 1e-3 of the window mass",
                            "rel_rmse": worst, "max_abs": worst_max,
                            "pixels_conditioned": f"{used} of {total}"}
    except Exception as ex:      # the accuracy pass must not hide the measurement
        line["accuracy"] = {"error": str(ex)[:200]}
    return line


def iir_extra(nyf, lib, f_dev, wl, steps, flush, stream):
    """The same workload with the recursive Gaussian (Young & van Vliet, Sec. IV) as
    omega: forward only, FP32; the two passes are HBM-bound."""
    H, W, n = wl.f.shape
    P = nyf.Params(sigma_s=wl.sigma_s, sigma_r=wl.sigma_r, K=wl.K, kmeans_iters=wl.kmeans_iters,
                   seed=wl.seed, spatial="gaussian_iir")
    ws = nyf.make_workspace(H, W, n, n, P)
    out = f_dev.new_empty(f_dev.shape)

    def step():
        nyf.blf(f_dev, P, out=out, ws=ws)
    lib.nyf_set_timing(1)
    for _ in range(3):
        step()
    ms, stages = timed_steps(step, steps, flush, stream, lib)
    lib.nyf_set_timing(0)
    st = nyf.stats(ws)
    planes = wl.K if st["rank"] > 0 else 0
    gb = iir_bytes_per_pixel(planes, n) * H * W / 1e9
    gb_design = iir_design_bytes_per_pixel(planes, n) * H * W / 1e9
    pk, how = hbm_peak()
    a = gb / (stages[3] / 1e3)
    return {"workload": wl.name + "_recursive_gaussian", "value": H * W / 1e6 / (ms / 1e3),
            "ms_per_step": ms, "unit": "megapixels/s", "mode": "fwd", "precision": "fp32",
            "status": st["status"], "conv_ms": stages[3],
            "roofline": {"kernel": "k_cols + k_rows (both passes)", "bound": "hbm",
                         "achieved": a, "peak": pk, "unit": "GB/s", "frac": a / pk,
                         "traffic": NCU_TRAFFIC[("recursive_pair", "fp32")]
                         if (H, W, planes) == (1080, 1920, 32) else None,
                         "algorithmic_GB": gb, "design_GB": gb_design,
                         "design_frac": gb_design / (stages[3] / 1e3) / pk,
                         "peak_basis": f"copy bandwidth ({how}); algorithmic bytes = f, phi "
                                       "read, g_hat, eta written; design bytes add the "
                                       "K (n+1)-plane intermediate"}}


def pca_nlm_extra(nyf, steps, flush, stream):
    """PCA-NLM at the paper's parameters (Sec. IV): 768 x 512 colour, 7x7x3 patches projected
    on 25 principal directions, K = 31, 21 x 21 box; the whole call (patch PCA, projection,
    k-means, eig, features, convolutions) per step."""
    import torch
    from paper_1901_06112_gb300 import synth
    w = synth.colour_pca_nlm()
    f = torch.from_numpy(w.f).cuda()
    P = nyf.Params(sigma_r=w.sigma_r, K=w.K, spatial="box", S=w.S, patch_radius=w.patch_radius,
                   sample_frac=w.sample_frac, seed=w.seed)
    ws = nyf.make_pca_workspace(w.H, w.W, 3, w.pca_dim, P)
    out = torch.empty_like(f)
    for _ in range(3):
        nyf.pca_nlm(f, w.pca_dim, P, out=out, ws=ws)
    torch.cuda.synchronize()

    def t(fn):
        ms = []
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return float(np.mean(ms))
    ms = t(lambda: nyf.pca_nlm(f, w.pca_dim, P, out=out, ws=ws))
    st = nyf.stats(ws)
    pca_ms = t(lambda: nyf.patch_pca(f, w.patch_radius, w.pca_dim))
    return {"workload": w.name, "value": w.H * w.W / 1e6 / (ms / 1e3), "ms_per_step": ms,
            "unit": "megapixels/s", "mode": "fwd", "patch_pca_ms": pca_ms, "status": st["status"],
            "rank": st["rank"]}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1901_06112_gb300 import _lib, build as _build
    _build.build()
    from paper_1901_06112_gb300 import nyf, synth

    lib = _lib.load()
    wl = {"colour_hd": synth.colour_blf_hd, "colour_256": synth.colour_blf_small,
          "hyperspectral": synth.hyperspectral_blf, "nlm": synth.colour_nlm}[args.workload]()
    if args.crop:
        ch, cw = min(args.crop[0], wl.f.shape[0]), min(args.crop[1], wl.f.shape[1])
        wl = dataclasses.replace(wl, name=f"{wl.name}_crop_{cw}x{ch}",
                                 f=np.ascontiguousarray(wl.f[:ch, :cw]))
        args.no_extras = True
    H, W, n = wl.f.shape
    nlm = wl.patch_radius > 0
    rho = n * (2 * wl.patch_radius + 1) ** 2 if nlm else n
    fwdbwd = args.mode == "fwdbwd" and not nlm
    iir = args.spatial == "gaussian_iir"
    if iir and (fwdbwd or args.precision != "fp32"):
        raise SystemExit("--spatial gaussian_iir runs the forward in fp32: add --mode fwd")

    def make(precision, bwd=False):
        return nyf.Params(sigma_s=wl.sigma_s, sigma_r=wl.sigma_r, K=wl.K,
                          kmeans_iters=wl.kmeans_iters, seed=replica_seed(wl.seed, rank),
                          precision=precision, save_for_backward=bwd,
                          spatial=args.spatial if not nlm else wl.spatial, S=wl.S,
                          patch_radius=wl.patch_radius, sample_frac=wl.sample_frac)

    P = make(args.precision, fwdbwd)
    f_dev = torch.from_numpy(wl.f).to(dev)
    out = torch.empty_like(f_dev)
    ws = nyf.make_workspace(H, W, n, rho, P, dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    G = torch.randn(f_dev.shape, generator=torch.Generator().manual_seed(0)).to(dev)
    grads = nyf.BackwardBuffers(f_dev)
    stream = torch.cuda.current_stream()

    def make_step(Pp, bwd):
        def step():
            if nlm:
                nyf.nlm(f_dev, Pp, out=out, ws=ws)
            else:
                nyf.blf(f_dev, Pp, out=out, ws=ws)
            if bwd:
                nyf.blf_backward(f_dev, Pp, out, G, ws, grads)
        return step

    step = make_step(P, fwdbwd)
    lib.nyf_set_timing(1)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    st = nyf.stats(ws)
    if st["status"] != 0:
        raise RuntimeError(f"device status {st['status']} after warm-up")

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    launches0 = lib.nyf_launch_count()
    ms, stage_mean = timed_steps(step, args.steps, flush, stream, lib)
    torch.cuda.synchronize()
    launches = lib.nyf_launch_count() - launches0
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    mp = H * W / 1e6
    ms_max, value = weak_scaling_value(ms, mp, world, dev, dist)

    r = st["rank"]
    planes = wl.K if r > 0 else 0
    peak = SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    fwd_flops = conv_flops_per_pixel(planes, n, P.radius) * H * W
    bwd_flops = conv_bwd_flops_per_pixel(planes, n, P.radius) * H * W

    captured = (H, W, wl.K) == (1080, 1920, 32)

    def roof(name, flops, ms_k):
        a = flops / (ms_k / 1e3) / 1e12
        tensor = args.precision == "bf16" and name == "conv_combine"   # the tcgen05 kernel
        if tensor:
            pk, how = bf16_tensor_peak()
            basis = f"dense BF16 tensor peak, burst ({how}); FLOPs = the FIR's algorithmic count"
        else:
            pk, basis = peak, "152 SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz (FP32 ALU)"
        return {"kernel": name, "bound": "tensor" if tensor else "alu", "achieved": a, "peak": pk,
                "unit": "TFLOP/s", "frac": a / pk,
                "traffic": NCU_TRAFFIC.get((name, args.precision)) if captured else None,
                "launch_ms": ms_k, "peak_basis": basis}

    roof_fwd = roof("conv_combine", fwd_flops, stage_mean[3])
    if iir:
        gb = iir_bytes_per_pixel(planes, n) * H * W / 1e9
        pk_h, how_h = hbm_peak()
        a_h = gb / (stage_mean[3] / 1e3)
        roof_fwd = {"kernel": "k_cols + k_rows (both recursive passes)", "bound": "hbm",
                    "achieved": a_h, "peak": pk_h, "unit": "GB/s", "frac": a_h / pk_h,
                    "traffic": NCU_TRAFFIC[("recursive_pair", "fp32")] if captured else None,
                    "launch_ms": stage_mean[3], "algorithmic_GB": gb,
                    "peak_basis": f"copy bandwidth ({how_h})"}
    if wl.spatial == "box" and not iir:   # running sums: the stage is bound by its HBM bytes
        gb = (4.0 * n + 4.0 * planes + 4.0 * n + 4.0) * H * W / 1e9
        pk_h, how_h = hbm_peak()
        a_h = gb / (stage_mean[3] / 1e3)
        roof_fwd = {"kernel": "conv_combine (box window, running sums)", "bound": "hbm",
                    "achieved": a_h, "peak": pk_h, "unit": "GB/s", "frac": a_h / pk_h,
                    "traffic": None, "launch_ms": stage_mean[3], "algorithmic_GB": gb,
                    "peak_basis": f"copy bandwidth ({how_h}); f and phi read, g_hat and eta written"}
    roof_bwd = roof("conv_bwd", bwd_flops, stage_mean[4]) if fwdbwd else None
    dominant = roof_bwd if (fwdbwd and stage_mean[4] > stage_mean[3]) else roof_fwd
    # Sec. 8(d) step roofline of the headline step
    counts = stage_counts(H * W, n, rho, planes, 2 * P.radius + 1, wl.kmeans_iters,
                          max(1, int(np.floor(wl.sample_frac * H * W + 0.5))), fwdbwd,
                          conv_tensor=args.precision == "bf16" and P.radius <= 16 and n <= 3,
                          nlm_r=wl.patch_radius, box=wl.spatial == "box")
    step_roof = step_roofline(counts, {k: v for k, v in zip(STAGES, stage_mean[:6 if fwdbwd else 4])
                                       if v is not None}, ms)
    accuracy = None
    if rank == 0 and not iir and not args.crop:
        try:
            blocks, errs = golden_landmarks(args.workload)
            accuracy = accuracy_blf(nyf, wl, blocks[0], args.precision, fwdbwd)
            accuracy["kmeans_qerr_rel"] = abs(st["qerr"] - errs[0]) / errs[0]
        except Exception as ex:           # the accuracy pass must not hide the measurement
            accuracy = {"error": str(ex)[:300]}

    extras = {}
    if not args.no_extras and rank == 0 and args.workload == "colour_hd":
        lib.nyf_set_timing(0)
        if fwdbwd:                                # forward only: no planes kept
            fwd_ms, _ = timed_steps(make_step(make(args.precision), False), max(3, args.steps // 2),
                                    flush, stream, lib)
            extras["fwd"] = {"value": mp / (fwd_ms / 1e3), "ms_per_step": fwd_ms,
                             "unit": "megapixels/s", "precision": args.precision}
        if fwdbwd and not iir:                    # the low-memory backward (C_kq recomputed)
            Pr = make(args.precision, True)
            Pr.backward_mode = "recompute"
            wsr = nyf.make_workspace(H, W, n, n, Pr, dev)

            def step_r():
                nyf.blf(f_dev, Pr, out=out, ws=wsr)
                nyf.blf_backward(f_dev, Pr, out, G, wsr, grads)
            lib.nyf_set_timing(1)
            for _ in range(2):
                step_r()
            r_ms, r_st = timed_steps(step_r, max(3, args.steps // 2), flush, stream, lib)
            lib.nyf_set_timing(0)
            extras["recompute_backward"] = {
                "value": mp / (r_ms / 1e3), "ms_per_step": r_ms, "unit": "megapixels/s",
                "bwd_conv_ms": r_st[4], "workspace_GB": wsr.nbytes / 1e9,
                "workspace_GB_planes_kept": ws.nbytes / 1e9,
                "mode": "fwd+bwd, C_kq convolved again 4 modes at a time"}
            del wsr
        other = "bf16" if args.precision == "fp32" else "fp32"
        if iir:
            other = None
        if other:
            Po = make(other, fwdbwd)
            for _ in range(2):
                make_step(Po, fwdbwd)()
            o_ms, _ = timed_steps(make_step(Po, fwdbwd), max(3, args.steps // 2), flush, stream, lib)
            f_ms, _ = timed_steps(make_step(make(other), False), max(3, args.steps // 2), flush,
                                  stream, lib)
            extras[other] = {"fwdbwd_value" if fwdbwd else "value": mp / (o_ms / 1e3),
                             "fwd_value": mp / (f_ms / 1e3), "unit": "megapixels/s"}
        for prec, key, tiles in (("bf16", "batched", None), ("fp32", "batched_fp32", None),
                                 ("bf16", "batched_tuned", "tuned")):
            try:
                extras[key] = batched_extra(nyf, max(3, args.steps // 4), 3, flush, stream, prec,
                                            tiles)
            except Exception as ex:               # the side measurement must not hide the main one
                extras[key] = {"error": str(ex)[:300]}
        if not iir:
            try:
                extras["recursive_gaussian"] = iir_extra(nyf, lib, f_dev, wl,
                                                         max(3, args.steps // 2), flush, stream)
            except Exception as ex:
                extras["recursive_gaussian"] = {"error": str(ex)[:300]}
            try:
                extras["pca_nlm"] = pca_nlm_extra(nyf, max(3, args.steps // 4), flush, stream)
            except Exception as ex:
                extras["pca_nlm"] = {"error": str(ex)[:300]}
        # the other single-GPU workloads, each measured like the headline
        configs = {}
        for key, make_w, golden, bwd in (("colour_256", synth.colour_blf_small, "colour_256", True),
                                         ("hyperspectral", synth.hyperspectral_blf, "hyperspectral",
                                          True),
                                         ("nlm", synth.colour_nlm, "nlm", False)):
            try:
                configs[key] = config_line(nyf, lib, make_w(), golden, "fp32", bwd,
                                           max(3, args.steps // 2), flush, stream)
            except Exception as ex:
                configs[key] = {"error": str(ex)[:300]}
        extras["configs"] = configs

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        f_host = torch.from_numpy(wl.f).pin_memory()
        o_host = torch.empty_like(f_host).pin_memory()
        lib.nyf_set_timing(0)
        e2e_ms = []
        for i in range(args.warmup + args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            f_dev.copy_(f_host, non_blocking=True)
            step()
            o_host.copy_(out, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            if i >= args.warmup:
                e2e_ms.append(e0.elapsed_time(e1))
        t2 = torch.tensor([float(np.mean(e2e_ms))], device=dev)
        if world > 1:
            dist.all_reduce(t2, op=dist.ReduceOp.MAX)
        nb = wl.f.nbytes
        e2e = {"value": world * mp / (float(t2.item()) / 1e3), "unit": "megapixels/s",
               "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "megapixels/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "bf16",
            "data": "synthetic",
            "config": {"workload": wl.name, "H": H, "W": W, "n": n, "sigma_s": wl.sigma_s,
                       "sigma_r": wl.sigma_r, "K": wl.K, "kmeans_iters": wl.kmeans_iters,
                       "precision": args.precision, "spatial": args.spatial,
                       "mode": "fwd+bwd" if fwdbwd else "fwd", "rank_r": r,
                       "l2": "flushed between steps (512 MB write)",
                       "parallelism": f"replicas x{world}"},
            "stages_ms": dict(zip(STAGES, stage_mean[:6 if fwdbwd else 4])),
            "accuracy": accuracy,
            "roofline": dominant,
            "roofline_step": step_roof,
            "roofline_conv_fwd": roof_fwd,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk,
            "extras": extras,
        }
        if not args.no_cpu_baseline and world == 1 and args.workload == "colour_hd" and not args.crop:
            try:
                line["cpu_baseline"] = cpu_baseline_obj(backward=fwdbwd)
            except Exception as ex:  # the oracle leg must not hide the GPU number
                line["cpu_baseline"] = {"error": str(ex)[:200]}
            try:
                line["cpu_baseline_fp32"] = cpu_fp32_baseline(wl)
            except Exception as ex:
                line["cpu_baseline_fp32"] = {"error": str(ex)[:200]}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
