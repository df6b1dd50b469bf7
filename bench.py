#!/usr/bin/env python3
"""Throughput of the Nystrom bilateral filter on GB300 (megapixels/s).

Workload (default): the 1920 x 1080 x 3 colour bilateral filter -- 400
Voronoi cells with sinusoidal shading and noise 15, sigma_s 5 (31 x 31
window), sigma_r 40, K 32 k-means landmarks (10 Lloyd iterations).  One step
is one pass of the whole path on one image: subsample/k-means, FP64
eigendecomposition, features, convolutions + combine (and the backward pass
when --mode fwdbwd).  Inputs are resident in HBM; L2 is flushed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|bf16]
                       [--mode fwd|fwdbwd] [--impl nyf|reference]
For N > 1 the script runs under torchrun: every rank filters its own image
(independent replicas, no collective on the data path) and rank 0 prints the
JSON line.
"""
from __future__ import annotations

import argparse
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
    ap.add_argument("--mode", default="fwd", choices=["fwd", "fwdbwd"])
    ap.add_argument("--impl", default="nyf", choices=["nyf", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


# ----------------------------------------------------------------------------- CPU oracle leg

CPU_SAMPLE = (384, 384)     # crop of the workload the oracle filters per step


def _oracle_step_code(h, w):
    return f"""
import os, sys, time, json
sys.path.insert(0, {ROOT!r})
import numpy as np
from paper_1901_06112_gb300 import synth
from oracle import pipeline as pl
wl = synth.colour_blf_hd()
f = wl.f[:{h}, :{w}].astype(np.float64)
t0 = time.perf_counter()
g, mu, info = pl.blf(f, wl.sigma_s, wl.sigma_r, wl.K, iters=wl.kmeans_iters, seed=wl.seed)
dt = time.perf_counter() - t0
print(json.dumps({{"seconds": dt, "pixels": {h * w}}}))
"""


def cpu_oracle_seconds(h=CPU_SAMPLE[0], w=CPU_SAMPLE[1]):
    """Time the FP64 oracle (k-means + Algorithm 1) on an h x w crop, one thread."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", _oracle_step_code(h, w)], capture_output=True,
                       text=True, env=env, timeout=900)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["seconds"], d["pixels"]


def cpu_baseline_obj():
    sec, px = cpu_oracle_seconds()
    return {"value": px / 1e6 / sec, "unit": "megapixels/s", "cores": 1, "kind": "oracle",
            "sample": f"FP64 oracle (k-means 10 iters + Algorithm 1) on a {CPU_SAMPLE[0]}x"
                      f"{CPU_SAMPLE[1]} crop of the workload, one thread, {sec:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps = max(1, args.steps)
    times = []
    px = 0
    for _ in range(max(0, min(args.warmup, 1))):
        cpu_oracle_seconds(128, 128)
    # each step is a bounded sample of the workload (a 256 x 256 crop)
    for _ in range(min(steps, 3)):
        sec, px = cpu_oracle_seconds(256, 256)
        times.append(sec)
    sec = float(np.median(times))
    v = px / 1e6 / sec
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "megapixels/s",
            "n_gpus": args.gpus, "steps": len(times), "warmup": args.warmup,
            "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "colour_blf_1920x1080_K32 (256x256 crop per step)",
                       "sigma_s": 5.0, "sigma_r": 40.0, "K": 32, "mode": "fwd"},
            "cpu_baseline": {"value": v, "unit": "megapixels/s", "cores": 1, "kind": "oracle",
                             "sample": "256x256 crop of the 1920x1080 workload per step"},
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
    """Algorithmic FLOPs of the convolution + combine stage per pixel.

    K (n + 1) planes, each a separable FIR of 2 passes x (2S + 1) taps x 2 FLOP,
    plus the combine multiply-add of every plane.
    """
    return K * (n + 1) * (2 * (2 * S + 1) * 2 + 2)


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
    wl = synth.colour_blf_hd()
    H, W, n = wl.f.shape
    P = nyf.Params(sigma_s=wl.sigma_s, sigma_r=wl.sigma_r, K=wl.K, kmeans_iters=wl.kmeans_iters,
                   seed=wl.seed + rank, precision=args.precision)
    f_dev = torch.from_numpy(wl.f).to(dev)
    out = torch.empty_like(f_dev)
    ws = nyf.make_workspace(H, W, n, n, P, dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    fwdbwd = args.mode == "fwdbwd"
    if fwdbwd:
        G = torch.randn_like(f_dev)
        grads = nyf.BackwardBuffers(f_dev)

    def step():
        nyf.blf(f_dev, P, out=out, ws=ws)
        if fwdbwd:
            nyf.blf_backward(f_dev, P, out, G, ws, grads)

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
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    launches0 = lib.nyf_launch_count()
    step_ms, stage_ms = [], []
    import ctypes as C
    buf = (C.c_float * 7)()
    for _ in range(args.steps):
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
    torch.cuda.synchronize()
    launches = lib.nyf_launch_count() - launches0
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    ms = float(np.mean(step_ms))
    t = torch.tensor([ms], device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    mp = H * W / 1e6
    value = world * mp / (ms_max / 1e3)

    stage = np.array(stage_ms)
    stage_mean = [float(np.mean(stage[:, i][stage[:, i] >= 0])) if np.any(stage[:, i] >= 0) else None
                  for i in range(7)]
    r = st["rank"]
    flops = conv_flops_per_pixel(r, n, P.radius) * H * W
    conv_ms = stage_mean[3]
    peak = SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    achieved = flops / (conv_ms / 1e3) / 1e12

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
            nyf.blf(f_dev, P, out=out, ws=ws)
            if fwdbwd:
                nyf.blf_backward(f_dev, P, out, G, ws, grads)
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
            "dtype": "f32" if args.precision == "fp32" else "bf16+f32",
            "data": "synthetic",
            "config": {"workload": wl.name, "H": H, "W": W, "n": n, "sigma_s": wl.sigma_s,
                       "sigma_r": wl.sigma_r, "K": wl.K, "kmeans_iters": wl.kmeans_iters,
                       "precision": args.precision, "mode": args.mode, "rank_r": r,
                       "l2": "flushed between steps (512 MB write)",
                       "parallelism": f"replicas x{world}"},
            "stages_ms": {"landmarks": stage_mean[0], "eig": stage_mean[1],
                          "features": stage_mean[2], "conv_combine": stage_mean[3],
                          "bwd_conv": stage_mean[4], "bwd_features": stage_mean[5],
                          "bwd_tail": stage_mean[6]},
            "roofline": {"kernel": "conv_combine", "bound": "alu", "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": None,
                         "peak_basis": "152 SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz"},
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk,
        }
        if not args.no_cpu_baseline and world >= 1 and rank == 0 and world == 1:
            try:
                line["cpu_baseline"] = cpu_baseline_obj()
            except Exception as ex:  # the oracle leg must not hide the GPU number
                line["cpu_baseline"] = {"error": str(ex)[:200]}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
