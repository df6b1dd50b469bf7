"""Build and load the FP32 C++/OpenMP CPU baseline (oracle/cpu_baseline.cpp).

Test and benchmark infrastructure: bench.py's CPU-baseline leg times it on the
host's cores and tests/test_cpu_baseline.py checks it against the FP64 oracle.
g++ only (no CUDA); plain -O3, no machine-specific flags, so the same source
builds on x86-64 and on Arm.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpu_baseline.cpp")
LIB = os.path.join(HERE, "_build", "libnyf_cpu.so")


def build() -> str:
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cmd = ["g++", "-O3", "-fopenmp", "-std=c++17", "-shared", "-fPIC", "-o", LIB, SRC]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"g++ failed on cpu_baseline.cpp:\n{r.stderr}")
    return LIB


def load():
    lib = C.CDLL(build())
    lib.nyf_cpu_blf.restype = C.c_int
    lib.nyf_cpu_blf.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_float, C.c_float,
                                C.c_int, C.c_int, C.c_uint64, C.c_double, C.c_void_p, C.c_void_p,
                                C.c_int]
    lib.nyf_cpu_threads.restype = C.c_int
    return lib


def blf(lib, f, sigma_s, sigma_r, K, iters=10, seed=0, tau=1e-7, landmarks=None, threads=0):
    """The FP32 CPU filter of f (H x W x n float32); returns (g_hat, status)."""
    import numpy as np
    f = np.ascontiguousarray(f, np.float32)
    out = np.empty_like(f)
    lm = None if landmarks is None else np.ascontiguousarray(landmarks, np.float32)
    H, W, n = f.shape
    code = lib.nyf_cpu_blf(f.ctypes.data, H, W, n, float(sigma_s), float(sigma_r), int(K),
                           int(iters), int(seed) & ((1 << 64) - 1), float(tau),
                           None if lm is None else lm.ctypes.data, out.ctypes.data, int(threads))
    return out, code
