"""Build step of libnyf.so: nvcc for sm_103a, one object per translation unit, in parallel."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libnyf.so")

SOURCES = ["api.cu", "kmeans.cu", "kmeans_tc.cu", "eig.cu", "features.cu", "features_tc.cu", "conv.cu", "conv_a.cu", "conv_b.cu",
           "conv_c.cu", "backward.cu", "backward_a.cu", "backward_b.cu", "backward_c.cu",
           "noalloc.cu", "conv_tc.cu", "umma_selftest.cu", "iir.cu", "iir_cols_a.cu",
           "iir_cols_b.cu", "iir_rows_a.cu", "iir_rows_b.cu", "pca.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", INCLUDE]


def nvcc_path() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    p = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(p):
        return p
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libnyf")


def _deps():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))] + \
        [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]


def _stale(target, sources):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def build(verbose: bool = False, extra_flags=None, jobs: int | None = None) -> str:
    """Compile every kernel source for sm_103a and link libnyf.so next to this file."""
    nvcc = nvcc_path()
    os.makedirs(BUILD, exist_ok=True)
    deps = _deps()
    extra = list(extra_flags or [])
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]

    def compile_one(src):
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        if not _stale(o, [s] + deps) and not extra:
            return o, ""
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", s, "-o", o]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return o, r.stderr

    jobs = jobs or max(1, min(len(srcs), os.cpu_count() or 4))
    with cf.ThreadPoolExecutor(jobs) as ex:
        results = list(ex.map(compile_one, srcs))
    objs = [o for o, _ in results]
    if verbose:
        for o, log in results:
            if log:
                print(log)
    if _stale(LIB, objs):
        cmd = [nvcc, *ARCH, "-shared", "-o", LIB, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link of libnyf.so failed:\n{r.stderr}")
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
