"""ctypes binding of libnyf.so (include/nyf.h): argument marshalling only.

The library is built in-tree by ``paper_1901_06112_gb300.build``; loading fails
loudly when it is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnyf.so")

NYF_OK = 0
STATUS_NAMES = {0: "NYF_OK", 1: "NYF_ERR_INVALID_ARG", 2: "NYF_ERR_UNSUPPORTED",
                3: "NYF_ERR_WORKSPACE", 4: "NYF_ERR_NUMERIC", 5: "NYF_ERR_CUDA",
                6: "NYF_ERR_TIMEOUT"}
FP32, BF16 = 0, 1
GAUSSIAN, BOX, GAUSSIAN_IIR = 0, 1, 2
TILE_AUTO, TILE_WIDE, TILE_NARROW, TILE_TENSOR = 0, 1, 2, 3
SAVE_NONE, SAVE_PLANES, SAVE_RECOMPUTE = 0, 1, 2
RECOMPUTE_MODES = 4
MAX_K, MAX_RHO, MAX_S, MAX_CHANNELS = 64, 160, 32, 64


class NyfParams(C.Structure):
    _fields_ = [("sigma_s", C.c_float), ("sigma_r", C.c_float), ("K", C.c_int),
                ("kmeans_iters", C.c_int), ("seed", C.c_uint64), ("eig_rel_tol", C.c_double),
                ("precision", C.c_int), ("spatial", C.c_int), ("S", C.c_int),
                ("patch_radius", C.c_int), ("sample_frac", C.c_float), ("conv_tile", C.c_int),
                ("save_for_backward", C.c_int)]


class NyfStats(C.Structure):
    _fields_ = [("status", C.c_int), ("rank", C.c_int), ("qerr", C.c_double),
                ("alpha_max", C.c_double), ("alpha_min_kept", C.c_double),
                ("eta_small", C.c_longlong), ("grad_sigma_r", C.c_float),
                ("grad_sigma_s", C.c_float)]


class NyfBatchItem(C.Structure):
    _fields_ = [("offset", C.c_int64), ("H", C.c_int), ("W", C.c_int), ("sigma_s", C.c_float),
                ("sigma_r", C.c_float), ("conv_tile", C.c_int), ("reserved", C.c_int)]


_P = C.c_void_p
_SIGNATURES = {
    "nyf_version": (C.c_int, []),
    "nyf_status_string": (C.c_char_p, [C.c_int]),
    "nyf_workspace_size": (C.c_size_t, [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(NyfParams)]),
    "nyf_kmeans": (C.c_int, [_P, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_uint64, _P, _P, _P, _P,
                             _P, C.c_size_t, _P]),
    "nyf_features": (C.c_int, [_P, C.c_int64, C.c_int, _P, C.c_int, C.c_float, C.c_double, C.c_int,
                               _P, _P, _P, _P, C.c_size_t, _P]),
    "nyf_filter_blf": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(NyfParams),
                                 _P, _P, _P, C.c_size_t, _P]),
    "nyf_filter_nlm": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.POINTER(NyfParams), _P, _P, _P,
                                 C.c_size_t, _P]),
    "nyf_filter_blf_backward": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_int,
                                          C.POINTER(NyfParams), _P, _P, _P, _P, _P, _P,
                                          C.c_size_t, _P]),
    "nyf_get_stats": (C.c_int, [_P, C.POINTER(NyfStats), _P]),
    "nyf_set_timing": (None, [C.c_int]),
    "nyf_get_timing": (C.c_int, [C.POINTER(C.c_float), C.c_int]),
    "nyf_launch_count": (C.c_longlong, []),
    "nyf_features_static": (C.c_int, [_P, C.c_int64, C.c_int, _P, C.c_int, C.c_float, C.c_double,
                                      C.c_int, _P, _P, _P, _P, _P]),
    "nyf_selftest_umma": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P]),
    "nyf_selftest_wait_timeout": (C.c_int, [C.c_int, _P, _P]),
}
OPTIONAL = {}
_SIGNATURES.update({
    "nyf_batched_workspace_size": (C.c_size_t, [_P, C.c_int, C.c_int, C.POINTER(NyfParams)]),
    "nyf_filter_blf_batched": (C.c_int, [_P, _P, C.c_int, C.c_int, C.POINTER(NyfParams), _P, _P,
                                         _P, C.c_size_t, _P]),
    "nyf_filter_blf_batched_backward": (C.c_int, [_P, _P, C.c_int, C.c_int, C.POINTER(NyfParams),
                                                  _P, _P, _P, _P, _P, C.c_size_t, _P]),
    "nyf_batched_stats": (C.c_int, [_P, _P, C.c_int, C.c_int, C.POINTER(NyfParams), C.c_int,
                                    C.POINTER(NyfStats), _P]),
    "nyf_iir_line_params": (C.c_int, [C.c_double, C.c_int, C.POINTER(C.c_float), C.c_int]),
    "nyf_draw_indices": (C.c_int, [C.c_uint64, C.c_int64, C.c_int, C.POINTER(C.c_int64)]),
    "nyf_gather_rows": (C.c_int, [_P, C.c_int64, C.c_int, C.c_int64, _P, C.c_int, _P, _P]),
    "nyf_kmeans_partials": (C.c_int, [_P, C.c_int64, C.c_int, C.c_int, _P, _P, _P, _P, C.c_size_t,
                                      _P]),
    "nyf_kmeans_apply_sums": (C.c_int, [_P, C.c_int, C.c_int, _P, _P]),
    "nyf_patch_pca_workspace_size": (C.c_size_t, [C.c_int, C.c_int]),
    "nyf_patch_pca": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P, _P, _P,
                                C.c_size_t, _P]),
    "nyf_pca_project": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P, _P, _P]),
    "nyf_pca_nlm_workspace_size": (C.c_size_t, [C.c_int, C.c_int, C.c_int, C.c_int,
                                                C.POINTER(NyfParams)]),
    "nyf_filter_pca_nlm": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(NyfParams),
                                     _P, _P, _P, _P, _P, C.c_size_t, _P]),
})

_lib = None


def declared_symbols(header=None):
    """Names of the functions include/nyf.h declares."""
    import re
    header = header or os.path.join(os.path.dirname(_HERE), "include", "nyf.h")
    text = open(header).read()
    return sorted(set(re.findall(r"^\s*(?:[\w\*]+\s+)+\**(nyf_\w+)\s*\(", text, re.M)))


def load():
    """Load libnyf.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_1901_06112_gb300.build.build() "
                           "(the CUDA path has no fallback)")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    for name, (res, args) in OPTIONAL.items():
        if hasattr(lib, name):
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
    _lib = lib
    return lib


class NyfError(RuntimeError):
    def __init__(self, code, where):
        lib = load()
        msg = lib.nyf_status_string(code).decode()
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)} ({msg})")
        self.code = code


def check(code, where):
    if code != NYF_OK:
        raise NyfError(code, where)
