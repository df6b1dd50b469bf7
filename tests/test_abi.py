"""The C-ABI library builds, loads and exports every symbol include/nyf.h declares (no GPU calls)."""
import ctypes as C
import os

import pytest

from paper_1901_06112_gb300 import _lib, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _lib.declared_symbols()
    assert {"nyf_kmeans", "nyf_features", "nyf_filter_blf", "nyf_filter_nlm",
            "nyf_filter_blf_backward", "nyf_workspace_size", "nyf_get_stats"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings_and_version(lib):
    assert lib.nyf_version() >= 100
    for code in range(7):
        assert lib.nyf_status_string(code)


def test_workspace_size_host_logic(lib):
    p = _lib.NyfParams(3.0, 30.0, 8, 10, 0, 1e-7, 0, 0, 0, 0, 1.0, 0)
    s1 = lib.nyf_workspace_size(256, 256, 3, 3, C.byref(p))
    s2 = lib.nyf_workspace_size(512, 256, 3, 3, C.byref(p))
    assert s1 > 0 and s2 > s1
    p.precision = 1                 # the filters keep their features in float32 either way
    assert lib.nyf_workspace_size(256, 256, 3, 3, C.byref(p)) == s1
    p.K = 0
    assert lib.nyf_workspace_size(256, 256, 3, 3, C.byref(p)) == 0
    p.K = 8
    p.save_for_backward = 1   # the forward keeps K (n + 1) convolved planes for the backward
    sb = lib.nyf_workspace_size(256, 256, 3, 3, C.byref(p))
    assert sb >= s1 + 4 * 8 * 4 * 256 * 256
    p.save_for_backward = 0
    p.patch_radius = 2        # NLM: rho is derived from n and r
    assert lib.nyf_workspace_size(64, 64, 3, 1, C.byref(p)) > 0


def test_argument_errors_return_before_any_launch(lib):
    p = _lib.NyfParams(3.0, 30.0, 8, 10, 0, 1e-7, 0, 0, 0, 0, 1.0, 0)
    bad = C.c_void_p(256)
    # null image
    assert lib.nyf_filter_blf(None, None, 8, 8, 3, 3, C.byref(p), None, bad, bad, 1 << 20, None) == 1
    # negative sigma_r
    q = _lib.NyfParams(3.0, -1.0, 8, 10, 0, 1e-7, 0, 0, 0, 0, 1.0, 0)
    assert lib.nyf_filter_blf(bad, None, 8, 8, 3, 3, C.byref(q), None, bad, bad, 1 << 20, None) == 1
    # too many landmarks
    q = _lib.NyfParams(3.0, 30.0, 65, 10, 0, 1e-7, 0, 0, 0, 0, 1.0, 0)
    assert lib.nyf_filter_blf(bad, None, 8, 8, 3, 3, C.byref(q), None, bad, bad, 1 << 20, None) == 1
    # window radius beyond the compiled maximum
    q = _lib.NyfParams(11.0, 30.0, 8, 10, 0, 1e-7, 0, 0, 0, 0, 1.0, 0)
    assert lib.nyf_filter_blf(bad, None, 8, 8, 3, 3, C.byref(q), None, bad, bad, 1 << 20, None) == 2
    # workspace too small / misaligned
    assert lib.nyf_filter_blf(bad, None, 8, 8, 3, 3, C.byref(p), None, bad, bad, 16, None) == 3
    assert lib.nyf_filter_blf(bad, None, 8, 8, 3, 3, C.byref(p), None, bad, C.c_void_p(260),
                              1 << 30, None) == 3
    # guide dimension must equal n when the guide is the image
    assert lib.nyf_filter_blf(bad, None, 8, 8, 3, 2, C.byref(p), None, bad, bad, 1 << 30, None) == 1
    # the backward needs a forward that kept its convolved planes
    assert lib.nyf_filter_blf_backward(bad, None, 8, 8, 3, 3, C.byref(p), bad, bad, bad, None, bad,
                                       bad, 1 << 30, None) == 1
    # k-means: more clusters than rows
    assert lib.nyf_kmeans(bad, 4, 3, 8, 1, 0, None, bad, None, None, bad, 1 << 20, None) == 1


def test_batched_workspace_is_the_sum_of_aligned_slices(lib):
    p = _lib.NyfParams(3.0, 30.0, 8, 10, 0, 1e-7, 0, 0, 0, 0, 1.0, 0)
    items = (_lib.NyfBatchItem * 3)(_lib.NyfBatchItem(0, 64, 80, 2.0, 30.0, 0, 0),
                                    _lib.NyfBatchItem(64 * 80 * 3, 1, 57, 1.0, 20.0, 0, 0),
                                    _lib.NyfBatchItem(64 * 80 * 3 + 57 * 3, 33, 7, 3.0, 50.0, 0, 0))
    total = lib.nyf_batched_workspace_size(items, 3, 3, C.byref(p))
    want = 0
    for it in items:
        q = _lib.NyfParams(it.sigma_s, it.sigma_r, 8, 10, 0, 1e-7, 0, 0, 0, 0, 1.0, 0)
        want = (want + lib.nyf_workspace_size(it.H, it.W, 3, 3, C.byref(q)) + 255) // 256 * 256
    assert total == want
    items[1].H = 0
    assert lib.nyf_batched_workspace_size(items, 3, 3, C.byref(p)) == 0


def test_recursive_gaussian_host_checks(lib):
    # spatial = NYF_GAUSSIAN_IIR (2): no window radius, a K (n + 1)-plane intermediate
    fir = _lib.NyfParams(3.0, 30.0, 8, 10, 0, 1e-7, 0, 0, 0, 0, 1.0, 0)
    iir = _lib.NyfParams(3.0, 30.0, 8, 10, 0, 1e-7, 0, 2, 0, 0, 1.0, 0)
    s_fir = lib.nyf_workspace_size(256, 200, 3, 3, C.byref(fir))
    s_iir = lib.nyf_workspace_size(256, 200, 3, 3, C.byref(iir))
    assert s_iir >= s_fir + 4 * 8 * 4 * 256 * 200
    bad = C.c_void_p(256)
    # sigma_s of 20 has no FIR window (S = 60 > NYF_MAX_S) but is fine recursively:
    # the call gets as far as the workspace check
    big = _lib.NyfParams(20.0, 30.0, 8, 10, 0, 1e-7, 0, 2, 0, 0, 1.0, 0)
    assert lib.nyf_filter_blf(bad, None, 8, 8, 3, 3, C.byref(big), None, bad, bad, 16, None) == 3
    big.spatial = 0
    assert lib.nyf_filter_blf(bad, None, 8, 8, 3, 3, C.byref(big), None, bad, bad, 16, None) == 2
    small = _lib.NyfParams(0.4, 30.0, 8, 10, 0, 1e-7, 0, 2, 0, 0, 1.0, 0)
    assert lib.nyf_filter_blf(bad, None, 8, 8, 3, 3, C.byref(small), None, bad, bad, 16, None) == 1
    bf16 = _lib.NyfParams(3.0, 30.0, 8, 10, 0, 1e-7, 1, 2, 0, 0, 1.0, 0)
    assert lib.nyf_filter_blf(bad, None, 8, 8, 3, 3, C.byref(bf16), None, bad, bad, 16, None) == 2
    saving = _lib.NyfParams(3.0, 30.0, 8, 10, 0, 1e-7, 0, 2, 0, 0, 1.0, 0)
    saving.save_for_backward = 1
    assert lib.nyf_filter_blf(bad, None, 8, 8, 3, 3, C.byref(saving), None, bad, bad, 16, None) == 2
    # lines longer than 32 lanes x 63 values are not implemented
    assert lib.nyf_filter_blf(bad, None, 2017, 8, 3, 3, C.byref(iir), None, bad, bad, 16, None) == 2
    assert lib.nyf_filter_blf(bad, None, 8, 2017, 3, 3, C.byref(iir), None, bad, bad, 16, None) == 2
    assert lib.nyf_filter_blf(bad, None, 2016, 2016, 3, 3, C.byref(iir), None, bad, bad, 16,
                              None) == 3


def test_pca_nlm_host_checks(lib):
    assert lib.nyf_patch_pca_workspace_size(3, 3) > 0          # 7x7x3 patches, rho 147
    assert lib.nyf_patch_pca_workspace_size(3, 4) == 0         # rho 243 > 160
    assert lib.nyf_patch_pca_workspace_size(3, 0) == 0
    p = _lib.NyfParams(3.0, 424.0, 31, 10, 0, 1e-7, 0, 1, 10, 3, 0.01, 0)
    s25 = lib.nyf_pca_nlm_workspace_size(512, 768, 3, 25, C.byref(p))
    p_blf = _lib.NyfParams(3.0, 424.0, 31, 10, 0, 1e-7, 0, 1, 10, 0, 0.01, 0)
    blf = lib.nyf_workspace_size(512, 768, 3, 25, C.byref(p_blf))
    assert s25 >= blf + 4 * 25 * 512 * 768                      # plus the 25-dim guide
    assert lib.nyf_pca_nlm_workspace_size(512, 768, 3, 33, C.byref(p)) == 0   # q > 32
    bad = C.c_void_p(256)
    # q out of range, mean without basis, saved planes (no PCA-NLM backward)
    assert lib.nyf_filter_pca_nlm(bad, 64, 64, 3, 0, C.byref(p), None, None, None, bad, bad, 16,
                                  None) == 1
    assert lib.nyf_filter_pca_nlm(bad, 64, 64, 3, 25, C.byref(p), bad, None, None, bad, bad, 16,
                                  None) == 1
    q = _lib.NyfParams(3.0, 424.0, 31, 10, 0, 1e-7, 0, 1, 10, 3, 0.01, 0)
    q.save_for_backward = 1
    assert lib.nyf_filter_pca_nlm(bad, 64, 64, 3, 25, C.byref(q), None, None, None, bad, bad, 16,
                                  None) == 1
    # a valid call gets as far as the workspace check
    assert lib.nyf_filter_pca_nlm(bad, 64, 64, 3, 25, C.byref(p), None, None, None, bad, bad, 16,
                                  None) == 3
    assert lib.nyf_patch_pca(bad, 64, 64, 3, 3, 26, bad, bad, bad, bad, 16, None) == 3
    assert lib.nyf_patch_pca(bad, 64, 64, 3, 3, 148, bad, bad, bad, bad, 16, None) == 1


def test_backward_workspace_holds_a_dphi_set_per_quantity_slice(lib):
    # n = 31 channels at S = 12: the 32 quantities form 8 slices of 4 per tile, so the
    # backward keeps 8 partial dL/dphi plane sets (summed in slice order) besides the
    # K (n + 1) convolved planes; n = 3 needs neither
    K, H, W = 8, 64, 64
    N = H * W
    p = _lib.NyfParams(4.0, 0.15, K, 10, 0, 1e-7, 0, 0, 0, 0, 1.0, 0)
    fwd = lib.nyf_workspace_size(H, W, 31, 31, C.byref(p))
    p.save_for_backward = 1
    bwd = lib.nyf_workspace_size(H, W, 31, 31, C.byref(p))
    assert bwd - fwd >= 4 * N * (K * 32 + 8 * K)
    p.save_for_backward = 0
    fwd3 = lib.nyf_workspace_size(H, W, 3, 3, C.byref(p))
    p.save_for_backward = 1
    bwd3 = lib.nyf_workspace_size(H, W, 3, 3, C.byref(p))
    assert bwd3 - fwd3 < 4 * N * (K * 4 + 2 * K) + 4 * N * 8 + (1 << 20)


def test_autotuner_size_classes():
    from paper_1901_06112_gb300 import tune
    assert [tune.size_class(H, W) for H, W in [(128, 128), (300, 400), (512, 512), (600, 650),
                                               (1024, 1024), (4000, 3000)]] == \
        [256, 256, 512, 512, 1024, 1024]
    assert tune.candidates(15, "fp32") == ["wide", "narrow"]
    assert tune.candidates(15, "bf16") == ["wide", "narrow", "tensor"]
    assert tune.candidates(21, "bf16") == ["wide"]
