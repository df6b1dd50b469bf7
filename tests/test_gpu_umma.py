"""The fifth-generation tensor-core path (tcgen05.mma with the accumulator in
tensor memory, K-major shared-memory operands) against the same product on the
host: the operands are small integers over powers of two, exact in bfloat16, so
the only difference is FP32 accumulation order."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1901_06112_gb300 import build
    build.build()
    from paper_1901_06112_gb300 import _lib
    return _lib.load()


def operands(N, K):
    m = np.arange(128)[:, None]
    n = np.arange(N)[:, None]
    k = np.arange(K)[None, :]
    A = (((3 * m + 5 * k) % 17) - 8) / 8.0
    B = (((7 * n + 3 * k) % 13) - 6) / 4.0
    return A, B


@pytest.mark.parametrize("a_in_tmem", [0, 1])
@pytest.mark.parametrize("N,K", [(16, 16), (64, 32), (96, 160 // 2), (128, 128), (256, 64)])
def test_tcgen05_gemm(lib, N, K, a_in_tmem):
    D = torch.full((128, N), float("nan"), dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = lib.nyf_selftest_umma(C.c_void_p(D.data_ptr()), N, K, a_in_tmem, C.c_void_p(status.data_ptr()),
                               C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    A, B = operands(N, K)
    want = A @ B.T
    got = D.cpu().numpy().astype(np.float64)
    err = np.abs(got - want).max()
    print(f"[parity] tcgen05 128x{N}x{K} (A in {'TMEM' if a_in_tmem else 'smem'}): max abs err {err:.2e}")
    assert err <= 1e-5 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("limit", [1, 64])
def test_bounded_wait_gives_up_and_reports_timeout(lib, limit):
    # an mbarrier phase nothing completes: the wait must give up after `limit`
    # polls and latch NYF_ERR_TIMEOUT (6); the context stays usable afterwards
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert lib.nyf_selftest_wait_timeout(limit, C.c_void_p(status.data_ptr()), stream) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 6
    D = torch.zeros((128, 64), dtype=torch.float32, device="cuda")
    assert lib.nyf_selftest_umma(C.c_void_p(D.data_ptr()), 64, 32, 0, C.c_void_p(status.data_ptr()),
                                 stream) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    A, B = operands(64, 32)
    assert np.abs(D.cpu().numpy() - A @ B.T).max() <= 1e-5 * np.abs(A @ B.T).max()


def test_bounded_wait_rejects_bad_limits(lib):
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert lib.nyf_selftest_wait_timeout(0, C.c_void_p(status.data_ptr()), None) == 1
    assert lib.nyf_selftest_wait_timeout(5000, C.c_void_p(status.data_ptr()), None) == 1
