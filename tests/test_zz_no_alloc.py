"""nyf_features_static: the entry point for callers that cannot allocate device
memory (no device allocator of their own, a host that owns all device memory,
or a loop where cudaMalloc would synchronise the device).  Its scratch is a
fixed array inside the library.  Checked through the C ABI against
nyf_features (which takes a caller workspace), on two calls in a row, since
calls share that array and must not depend on what the previous call left."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1901_06112_gb300 import _lib, build
    build.build()
    return _lib.load()


def _run(lib, fn, X, mu, sr, tau, ws=None):
    N, rho = X.shape
    K = mu.shape[0]
    phi = torch.zeros((K, N), dtype=torch.float32, device="cuda")
    rank = torch.zeros(1, dtype=torch.int32, device="cuda")
    alphas = torch.zeros(K, dtype=torch.float64, device="cuda")
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = [C.c_void_p(X.data_ptr()), N, rho, C.c_void_p(mu.data_ptr()), K, sr, tau, 0,
         C.c_void_p(phi.data_ptr()), C.c_void_p(rank.data_ptr()), C.c_void_p(alphas.data_ptr())]
    if ws is None:
        code = lib.nyf_features_static(*p, st)
    else:
        code = lib.nyf_features(*p, C.c_void_p(ws.ptr), ws.nbytes, st)
    torch.cuda.synchronize()
    assert code == 0
    return phi.cpu().numpy(), int(rank.cpu()), alphas.cpu().numpy()


def test_static_scratch_matches_workspace_entry_point(lib):
    from paper_1901_06112_gb300 import nyf, synth
    cases = [(synth.voronoi_colour(64, 48, 30, 10.0, 1), 16, 40.0),
             (synth.voronoi_colour(33, 71, 12, 5.0, 2), 5, 25.0)]
    for f, K, sr in cases:          # two different calls in a row share the scratch
        X = torch.from_numpy(f.reshape(-1, 3).copy()).cuda()
        mu = X[torch.arange(0, X.shape[0], X.shape[0] // K)[:K]].contiguous()
        ws = nyf.make_workspace(X.shape[0], 1, 3, 3, nyf.Params(K=K))
        want = _run(lib, None, X, mu, sr, 1e-7, ws=ws)
        got = _run(lib, None, X, mu, sr, 1e-7)
        assert got[1] == want[1]
        assert np.allclose(got[2], want[2], rtol=0, atol=1e-12 * want[2][0])
        rel = np.linalg.norm(got[0] - want[0]) / np.linalg.norm(want[0])
        assert rel < 1e-5


def test_static_scratch_rejects_sizes_beyond_its_limit(lib):
    X = torch.zeros((16, 3), dtype=torch.float32, device="cuda")
    mu = torch.zeros((65, 3), dtype=torch.float32, device="cuda")
    out = torch.zeros((65, 16), dtype=torch.float32, device="cuda")
    code = lib.nyf_features_static(C.c_void_p(X.data_ptr()), 16, 3, C.c_void_p(mu.data_ptr()), 65,
                                   30.0, 1e-7, 0, C.c_void_p(out.data_ptr()), None, None,
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 2        # NYF_ERR_UNSUPPORTED
