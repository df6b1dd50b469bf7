"""nyf_features_static: the entry point for callers that cannot allocate device
memory (no device allocator of their own, a host that owns all device memory,
or a loop where cudaMalloc would synchronise the device).  Its scratch is a
fixed array inside the library.  Checked through the C ABI against
nyf_features (which takes a caller workspace) and against the FP64 oracle's
features, on calls in a row, since calls share that array and must not depend
on what the previous call left.  Also: its device status output reports a
latched rank-0 failure, and it rejects the same arguments as nyf_features."""
import ctypes as C

import numpy as np
import pytest

from _util import report

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1901_06112_gb300 import _lib, build
    build.build()
    return _lib.load()


def _run(lib, X, mu, sr, tau, prec=0, ws=None, outputs=True):
    """One call of nyf_features_static (ws None) or nyf_features; returns
    (code, phi K x N float64, rank, alphas, status)."""
    N, rho = X.shape
    K = mu.shape[0]
    dt = torch.bfloat16 if prec == 1 else torch.float32
    phi = torch.full((K, N), 7.0, dtype=dt, device="cuda")
    rank = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    alphas = torch.zeros(K, dtype=torch.float64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = [C.c_void_p(X.data_ptr()), N, rho, C.c_void_p(mu.data_ptr()), K, sr, tau, prec,
         C.c_void_p(phi.data_ptr()),
         C.c_void_p(rank.data_ptr()) if outputs else None,
         C.c_void_p(alphas.data_ptr()) if outputs else None]
    if ws is None:
        code = lib.nyf_features_static(*p, C.c_void_p(status.data_ptr()), st)
    else:
        code = lib.nyf_features(*p, C.c_void_p(ws.ptr), ws.nbytes, st)
    torch.cuda.synchronize()
    return (code, phi.double().cpu().numpy(), int(rank.cpu()), alphas.cpu().numpy(),
            int(status.cpu()))


def _cases():
    from paper_1901_06112_gb300 import synth
    hyper = synth.hyperspectral(40, 36, 31, 6, 10.0, 0.02, 5).reshape(-1, 31)
    return [(synth.voronoi_colour(64, 48, 30, 10.0, 1).reshape(-1, 3), 16, 40.0, 0),
            (synth.voronoi_colour(33, 71, 12, 5.0, 2).reshape(-1, 3), 5, 25.0, 0),
            (hyper, 64, 0.15, 0),            # the documented limit K = 64, rho = 31 guide
            (hyper, 64, 0.15, 1)]            # same, features stored in bfloat16


def test_static_scratch_matches_workspace_entry_point_and_oracle(lib):
    from oracle import nystrom as ny
    from oracle import pipeline as pl
    from paper_1901_06112_gb300 import nyf
    for X_np, K, sr, prec in _cases():   # calls in a row share the scratch
        mu_np, _ = pl.landmarks(X_np.astype(np.float64), K, 4, 3)
        mu_np = mu_np.astype(np.float32)
        X = torch.from_numpy(np.ascontiguousarray(X_np)).cuda()
        mu = torch.from_numpy(mu_np).cuda()
        rho = X.shape[1]
        ws = nyf.make_workspace(X.shape[0], 1, rho, rho,
                                nyf.Params(K=K, precision="bf16" if prec else "fp32"))
        want = _run(lib, X, mu, sr, 1e-7, prec, ws=ws)
        got = _run(lib, X, mu, sr, 1e-7, prec)
        assert got[0] == 0 and want[0] == 0
        assert got[4] == 0                   # no device-side error latched
        assert got[2] == want[2] > 0
        assert np.allclose(got[3], want[3], rtol=0, atol=1e-12 * want[3][0])
        rel = np.linalg.norm(got[1] - want[1]) / np.linalg.norm(want[1])
        assert rel < 1e-5
        sr32 = float(np.float32(sr))
        phi_o, _, _ = ny.features_symmetric(X_np.astype(np.float64), mu_np.astype(np.float64),
                                            sr32, 1e-7)
        r, _ = report(f"static features K={K} rho={rho} prec={prec}", got[1].T, phi_o)
        # bfloat16 storage rounds each feature by at most 2^-8 of its value, which
        # bounds the relative RMSE of the stored planes too
        assert r < (2.0 ** -8 if prec else 1e-5)


def test_static_scratch_without_rank_and_alphas(lib):
    from paper_1901_06112_gb300 import synth
    X_np = synth.voronoi_colour(24, 40, 9, 8.0, 3).reshape(-1, 3)
    X = torch.from_numpy(np.ascontiguousarray(X_np)).cuda()
    mu = X[::97][:8].contiguous()
    full = _run(lib, X, mu, 30.0, 1e-7)
    bare = _run(lib, X, mu, 30.0, 1e-7, outputs=False)
    assert bare[0] == 0 and bare[4] == 0
    assert np.array_equal(bare[1], full[1])


def test_static_scratch_reports_rank_zero(lib):
    # tau > 1 keeps no mode: the device latches NYF_ERR_NUMERIC and phi is not
    # written; the status output is how a caller sees that.
    X = torch.rand((500, 3), device="cuda") * 255
    mu = X[:6].contiguous()
    code, phi, rank, _, status = _run(lib, X, mu, 30.0, 2.0)
    assert code == 0 and status == 4 and rank == 0
    assert np.all(phi == 7.0)               # untouched
    ok = _run(lib, X, mu, 30.0, 1e-7)       # the next call starts from a clear status
    assert ok[4] == 0 and ok[2] > 0


def test_static_scratch_rejects_what_nyf_features_rejects(lib):
    from paper_1901_06112_gb300 import nyf
    X = torch.rand((64, 3), device="cuda")
    mu = X[:4].contiguous()
    ws = nyf.make_workspace(64, 1, 3, 3, nyf.Params(K=4))
    for sr in (float("inf"), float("nan"), 0.0, -1.0):
        assert _run(lib, X, mu, sr, 1e-7)[0] == 1
        assert _run(lib, X, mu, sr, 1e-7, ws=ws)[0] == 1


def test_static_scratch_rejects_sizes_beyond_its_limit(lib):
    X = torch.zeros((16, 3), dtype=torch.float32, device="cuda")
    mu = torch.zeros((65, 3), dtype=torch.float32, device="cuda")
    out = torch.zeros((65, 16), dtype=torch.float32, device="cuda")
    code = lib.nyf_features_static(C.c_void_p(X.data_ptr()), 16, 3, C.c_void_p(mu.data_ptr()), 65,
                                   30.0, 1e-7, 0, C.c_void_p(out.data_ptr()), None, None, None,
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 2        # NYF_ERR_UNSUPPORTED
