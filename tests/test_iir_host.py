"""Host-side parameters of the recursive Gaussian (NYF_GAUSSIAN_IIR), no GPU:
the FP32 difference-form coefficients, the lane-scan matrices T^(LS 2^d) and
the zero-padding boundary map Rm that libnyf computes in FP64 on the host.

The segmented scheme the kernels run (each of 32 lanes filters LS values of the
line padded with zeros to 32 LS from a zero state; the incoming states follow
from a prefix scan of the lanes' end states with T^(LS 2^d); the anticausal pass
starts at the padded end from Rm applied to the causal end state and repeats
with a suffix scan) is evaluated here in FP64 with exactly those parameters and
compared with the FP64 recursive oracle on the zero-padded line."""
import ctypes as C

import numpy as np
import pytest

from oracle import iir
from paper_1901_06112_gb300 import _lib, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def _params(lib, sigma, length):
    out = (C.c_float * 60)()
    assert lib.nyf_iir_line_params(sigma, length, out, 60) == 0
    a = np.array(out[:], np.float64)
    return dict(B=a[0], nB=a[1], g1=a[2], ne2=a[3], LS=int(a[4]), len=int(a[5]),
                P=[a[6 + 9 * d:15 + 9 * d].reshape(3, 3) for d in range(5)], Rm=a[51:60].reshape(3, 3))


def _segmented(x, p):
    """The lanes' scheme in FP64 on the line padded to 32 LS (state (w, d1, d2))."""
    LS = p["LS"]
    v = np.zeros(32 * LS)
    v[:len(x)] = x
    v = v.reshape(32, LS).copy()
    B, nB, g1, ne2 = p["B"], p["nB"], p["g1"], p["ne2"]

    def run(seg, w1, w2, d1, d2, free, reverse):
        out = seg.copy()
        idx = range(LS - 1, -1, -1) if reverse else range(LS)
        for j in idx:
            pre = (nB * w2 + ne2 * d2) if free else (B * seg[j] + nB * w2 + ne2 * d2)
            dl = g1 * d1 + pre
            w = w1 + dl
            w2, w1, d2, d1 = w1, w, d1, dl
            out[j] = (seg[j] + w) if free else w
        return out, np.array([w1, d1, d2]), (w1, w2, d1, d2)

    E = np.zeros((32, 3))
    for l in range(32):
        v[l], E[l], _ = run(v[l], 0.0, 0.0, 0.0, 0.0, False, False)
    Pfx = E.copy()
    for d in range(5):
        off = 1 << d
        Pfx = np.array([Pfx[l] + (p["P"][d] @ Pfx[l - off] if l >= off else 0) for l in range(32)])
    Hin = np.vstack([np.zeros(3), Pfx[:-1]])
    for l in range(32):
        h0, h1, h2 = Hin[l]
        v[l], _, st = run(v[l], h0, h0 - h1, h1, h2, True, False)
        if l == 31:
            end = E[l] + np.array([st[0], st[2], st[3]])
    r = p["Rm"] @ end
    A = np.zeros((32, 3))
    for l in range(32):
        v[l], A[l], _ = run(v[l], 0.0, 0.0, 0.0, 0.0, False, True)
    G = A.copy()
    G[31] += p["P"][0] @ r
    for d in range(5):
        off = 1 << d
        G = np.array([G[l] + (p["P"][d] @ G[l + off] if l + off < 32 else 0) for l in range(32)])
    Kin = np.vstack([G[1:], r])
    for l in range(32):
        k0, k1, k2 = Kin[l]
        v[l], _, _ = run(v[l], k0, k0 - k1, k1, k2, True, True)
    return v.reshape(-1)[:len(x)]


@pytest.mark.parametrize("sigma,length", [(0.5, 1), (1.3, 37), (2.5, 96), (3.0, 1080), (5.0, 1920),
                                          (8.0, 700), (20.0, 45), (20.0, 2016)])
def test_segmented_scheme_with_host_parameters_equals_the_oracle(lib, sigma, length):
    p = _params(lib, sigma, length)
    LS = p["LS"]
    assert LS % 4 == 3 and 32 * LS >= length and (LS == 3 or 32 * (LS - 4) < length)
    x = np.random.default_rng(length).uniform(0, 255, size=length)
    got = _segmented(x, p)
    want = iir.iir_1d(x, sigma)
    rel = np.sqrt(np.mean((got - want) ** 2) / np.mean(want ** 2))
    # the only difference is the FP32 rounding of the parameters (6e-8); on lines
    # shorter than the filter's support the result comes mostly from the
    # boundary map, whose difference-state entries grow about like sigma
    assert rel < 2e-6 * max(1.0, sigma / 5.0), rel


def test_host_parameters_reject_bad_input(lib):
    out = (C.c_float * 60)()
    assert lib.nyf_iir_line_params(0.4, 10, out, 60) == 1
    assert lib.nyf_iir_line_params(3.0, 0, out, 60) == 1
    assert lib.nyf_iir_line_params(3.0, 10, out, 59) == 1
    assert lib.nyf_iir_line_params(3.0, 2017, out, 60) == 2
