"""Shared helpers of the parity tests (no method arithmetic here)."""
import numpy as np

FP32_REL_RMSE = 1e-4      # relative RMSE bar of the FP32 path against the FP64 oracle
BF16_REL_RMSE = 2e-3      # relative RMSE bar of the BF16 path against the FP64 oracle


def rel_rmse(got, want):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    return float(np.linalg.norm(got - want) / np.linalg.norm(want))


def max_abs(got, want):
    return float(np.max(np.abs(np.asarray(got, np.float64) - np.asarray(want, np.float64))))


def report(tag, got, want):
    r, m = rel_rmse(got, want), max_abs(got, want)
    print(f"[parity] {tag}: rel_rmse={r:.3e} max_abs={m:.3e}")
    return r, m


def sign_fix(W):
    """Flip each column so that its entry of largest magnitude (first on ties) is positive."""
    W = np.array(W, dtype=np.float64, copy=True)
    for k in range(W.shape[1]):
        i = int(np.argmax(np.abs(W[:, k])))
        if W[i, k] < 0:
            W[:, k] = -W[:, k]
    return W
