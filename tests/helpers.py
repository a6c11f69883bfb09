"""Shared helpers for the GPU parity tests (comparison rules against the
FP64 oracle)."""
import numpy as np
import pytest

TOL_F32 = 1e-4       # max abs pixel error, float32 storage
TOL_HALF = 2e-3      # max abs pixel error against the FP64 oracle on the float32 cube
MARGIN_N = 1e-3      # sample-count decisions closer than this (in steps) may differ in FP32
MARGIN_ERT = 1e-4    # early-termination decisions closer than this (in opacity) may differ


def cuda_or_skip():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def compare(gpu_rgba, gpu_ns, ref, tol, rows=None):
    """Element-wise comparison with the oracle.

    Pixels whose composited-sample count differs from the oracle's must sit
    on a decision tie (sample count or early termination within the margins
    above); they are checked to be few and are excluded from the error.
    Returns (max_err, mean_err, n_excluded)."""
    g = np.asarray(gpu_rgba, dtype=np.float64)
    ns = np.asarray(gpu_ns).astype(np.int64)
    r = ref["rgba"]
    rn = ref["n_used"].astype(np.int64)
    if rows is not None:
        g, ns, r, rn = g[rows], ns[rows], r[rows], rn[rows]
        mn, me = ref["margin_n"][rows], ref["margin_ert"][rows]
    else:
        mn, me = ref["margin_n"], ref["margin_ert"]
    diff = ns != rn
    tie = (mn < MARGIN_N) | (me < MARGIN_ERT)
    bad = diff & ~tie
    assert not bad.any(), "sample counts differ off a decision tie at %s (gpu %s, oracle %s)" % (
        np.argwhere(bad)[:5].tolist(), ns[bad][:5].tolist(), rn[bad][:5].tolist())
    assert diff.sum() <= max(2, 0.001 * diff.size), "too many tie pixels: %d" % diff.sum()
    keep = ~diff
    err = np.abs(g - r)[keep]
    mx = float(err.max()) if err.size else 0.0
    mean = float(err.mean()) if err.size else 0.0
    assert mx <= tol, "max abs pixel error %.3g > %.3g" % (mx, tol)
    return mx, mean, int(diff.sum())
