"""Shared helpers for the GPU parity tests (comparison rules against the
FP64 oracle).  The pixel rule itself lives in ``oracle.parity`` so that the
benchmark's pixel-error leg applies the same one."""
import pytest

from oracle.parity import MARGIN_ERT, MARGIN_N, compare_pixels  # noqa: F401

TOL_F32 = 1e-4       # max abs pixel error, float32 storage
TOL_HALF = 2e-3      # max abs pixel error against the FP64 oracle on the float32 cube


def cuda_or_skip():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def compare(gpu_rgba, gpu_ns, ref, tol, rows=None):
    """Element-wise comparison with the oracle (``oracle.parity`` rule):
    pixels whose composited-sample count differs from the oracle's must sit
    on a decision tie, be few, and are excluded from the error; any other
    count difference or an error above tol fails.
    Returns (max_err, mean_err, n_excluded)."""
    r = compare_pixels(gpu_rgba, gpu_ns, ref, tol, rows=rows)
    return r["max_abs"], r["mean_abs"], r["excluded_ties"]
