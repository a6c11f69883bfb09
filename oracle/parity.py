"""The comparison rule between a GPU render and the FP64 oracle.

TEST INFRASTRUCTURE, like the rest of this package: used by ``tests/`` and by
the pixel-error leg of ``bench.py``; it holds no arithmetic of the method.

Rule.  A pixel's composited-sample count must equal the oracle's, except
where the oracle reports that count as decided by a rounding tie: the sample
count (``margin_n``: (t_out - t_in)/step + 1/2 within MARGIN_N of an integer,
the constant-step rule of Section 4.4) or the early-termination stop
(``margin_ert``: the running opacity of a composited sample within
MARGIN_ERT of the threshold, front-to-back composition of Section 3.4).  FP32
and FP64 may decide such a tie differently and both are right.  Tie pixels
are excluded from the error and counted; they may be at most
max(2, 0.1%) of the pixels compared.  Any count mismatch off a tie fails.
The maximum absolute error over the remaining pixels and all four channels
must be within the caller's tolerance.
"""
from __future__ import annotations

import numpy as np

MARGIN_N = 1e-3       # sample-count decisions closer than this (in steps) may differ in FP32
MARGIN_ERT = 1e-4     # early-termination decisions closer than this (in opacity) may differ


class ParityError(AssertionError):
    pass


def compare_pixels(gpu_rgba, gpu_ns, ref, tol, rows=None, raise_on_fail=True):
    """Element-wise comparison of a GPU image (H, W, 4) and its per-pixel
    sample counts (H, W) with the oracle's ``render`` result ``ref``, over
    ``rows`` (all rows if None).

    Returns dict(max_abs, mean_abs, pixels, excluded_ties, off_tie, passed).
    With raise_on_fail, a failed rule raises ParityError instead."""
    g = np.asarray(gpu_rgba, dtype=np.float64)
    ns = np.asarray(gpu_ns).astype(np.int64)
    r = np.asarray(ref["rgba"])
    rn = np.asarray(ref["n_used"]).astype(np.int64)
    mn, me = np.asarray(ref["margin_n"]), np.asarray(ref["margin_ert"])
    if rows is not None:
        rows = list(rows)
        g, ns, r, rn, mn, me = g[rows], ns[rows], r[rows], rn[rows], mn[rows], me[rows]
    diff = ns != rn
    tie = (mn < MARGIN_N) | (me < MARGIN_ERT)
    off_tie = diff & ~tie
    keep = ~diff
    err = np.abs(g - r)[keep]
    out = {"max_abs": float(err.max()) if err.size else 0.0,
           "mean_abs": float(err.mean()) if err.size else 0.0,
           "pixels": int(keep.sum()), "excluded_ties": int((diff & tie).sum()), "off_tie": int(off_tie.sum())}
    problems = []
    if off_tie.any():
        problems.append("sample counts differ off a decision tie at %s (gpu %s, oracle %s)" % (
            np.argwhere(off_tie)[:5].tolist(), ns[off_tie][:5].tolist(), rn[off_tie][:5].tolist()))
    if diff.sum() > max(2, 0.001 * diff.size):
        problems.append("too many tie pixels: %d of %d" % (int(diff.sum()), diff.size))
    if out["max_abs"] > tol:
        problems.append("max abs pixel error %.3g > %.3g" % (out["max_abs"], tol))
    out["passed"] = not problems
    if problems and raise_on_fail:
        raise ParityError("; ".join(problems))
    if problems:
        out["problems"] = problems
    return out
