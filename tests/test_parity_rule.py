"""The GPU-vs-oracle pixel rule (oracle.parity) on hand-made images: a count
difference is excused only on a reported tie, and the error is taken over the
remaining pixels."""
import numpy as np
import pytest

from oracle.parity import MARGIN_ERT, MARGIN_N, ParityError, compare_pixels


def _ref(H=4, W=5):
    rng = np.random.default_rng(0)
    return {"rgba": rng.uniform(size=(H, W, 4)), "n_used": np.full((H, W), 7, np.int32),
            "margin_n": np.full((H, W), 0.3), "margin_ert": np.full((H, W), np.inf)}


def test_equal_images_pass():
    ref = _ref()
    r = compare_pixels(ref["rgba"] + 1e-6, ref["n_used"], ref, 1e-4)
    assert r["passed"] and r["pixels"] == 20 and r["excluded_ties"] == 0
    assert abs(r["max_abs"] - 1e-6) < 1e-12


def test_count_difference_off_a_tie_fails():
    ref = _ref()
    ns = ref["n_used"].copy()
    ns[1, 2] += 1
    with pytest.raises(ParityError, match="off a decision tie"):
        compare_pixels(ref["rgba"], ns, ref, 1e-4)
    r = compare_pixels(ref["rgba"], ns, ref, 1e-4, raise_on_fail=False)
    assert not r["passed"] and r["off_tie"] == 1


@pytest.mark.parametrize("which", ["n", "ert"])
def test_count_difference_on_a_tie_is_excluded(which):
    ref = _ref()
    ns = ref["n_used"].copy()
    ns[1, 2] += 1
    img = ref["rgba"].copy()
    img[1, 2] += 0.5                          # that pixel's colour is not compared
    if which == "n":
        ref["margin_n"][1, 2] = 0.5 * MARGIN_N
    else:
        ref["margin_ert"][1, 2] = 0.5 * MARGIN_ERT
    r = compare_pixels(img, ns, ref, 1e-4)
    assert r["passed"] and r["excluded_ties"] == 1 and r["pixels"] == 19 and r["max_abs"] == 0.0


def test_margin_just_above_the_tie_threshold_is_not_a_tie():
    ref = _ref()
    ns = ref["n_used"].copy()
    ns[0, 0] -= 1
    ref["margin_n"][0, 0] = 2 * MARGIN_N
    ref["margin_ert"][0, 0] = 2 * MARGIN_ERT
    with pytest.raises(ParityError):
        compare_pixels(ref["rgba"], ns, ref, 1e-4)


def test_error_above_tolerance_fails_and_rows_select():
    ref = _ref()
    img = ref["rgba"].copy()
    img[3, 4, 2] += 2e-4
    with pytest.raises(ParityError, match="max abs pixel error"):
        compare_pixels(img, ref["n_used"], ref, 1e-4)
    r = compare_pixels(img, ref["n_used"], ref, 1e-4, rows=[0, 1, 2])
    assert r["passed"] and r["pixels"] == 15


def test_too_many_ties_fail():
    ref = _ref(40, 50)
    ns = ref["n_used"].copy()
    ns[:2, :2] += 1                            # 4 tie pixels of 2000 (> max(2, 0.1%))
    ref["margin_n"][:2, :2] = 0.0
    with pytest.raises(ParityError, match="too many tie pixels"):
        compare_pixels(ref["rgba"], ns, ref, 1e-4)
