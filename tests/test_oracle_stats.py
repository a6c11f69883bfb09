"""Pins for the oracle's global statistics (Sections 4.1-4.3 and the
appendix's Torben median): closed forms on ramps and permutations, the
library's histogram and order statistics on random data, NULL (NaN) voxels
left out."""
import numpy as np
import pytest


def test_moments_of_a_ramp_with_null_rows(oracle_lib):
    """v = x on every row: mean (nx-1)/2, population sd sqrt((nx^2-1)/12),
    min 0, max nx-1; NaN rows drop out of every figure."""
    nz, ny, nx = 4, 5, 13
    cube = np.broadcast_to(np.arange(nx, dtype=np.float32), (nz, ny, nx)).copy()
    cube[1, 2, :] = np.nan
    cube[3, 0, :] = np.nan
    m = oracle_lib.moments(cube)
    assert m["count"] == nz * ny * nx - 2 * nx
    assert m["mean"] == pytest.approx((nx - 1) / 2, abs=1e-12)
    assert m["sd"] == pytest.approx(np.sqrt((nx * nx - 1) / 12.0), abs=1e-12)
    assert (m["min"], m["max"]) == (0.0, nx - 1.0)


def test_moments_of_sixteen_bit_storage_use_the_stored_values(oracle_lib):
    """bfloat16 bits of 1.0 and 3.0 in equal numbers: mean 2, sd 1."""
    bits = np.where(np.arange(64).reshape(4, 4, 4) % 2 == 0, 0x3F80, 0x4040).astype(np.uint16)
    m = oracle_lib.moments(bits, bits="bf16")
    assert (m["count"], m["mean"], m["sd"], m["min"], m["max"]) == (64, 2.0, 1.0, 1.0, 3.0)


def test_histogram_of_a_ramp_and_its_top_edge(oracle_lib):
    """Integer ramp 0..nx-1 over [0, nx) in nx bins: each value its own bin,
    ny*nz counts each; over [0, nx-1] in one bin the top value is included."""
    nz, ny, nx = 3, 4, 9
    cube = np.broadcast_to(np.arange(nx, dtype=np.float32), (nz, ny, nx)).copy()
    assert (oracle_lib.histogram(cube, 0.0, float(nx), nx) == ny * nz).all()
    assert oracle_lib.histogram(cube, 0.0, float(nx - 1), 1)[0] == nx * ny * nz
    h = oracle_lib.histogram(cube, 2.0, 5.0, 3)              # bins hold 2 | 3 | 4 and the top edge 5
    assert h.tolist() == [ny * nz, ny * nz, 2 * ny * nz]


def test_histogram_matches_numpy_and_skips_nan(oracle_lib):
    rng = np.random.default_rng(5)
    cube = rng.standard_normal((9, 8, 7)).astype(np.float32)
    cube[0, 0, :3] = np.nan
    for lo, hi, nb in ((-3.0, 3.0, 12), (-1.0, 0.5, 7), (float(np.nanmin(cube)), float(np.nanmax(cube)), 64)):
        finite = cube[np.isfinite(cube)].astype(np.float64)
        want = np.histogram(finite, nb, (lo, hi))[0]
        assert np.array_equal(oracle_lib.histogram(cube, lo, hi, nb), want.astype(np.uint64))


def test_median_of_a_permutation(oracle_lib):
    """A permutation of 0..n-1: the rank (n+1)//2 value is (n+1)//2 - 1, for
    odd and even n (the lower median)."""
    rng = np.random.default_rng(6)
    for shape in ((5, 5, 5), (4, 5, 6), (2, 2, 3)):
        n = int(np.prod(shape))
        cube = rng.permutation(n).astype(np.float32).reshape(shape)
        med, passes = oracle_lib.median(cube)
        assert med == (n + 1) // 2 - 1
        assert passes >= 1


def test_median_matches_order_statistic_with_ties_and_nan(oracle_lib):
    rng = np.random.default_rng(7)
    for shape in ((11, 9, 7), (6, 6, 6)):
        cube = np.round(rng.standard_normal(shape) * 3).astype(np.float32)     # many equal values
        cube.ravel()[::17] = np.nan
        finite = np.sort(cube[np.isfinite(cube)].astype(np.float64))
        k = (finite.size + 1) // 2
        assert oracle_lib.median(cube)[0] == finite[k - 1]
        cube2 = rng.standard_normal(shape).astype(np.float32)
        f2 = np.sort(cube2.ravel().astype(np.float64))
        assert oracle_lib.median(cube2)[0] == f2[(f2.size + 1) // 2 - 1]


def test_median_degenerate_cubes(oracle_lib):
    assert oracle_lib.median(np.full((3, 3, 3), 2.5, np.float32))[0] == 2.5
    one = np.full((2, 2, 2), np.nan, np.float32)
    one[1, 0, 1] = -4.0
    assert oracle_lib.median(one)[0] == -4.0
    with pytest.raises(ValueError):
        oracle_lib.median(np.full((2, 2, 2), np.nan, np.float32))
