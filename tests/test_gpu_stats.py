"""GPU global statistics (Sections 4.1-4.3) against the FP64 oracle through
the C ABI: moments, histogram and median over ragged cubes and every brick
size (each voxel must be counted once although the bricks repeat their
apron), 16-bit storage, NULL (NaN) voxels, ties and degenerate cubes."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import cuda_or_skip

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


@pytest.fixture(scope="module")
def P(torch):
    import paper_1211_4896_gb300 as P
    return P


SHAPES = [((37, 29, 41), 16), ((17, 33, 65), 16), ((50, 20, 34), 32), ((66, 65, 64), 64), ((2, 2, 3), 16)]


def _stored(torch, cube, store):
    t = torch.from_numpy(np.ascontiguousarray(cube)).cuda()
    if store == "f16":
        return t, t.half().float().cpu().numpy()
    if store == "bf16":
        return t, t.bfloat16().float().cpu().numpy()
    return t, cube


@pytest.mark.parametrize("store", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("dims,brick", SHAPES)
def test_moments_histogram_median(P, torch, dims, brick, store):
    rng = np.random.default_rng(sum(dims) + brick)
    cube = (2.0 + 3.0 * rng.standard_normal(dims[::-1])).astype(np.float32)
    cube.ravel()[::29] = np.nan
    cube.ravel()[5::31] = 1.25                           # ties
    t, ref_cube = _stored(torch, cube, store)
    vol = P.Volume(t, store, brick=brick)
    try:
        m = P.moments(vol)
        r = oracle.moments(ref_cube)
        assert m["count"] == r["count"]
        assert m["mean"] == pytest.approx(r["mean"], rel=1e-6, abs=1e-6)
        assert m["sd"] == pytest.approx(r["sd"], rel=1e-6)
        assert (m["min"], m["max"]) == (r["min"], r["max"])
        for lo, hi, nb in ((r["min"], r["max"], 256), (-1.0, 5.0, 7), (0.0, 2.5, 16384)):
            h = P.histogram(vol, lo, hi, nb).cpu().numpy()
            assert np.array_equal(h, oracle.histogram(ref_cube, lo, hi, nb).astype(np.int64))
        assert P.median(vol) == oracle.median(ref_cube)[0]
    finally:
        vol.close()


def test_histogram_bin_edges_exactly(P, torch):
    """Values on bin edges (a ramp of multiples of the bin width, and values
    far from 0 with narrow bins, where the FP32 estimate is not used) land in
    the bins the FP64 definition gives."""
    ramp = np.broadcast_to(np.arange(64, dtype=np.float32) * 0.125, (4, 3, 64)).copy()
    far = (1000.0 + np.arange(64, dtype=np.float32) * np.float32(2 ** -10)).astype(np.float32)
    far = np.broadcast_to(far, (4, 3, 64)).copy()
    for cube, lo, hi, nb in ((ramp, 0.0, 8.0, 64), (ramp, 0.0, 7.875, 63), (far, 1000.0, 1000.0625, 64)):
        vol = P.Volume(torch.from_numpy(cube).cuda(), "f32")
        try:
            h = P.histogram(vol, lo, hi, nb).cpu().numpy()
            assert np.array_equal(h, oracle.histogram(cube, lo, hi, nb).astype(np.int64))
        finally:
            vol.close()


def test_median_of_permutation_and_degenerate_cubes(P, torch):
    rng = np.random.default_rng(3)
    for shape in ((5, 7, 9), (4, 6, 10)):                 # odd and even counts
        n = int(np.prod(shape))
        cube = rng.permutation(n).astype(np.float32).reshape(shape) - 7.0
        vol = P.Volume(torch.from_numpy(cube).cuda(), "f32")
        try:
            assert P.median(vol) == (n + 1) // 2 - 1 - 7.0
        finally:
            vol.close()
    neg = -np.abs(rng.standard_normal((6, 6, 6))).astype(np.float32)       # all negative keys
    for cube in (np.full((3, 4, 5), -2.5, np.float32), neg):
        vol = P.Volume(torch.from_numpy(cube).cuda(), "f32")
        try:
            assert P.median(vol) == oracle.median(cube)[0]
        finally:
            vol.close()
    empty = np.full((3, 3, 3), np.nan, np.float32)
    vol = P.Volume(torch.from_numpy(empty).cuda(), "f32")
    try:
        assert np.isnan(P.median(vol))
        m = P.moments(vol)
        assert m["count"] == 0 and np.isnan(m["mean"])
        assert P.histogram(vol, 0.0, 1.0, 4).sum().item() == 0
    finally:
        vol.close()


def test_stats_on_the_hi_cube(P, torch):
    """A 256^3 HI-like cube: the figures the bench reports, against the oracle."""
    cube = synth.hi_cube((256, 256, 256), 160, 16, 5)
    vol = P.Volume(cube.cuda(), "f32")
    c = cube.numpy()
    try:
        m, r = P.moments(vol), oracle.moments(c)
        assert m["count"] == r["count"] and m["sd"] == pytest.approx(r["sd"], rel=1e-6)
        h = P.histogram(vol, r["min"], r["max"], 1024).cpu().numpy()
        assert np.array_equal(h, oracle.histogram(c, r["min"], r["max"], 1024).astype(np.int64))
        assert P.median(vol) == oracle.median(c)[0]
    finally:
        vol.close()
