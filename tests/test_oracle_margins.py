"""Pins for the oracle's two decision margins, which the GPU parity tests
use to tell a sample-count difference that sits on a rounding tie from one
that does not.

margin_n   = distance of (t_out - t_in)/step + 1/2 to the nearest integer
             (the sample-count rule of the constant step, Section 4.4: samples
             at t_in + (k + 1/2) step while <= t_out, so the count flips where
             that quantity crosses an integer);
margin_ert = smallest |opacity after sample k - threshold| over the samples
             the ray composited, up to and including the one that stopped it
             (early termination of the front-to-back composite, Section 3.4);
             +inf without early termination or without samples.

Each pin builds the tie by hand (a chord of known length, a constant opacity
whose running opacity is known in closed form) or measures it independently
of the oracle's clipping (a brute-force chord search), so that a margin that
is always zero, measured only at the stop sample, measured only before it, or
measured on the wrong quantity fails here.
"""
import numpy as np
import pytest

from test_oracle_pins import _chord_brute_force, cam_ortho, cam_persp


def _slab_z(nz, value=1.0):
    return np.full((nz, 4, 4), value, np.float32)


@pytest.mark.parametrize("k,delta", [(10, 0.3), (10, 0.7), (25, 0.01), (25, 0.99), (4, 1e-6), (7, 0.5)])
def test_margin_n_of_a_chord_of_known_length(oracle_lib, k, delta):
    """An orthographic ray along z through nz voxels has a chord of exactly
    nz - 1.  With step = L / (k + delta - 1/2), (L/step + 1/2) = k + delta, so
    the ray takes k samples and its count margin is min(delta, 1 - delta)."""
    nz = 8
    L = nz - 1.0
    step = L / (k + delta - 0.5)
    cam = cam_ortho((1.5, 1.5, -10.0), (0, 0, 1), (0, 1, 0), 2.0, 2, 2)
    tf = np.array([[1.0, 1.0, 1.0, 0.01]] * 2)
    r = oracle_lib.render(_slab_z(nz), cam, tf, 0.0, 2.0, step)
    want = min(delta, 1.0 - delta)
    assert (r["n_used"] == k).all(), r["n_used"]
    np.testing.assert_allclose(r["margin_n"], want, rtol=0, atol=1e-9)
    # no early termination: the opacity margin is undefined (+inf)
    assert np.isinf(r["margin_ert"]).all()


def test_margin_n_on_oblique_rays_against_brute_force_chords(oracle_lib):
    """Perspective rays at random angles: the margin equals the distance of
    (chord/step + 1/2) to the nearest integer with the chord measured by a
    brute-force membership search (not the oracle's slab clipping); a miss
    reports +inf."""
    rng = np.random.default_rng(11)
    dims = (9, 7, 11)
    cube = np.full(dims[::-1], 2.0, np.float32)
    tf = np.array([[1.0, 1.0, 1.0, 0.02]] * 2)
    checked = misses = 0
    for trial in range(6):
        eye = (rng.uniform(-8, 16), rng.uniform(-8, 16), -12.0 + 30.0 * (trial % 2))
        target = rng.uniform(2, 6, size=3)
        fwd = tuple(target - np.array(eye))
        cam = cam_persp(eye, fwd, (0, 1, 0), 60.0, 5, 4)
        step = rng.uniform(0.3, 0.9)
        r = oracle_lib.render(cube, cam, tf, 0.0, 4.0, step)
        for j in range(4):
            for i in range(5):
                _, ov, dv, _ = oracle_lib.ray(dims[::-1], cam, step, i, j)
                ch = _chord_brute_force(ov, dv, dims, 0.0, 80.0)
                if ch is None:
                    assert np.isinf(r["margin_n"][j, i])
                    misses += 1
                    continue
                q = (ch[1] - ch[0]) / step + 0.5
                np.testing.assert_allclose(r["margin_n"][j, i], abs(q - np.round(q)), atol=1e-8)
                checked += 1
    assert checked >= 20 and misses >= 1


@pytest.mark.parametrize("m,delta,side", [(5, 1e-3, "stop"), (5, 1e-3, "before"), (12, 2e-5, "stop"),
                                          (12, 2e-5, "before"), (1, 1e-4, "stop")])
def test_margin_ert_of_a_constant_opacity_slab(oracle_lib, m, delta, side):
    """Constant opacity a: after sample k the opacity is 1 - (1 - a)^k.  With
    thr = O_m - delta the ray stops at sample m, which lands delta above the
    threshold ('stop'); with thr = O_m + delta sample m lands delta below it
    and the ray stops one sample later ('before').  delta is far below the
    opacity gap between neighbouring samples, so the margin is delta."""
    a = 0.1
    O = lambda k: 1.0 - (1.0 - a) ** k            # noqa: E731
    assert delta < 0.1 * (O(m + 1) - O(m))
    thr = O(m) - delta if side == "stop" else O(m) + delta
    want_n = m if side == "stop" else m + 1
    cam = cam_ortho((1.5, 1.5, -10.0), (0, 0, 1), (0, 1, 0), 2.0, 2, 2)
    tf = np.array([[0.3, 0.6, 0.9, a]] * 2)
    r = oracle_lib.render(_slab_z(64), cam, tf, 0.0, 2.0, 1.0, ert=thr)
    assert (r["n_used"] == want_n).all(), r["n_used"]
    np.testing.assert_allclose(r["margin_ert"], delta, rtol=1e-6, atol=0)
    np.testing.assert_allclose(r["rgba"][..., 3], O(want_n), atol=1e-14)


def test_margin_ert_is_the_minimum_over_the_composited_samples(oracle_lib):
    """Two constant slabs along z (v = 0 transparent, v = 1 opacity 0.5) with
    one blended cell between them: the running opacity is 0 over the
    transparent part, then 0.25 (the sample at z = 19.5 blends 0 and 1), 0.625,
    0.8125, ...  With thr = 0.65 the ray stops at 0.8125 (0.1625 above), but
    the sample before it is 0.025 below: the margin is the minimum over every
    composited sample, 0.025, not the stop sample's distance."""
    nz = 40
    cube = np.zeros((nz, 4, 4), np.float32)
    cube[20:] = 1.0
    tf = np.array([[1.0, 1.0, 1.0, 0.0], [1.0, 1.0, 1.0, 0.5]])
    cam = cam_ortho((1.5, 1.5, -10.0), (0, 0, 1), (0, 1, 0), 2.0, 2, 2)
    r = oracle_lib.render(cube, cam, tf, 0.0, 1.0, 1.0, ert=0.65)
    # samples at z = 0.5, 1.5, ...: the stop is the one at z = 21.5, the 22nd
    assert (r["n_used"] == 22).all(), r["n_used"]
    np.testing.assert_allclose(r["rgba"][..., 3], 0.8125, atol=1e-14)
    np.testing.assert_allclose(r["margin_ert"], 0.025, atol=1e-14)
    # with thr = 0.8 the stop sample itself is the closest (0.0125 above)
    r = oracle_lib.render(cube, cam, tf, 0.0, 1.0, 1.0, ert=0.8)
    assert (r["n_used"] == 22).all()
    np.testing.assert_allclose(r["margin_ert"], 0.0125, atol=1e-14)


def test_margins_on_random_rays_against_brute_force(oracle_lib):
    """Random 8^3 cubes and cameras with early termination: both margins
    equal the values recomputed from an independent per-sample evaluation
    (brute-force chord, scipy trilinear, np.interp lookup, cumulative-product
    opacity), over the samples up to and including the stop."""
    from scipy.interpolate import RegularGridInterpolator
    rng = np.random.default_rng(21)
    nchecked = 0
    for trial in range(4):
        V = (rng.normal(size=(8, 8, 8)) * 4 + 3).astype(np.float32)
        K = 8
        tf = rng.uniform(size=(K, 4))
        tf[:, 3] *= 0.5
        vmin, vmax = -4.0, 12.0
        knots = np.linspace(vmin, vmax, K)
        ip = RegularGridInterpolator((np.arange(8),) * 3, V.astype(np.float64))
        eye = rng.uniform(-6, 14, size=3)
        eye[2] = -8.0 if trial % 2 == 0 else 16.0
        fwd = rng.uniform(2, 5, size=3) - eye
        cam = cam_persp(tuple(eye), tuple(fwd), (0, 1, 0), 35.0, 4, 4)
        thr = (0.3, 0.5, 0.7, 0.9)[trial]
        step = 0.45
        r = oracle_lib.render(V, cam, tf, vmin, vmax, step, ert=thr)
        for j in range(4):
            for i in range(4):
                _, ov, dv, _ = oracle_lib.ray(V.shape, cam, step, i, j)
                ch = _chord_brute_force(ov, dv, (8, 8, 8), 0.0, 60.0)
                if ch is None:
                    assert np.isinf(r["margin_n"][j, i]) and np.isinf(r["margin_ert"][j, i])
                    continue
                q = (ch[1] - ch[0]) / step + 0.5
                np.testing.assert_allclose(r["margin_n"][j, i], abs(q - np.round(q)), atol=1e-8)
                n = int(np.floor(q))
                if n == 0:
                    assert np.isinf(r["margin_ert"][j, i])
                    continue
                t = ch[0] + (np.arange(n) + 0.5) * step
                v = ip((ov[None, :] + t[:, None] * dv[None, :])[:, ::-1])
                alpha = np.interp(v, knots, tf[:, 3])
                O = 1.0 - np.cumprod(1.0 - alpha)
                stop = np.nonzero(O >= thr)[0]
                m = stop[0] + 1 if stop.size else n
                assert r["n_used"][j, i] == m
                np.testing.assert_allclose(r["margin_ert"][j, i], np.abs(O[:m] - thr).min(), atol=1e-9)
                nchecked += 1
    assert nchecked >= 30
