"""Pins for the oracle's further uses of the ray: the 3D spectrum tool
(Section 4.4), maximum intensity projection (Section 3.3.1) and the
sigma-clipping transfer function with its statistical mini-map (Section 4.5).
Closed forms, brute force with library interpolation, and invariants; none
re-types the oracle's formulas."""
import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator


def cam_ortho(eye, fwd, up, h, W, H):
    return dict(kind=0, eye=eye, forward=fwd, up=up, ortho_height=h, fov_y_deg=0.0, width=W, height=H)


def cam_persp(eye, fwd, up, fov, W, H):
    return dict(kind=1, eye=eye, forward=fwd, up=up, ortho_height=0.0, fov_y_deg=fov, width=W, height=H)


def _interp(cube):
    nz, ny, nx = cube.shape
    f = RegularGridInterpolator((np.arange(nz), np.arange(ny), np.arange(nx)), cube.astype(np.float64))
    return lambda p: f(np.clip(np.asarray(p)[:, ::-1], 0, np.array([nz - 1, ny - 1, nx - 1])))


# ---------------------------------------------------------------------------
# 3D spectrum tool
# ---------------------------------------------------------------------------

def test_profile_axis_column_is_linear_in_z(oracle_lib):
    """An orthographic ray along +z through voxel centre (x, y) samples
    z_k = (k + 1/2) step: trilinear reduces to linear interpolation of the
    voxel column, which np.interp gives independently; n = floor(L/step + 1/2)."""
    rng = np.random.default_rng(3)
    cube = rng.standard_normal((9, 6, 5)).astype(np.float32)
    # 5x6 pixels of pitch 1 centred on the box; r = f x up = -x, u = +y, so
    # pixel (i, j) is column (x = 4 - i, y = 5 - j)
    cam = cam_ortho((2.0, 2.5, -20.0), (0, 0, 1), (0, 1, 0), 6.0, 5, 6)
    for step in (0.5, 0.7, 1.0):
        for (i, j) in ((1, 1), (2, 3), (3, 4)):           # interior columns (not on the box faces)
            x, y = 4 - i, 5 - j
            vals = oracle_lib.profile(cube, cam, step, i, j)
            n = int(np.floor(8.0 / step + 0.5))
            assert vals.shape == (n,)
            z = (np.arange(n) + 0.5) * step
            np.testing.assert_allclose(vals, np.interp(z, np.arange(9), cube[:, y, x].astype(np.float64)),
                                       rtol=0, atol=1e-12)


def test_profile_oblique_matches_library_interpolation(oracle_lib):
    """An oblique perspective ray: the profile equals scipy's trilinear
    interpolation at the positions of the independent ray probe."""
    rng = np.random.default_rng(4)
    cube = rng.standard_normal((7, 8, 9)).astype(np.float32)
    cam = cam_persp((-6.0, 11.0, -9.0), (0.6, -0.5, 0.7), (0, 1, 0), 35.0, 9, 7)
    f = _interp(cube)
    for (i, j) in ((4, 3), (1, 5), (7, 1)):
        n, ov, dv, tin = oracle_lib.ray(cube.shape, cam, 0.4, i, j)
        vals = oracle_lib.profile(cube, cam, 0.4, i, j)
        assert vals.shape == (n,)
        if n:
            t = tin + (np.arange(n) + 0.5) * 0.4
            np.testing.assert_allclose(vals, f(ov[None, :] + t[:, None] * dv[None, :]), atol=1e-12)


def test_profile_miss_is_empty(oracle_lib):
    cube = np.zeros((4, 4, 4), np.float32)
    cam = cam_ortho((30.0, 30.0, -10.0), (0, 0, 1), (0, 1, 0), 2.0, 2, 2)
    assert oracle_lib.profile(cube, cam, 0.5, 0, 0).shape == (0,)


# ---------------------------------------------------------------------------
# Maximum intensity projection
# ---------------------------------------------------------------------------

def test_mip_constant_cube(oracle_lib):
    """MIP of a constant cube is the constant: the pixel is its table entry
    composited once over the background (hand-computed blend)."""
    cube = np.full((6, 6, 6), 3.0, np.float32)
    tf = np.array([[0.0, 0.0, 0.0, 0.0], [1.0, 0.5, 0.25, 0.8]])       # u = 3/4 of the way
    cam = cam_ortho((2.5, 2.5, -9.0), (0, 0, 1), (0, 1, 0), 4.0, 3, 3)
    bg = (0.1, 0.2, 0.3, 0.4)
    r = oracle_lib.render_mip(cube, cam, tf, -3.0, 5.0, 0.5, bg=bg)
    a = 0.75 * 0.8
    c = 0.75 * np.array([1.0, 0.5, 0.25])
    want = [a * c[0] + (1 - a) * 0.1, a * c[1] + (1 - a) * 0.2, a * c[2] + (1 - a) * 0.3, a + (1 - a) * 0.4]
    np.testing.assert_allclose(r["rgba"], np.broadcast_to(want, (3, 3, 4)), atol=1e-14)
    np.testing.assert_allclose(r["vmax"], 3.0, atol=1e-14)
    assert (r["n_used"] == 10).all()                      # floor(5/0.5 + 1/2): all samples, no termination


def test_mip_single_bright_voxel(oracle_lib):
    """One voxel of value 8 in a zero cube, an axis ray through its column:
    the nearest samples at step 0.5 sit 0.25 from it, so the maximum is
    8 x 0.75 = 6 (a half-step offset or a dropped weight changes it)."""
    cube = np.zeros((9, 5, 5), np.float32)
    cube[4, 2, 2] = 8.0
    cam = cam_ortho((2.0, 2.0, -5.0), (0, 0, 1), (0, 1, 0), 1.0, 1, 1)
    tf = np.array([[0, 0, 0, 0], [1, 1, 1, 1.0]])
    r = oracle_lib.render_mip(cube, cam, tf, 0.0, 8.0, 0.5)
    assert r["vmax"][0, 0] == pytest.approx(6.0, abs=1e-14)
    r = oracle_lib.render_mip(cube, cam, tf, 0.0, 8.0, 0.4)          # samples at 0.2 + 0.4k: 4.2 nearest
    assert r["vmax"][0, 0] == pytest.approx(8.0 * 0.8, abs=1e-12)


def test_mip_brute_force_and_miss(oracle_lib):
    """Every pixel of a random perspective view: the maximum of scipy's
    trilinear values at the probe's sample positions; misses show bg."""
    rng = np.random.default_rng(8)
    cube = rng.standard_normal((8, 7, 9)).astype(np.float32)
    cam = cam_persp((-5.0, 9.0, -8.0), (0.5, -0.6, 0.6), (0, 1, 0), 50.0, 8, 6)
    f = _interp(cube)
    bg = (0.0, 0.1, 0.0, 0.2)
    r = oracle_lib.render_mip(cube, cam, [[0, 0, 0, 0], [1, 1, 1, 1]], -4.0, 4.0, 0.35, bg=bg)
    hits = 0
    for j in range(6):
        for i in range(8):
            n, ov, dv, tin = oracle_lib.ray(cube.shape, cam, 0.35, i, j)
            assert r["n_used"][j, i] == n
            if n == 0:
                np.testing.assert_allclose(r["rgba"][j, i], bg)
                assert np.isnan(r["vmax"][j, i])
                continue
            hits += 1
            t = tin + (np.arange(n) + 0.5) * 0.35
            assert r["vmax"][j, i] == pytest.approx(f(ov[None, :] + t[:, None] * dv[None, :]).max(), abs=1e-12)
    assert hits > 10


def test_mip_independent_of_march_direction(oracle_lib):
    """Max is order-free: viewing along -z instead of +z (same rays reversed,
    image mirrored left-right) gives the same maxima."""
    rng = np.random.default_rng(9)
    cube = rng.standard_normal((6, 5, 7)).astype(np.float32)
    tf = [[0, 0, 0, 0], [1, 1, 1, 1]]
    a = oracle_lib.render_mip(cube, cam_ortho((3.0, 2.0, -9.0), (0, 0, 1), (0, 1, 0), 4.0, 6, 4), tf, -4, 4, 0.5)
    b = oracle_lib.render_mip(cube, cam_ortho((3.0, 2.0, 14.0), (0, 0, -1), (0, 1, 0), 4.0, 6, 4), tf, -4, 4, 0.5)
    np.testing.assert_allclose(a["vmax"], b["vmax"][:, ::-1], atol=1e-12)


# ---------------------------------------------------------------------------
# Sigma clipping: mini-map and scaled lookup
# ---------------------------------------------------------------------------

def test_minimap_of_a_ramp(oracle_lib):
    """v = x + 10 y: a region spanning x0..x1 (L voxels) and y0..y1 (M) has mean
    (x0+x1)/2 + 10 (y0+y1)/2 and, x and y independent and uniform, variance
    (L^2-1)/12 + 100 (M^2-1)/12 -- including the short last regions."""
    nz, ny, nx = 5, 7, 10
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cube = (x + 10.0 * y).astype(np.float32)
    region = (4, 3, 2)
    st = oracle_lib.minimap(cube, region)
    assert st.shape == (3, 3, 3, 2)
    for k in range(3):
        for j in range(3):
            for i in range(3):
                x0, x1 = 4 * i, min(4 * i + 4, nx) - 1
                y0, y1 = 3 * j, min(3 * j + 3, ny) - 1
                L, M = x1 - x0 + 1, y1 - y0 + 1
                assert st[k, j, i, 0] == pytest.approx((x0 + x1) / 2 + 10 * (y0 + y1) / 2, abs=1e-12)
                assert st[k, j, i, 1] == pytest.approx(np.sqrt((L * L - 1) / 12 + 100 * (M * M - 1) / 12),
                                                       abs=1e-12)


def test_minimap_interpolation_recovers_a_ramp(oracle_lib):
    """With v = x and full regions of 4 voxels the region means sit exactly at
    the region centres' x, so the interpolated mean at x is x between the
    first and last centres and clamps beyond them; y and z do not matter."""
    cube = np.broadcast_to(np.arange(16, dtype=np.float32), (6, 5, 16)).copy()
    region = (4, 5, 3)
    st = oracle_lib.minimap(cube, region)
    for xq in (0.0, 1.5, 2.0, 5.25, 9.9, 13.5, 15.0):
        mean, sd = oracle_lib.minimap_sample(st, region, (xq, 2.2, 3.7))
        assert mean == pytest.approx(min(max(xq, 1.5), 13.5), abs=1e-12)
        assert sd == pytest.approx(np.sqrt(15.0 / 12.0), abs=1e-12)


def test_sigma_with_one_region_is_a_rescaled_table(oracle_lib):
    """A single region: mean and sd are constants, so the sigma-clipped render
    over [vmin, vmax] (units of sd) equals the plain render over
    [mu + vmin sd, mu + vmax sd]."""
    rng = np.random.default_rng(11)
    cube = (2.0 + 1.5 * rng.standard_normal((10, 9, 8))).astype(np.float32)
    st = oracle_lib.minimap(cube, (8, 9, 10))
    mu, sd = st[0, 0, 0]
    assert mu == pytest.approx(cube.astype(np.float64).mean(), rel=1e-12)
    assert sd == pytest.approx(cube.astype(np.float64).std(), rel=1e-12)
    tf = rng.uniform(0, 1, (16, 4)) * np.array([1, 1, 1, 0.3])
    cam = cam_persp((-9.0, 14.0, -12.0), (0.5, -0.6, 0.6), (0, 1, 0), 40.0, 12, 9)
    s = oracle_lib.render_sigma(cube, cam, tf, -1.0, 3.0, 0.6, st, (8, 9, 10), ert=0.9, bg=(0, 0, 0.2, 0.1))
    p = oracle_lib.render(cube, cam, tf, mu - sd, mu + 3.0 * sd, 0.6, ert=0.9, bg=(0, 0, 0.2, 0.1))
    np.testing.assert_allclose(s["rgba"], p["rgba"], atol=1e-10)
    assert (s["n_used"] == p["n_used"]).all()
    assert p["rgba"][..., 3].max() > 0.2


def test_sigma_local_threshold_hides_bright_background(oracle_lib):
    """Two halves with different noise levels and means: in units of the local
    sd both halves look alike, so a table opaque only above 3 sigma renders the
    same (small) opacity on both halves, where the plain render saturates on
    the bright half.  Checked on the brute-force definition at the centre."""
    rng = np.random.default_rng(12)
    cube = rng.standard_normal((16, 8, 16)).astype(np.float64)
    cube[:, :, 8:] = 50.0 + 10.0 * cube[:, :, 8:]
    cube = cube.astype(np.float32)
    region = (8, 8, 16)
    st = oracle_lib.minimap(cube, region)
    assert st.shape == (1, 1, 2, 2)
    tf = np.zeros((8, 4))
    tf[-1] = (1, 1, 1, 1)
    cam = cam_ortho((7.5, 3.5, -20.0), (0, 0, 1), (0, 1, 0), 8.0, 16, 8)
    s = oracle_lib.render_sigma(cube, cam, tf, 0.0, 4.0, 1.0, st, region)
    p = oracle_lib.render(cube, cam, tf, 0.0, 4.0, 1.0)
    # r = f x up = -x: image columns 0..7 look at x = 15..8, the bright half
    assert p["rgba"][..., 3][:, :4].min() > 0.99           # plain: bright half fully opaque
    assert s["rgba"][..., 3][:, :4].max() < 0.9             # local threshold: not
    assert p["rgba"][..., 3][:, 12:].max() < 0.9            # the quiet half, plain and local alike
    assert s["rgba"][..., 3][:, 12:].max() < 0.9
