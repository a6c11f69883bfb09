"""Pins for the FP64 oracle: closed forms, hand-derived cases, library
routines, brute force and invariants.  None of these re-types the oracle's own
formulas; each is chosen so that a plausible slip in the oracle (a dropped
term, a sign, a transposed axis, a half-step offset) fails at least one.

Method: Section 3.3-3.4 of the paper (generic transfer function, front-to-back
compositing) with the constant-step trilinear sampling of Section 4.4.
"""
import math
from fractions import Fraction

import numpy as np
import pytest


def cam_ortho(eye, fwd, up, h, W, H):
    return dict(kind=0, eye=eye, forward=fwd, up=up, ortho_height=h, fov_y_deg=0.0, width=W, height=H)


def cam_persp(eye, fwd, up, fov, W, H):
    return dict(kind=1, eye=eye, forward=fwd, up=up, ortho_height=0.0, fov_y_deg=fov, width=W, height=H)


# ---------------------------------------------------------------------------
# Closed forms
# ---------------------------------------------------------------------------

def test_constant_slab_axis_aligned(oracle_lib):
    """Constant density, constant table: opacity 1-(1-a)^n and colour c(1-(1-a)^n).
    A ray along z through an 8^3 box has length 7; step 0.5 puts samples at
    0.25, 0.75, ..., 6.75 (14 of them), step 0.3 at 0.15 ... 6.75 (23)."""
    cube = np.full((8, 8, 8), 10.0, np.float32)
    col = np.array([0.2, 0.4, 0.6])
    a = 0.05
    tf = np.array([[*col, a], [*col, a]])
    cam = cam_ortho((3.5, 3.5, -10.0), (0, 0, 1), (0, 1, 0), 6.0, 4, 4)
    for step, n in ((0.5, 14), (0.3, 23), (1.0, 7), (7.5, 1), (14.5, 0)):
        r = oracle_lib.render(cube, cam, tf, 0.0, 20.0, step)
        assert (r["n_used"] == n).all(), (step, r["n_used"])
        op = 1.0 - (1.0 - a) ** n
        np.testing.assert_allclose(r["rgba"][..., 3], op, rtol=0, atol=1e-14)
        np.testing.assert_allclose(r["rgba"][..., :3], np.broadcast_to(col * op, (4, 4, 3)), atol=1e-14)


def _chord_brute_force(ov, dv, dims, t_lo, t_hi):
    """Entry and exit parameters of a ray in the closed box [0, n-1]^3 found by
    scanning membership on a fine grid and bisecting the two transitions."""
    def inside(t):
        p = ov + t * dv
        return all(0.0 <= p[a] <= dims[a] - 1 for a in range(3))
    ts = np.linspace(t_lo, t_hi, 200001)
    P = ov[None, :] + ts[:, None] * dv[None, :]
    hi = np.array(dims, dtype=np.float64) - 1
    mask = ((P >= 0.0) & (P <= hi[None, :])).all(axis=1)
    idx = np.nonzero(mask)[0]
    if idx.size == 0:
        return None
    def bisect(a, b, want_inside_at_b):
        for _ in range(100):
            m = 0.5 * (a + b)
            if inside(m) == want_inside_at_b:
                b = m
            else:
                a = m
        return b
    i0, i1 = idx[0], idx[-1]
    t_in = ts[0] if i0 == 0 else bisect(ts[i0 - 1], ts[i0], True)
    t_out = ts[-1] if i1 == len(ts) - 1 else bisect(ts[i1 + 1], ts[i1], True)
    return t_in, t_out


def test_constant_slab_oblique_perspective(oracle_lib):
    """Oblique perspective rays through a constant box: the opacity is
    1-(1-a)^n with n = #{k >= 0 : (k+1/2) step <= chord}, the chord measured by
    brute-force membership search (independent of the slab clipping)."""
    dims = (9, 7, 11)
    cube = np.full(dims[::-1], 3.0, np.float32)
    a = 0.07
    tf = np.array([[1, 1, 1, a], [1, 1, 1, a]])
    cam = cam_persp((-6.0, 14.0, -9.0), (0.6, -0.55, 0.75), (0, 1, 0), 50.0, 5, 4)
    step = 0.37
    r = oracle_lib.render(cube, cam, tf, 0.0, 10.0, step)
    hits = 0
    for j in range(4):
        for i in range(5):
            n_o, ov, dv, tin = oracle_lib.ray(dims[::-1], cam, step, i, j)
            ch = _chord_brute_force(ov, dv, dims, 0.0, 60.0)
            if ch is None:
                assert n_o == 0 and r["rgba"][j, i, 3] == 0.0
                continue
            L = ch[1] - ch[0]
            n = 0
            while (n + 0.5) * step <= L:
                n += 1
            assert n == n_o
            assert abs(tin - ch[0]) < 1e-9
            np.testing.assert_allclose(r["rgba"][j, i, 3], 1.0 - (1.0 - a) ** n, atol=1e-13)
            hits += n > 0
    assert hits >= 6


def test_zero_alpha_gives_background_exactly(oracle_lib):
    rng = np.random.default_rng(0)
    cube = rng.normal(size=(6, 7, 8)).astype(np.float32) * 5
    tf = rng.uniform(size=(16, 4))
    tf[:, 3] = 0.0
    bg = (0.1, 0.2, 0.3, 0.4)
    cam = cam_persp((3.5, 3.0, -12.0), (0.1, 0.05, 1.0), (0, 1, 0), 40.0, 6, 5)
    r = oracle_lib.render(cube, cam, tf, -5.0, 5.0, 0.4, bg=bg)
    assert (r["rgba"] == np.array(bg)).all()
    assert r["n_used"].max() > 0


def test_early_termination_closed_form(oracle_lib):
    """Constant opacity a: the ray stops at the first k+1 with 1-(1-a)^(k+1) >= thr."""
    cube = np.full((40, 4, 4), 1.0, np.float32)      # long in z
    a = 0.1
    tf = np.array([[0.5, 0.5, 0.5, a]] * 2)
    cam = cam_ortho((1.5, 1.5, -5.0), (0, 0, 1), (0, 1, 0), 2.0, 2, 2)
    for thr in (0.5, 0.9, 0.99):
        r = oracle_lib.render(cube, cam, tf, 0.0, 2.0, 0.5, ert=thr)
        n_stop = math.ceil(math.log(1.0 - thr) / math.log(1.0 - a))
        assert (r["n_used"] == n_stop).all(), (thr, r["n_used"], n_stop)
        np.testing.assert_allclose(r["rgba"][..., 3], 1 - (1 - a) ** n_stop, atol=1e-14)


# ---------------------------------------------------------------------------
# Hand-derived column (orientation, sample placement, interpolation, lookup)
# ---------------------------------------------------------------------------

def _column_cube():
    # V[z, y, x]; column (x=1, y=1) holds 0, 10, 20, 30 along z.
    V = np.zeros((4, 2, 2), np.float32)
    V[:, 1, 1] = [0, 10, 20, 30]
    V[:, 1, 0] = [40, 40, 40, 40]
    V[:, 0, 1] = [5, 5, 5, 5]
    V[:, 0, 0] = [0, 0, 0, 0]
    return V


def _over(samples):
    """Textbook front-to-back 'over' of (rgb, a) pairs, exact fractions."""
    C = [Fraction(0)] * 3
    T = Fraction(1)
    for rgb, a in samples:
        for ch in range(3):
            C[ch] += T * a * rgb[ch]
        T *= 1 - a
    return [float(c) for c in C] + [float(1 - T)]


def test_hand_summed_column(oracle_lib):
    """2x2x4 cube, orthographic view along +z with up = +y.  The camera basis
    is r = f x up = -x, u = +y, so pixel (0,0) (top-left) sees the column
    x=1, y=1 and pixel (1,1) sees x=0, y=0.  The column is 3 voxels long; step
    1/2 gives samples at z = 1/4, 3/4, ..., 11/4, whose linear values are
    2.5, 7.5, ..., 27.5.  A 2-entry table over [0, 40] blends linearly."""
    V = _column_cube()
    cam = cam_ortho((0.5, 0.5, -5.0), (0, 0, 1), (0, 1, 0), 2.0, 2, 2)
    top = Fraction(4, 10)
    tf = np.array([[0, 0, 0, 0], [1.0, 0.5, 0.25, 0.4]])
    r = oracle_lib.render(V, cam, tf, 0.0, 40.0, 0.5)
    assert (r["n_used"] == 6).all()
    vals = [Fraction(5, 2), Fraction(15, 2), Fraction(25, 2), Fraction(35, 2), Fraction(45, 2),
            Fraction(55, 2)]
    samples = [((v / 40, v / 80, v / 160), top * v / 40) for v in vals]
    np.testing.assert_allclose(r["rgba"][0, 0], _over(samples), atol=1e-15)
    # constant columns
    for (j, i), val in (((0, 1), 40), ((1, 0), 5), ((1, 1), 0)):
        v = Fraction(val)
        s = min(v / 40, Fraction(1))
        samples = [((s, s / 2, s / 4), top * s)] * 6
        np.testing.assert_allclose(r["rgba"][j, i], _over(samples), atol=1e-15)


def test_hand_summed_column_five_entry_table(oracle_lib):
    """Same column through a 5-entry table over [0, 40]: v = 2.5 sits at
    u = 0.25 (entries 0,1), 7.5 at 0.75, 12.5 at 1.25 (entries 1,2), ..."""
    V = _column_cube()
    cam = cam_ortho((0.5, 0.5, -5.0), (0, 0, 1), (0, 1, 0), 2.0, 2, 2)
    TF = [[Fraction(1, 10), Fraction(2, 10), Fraction(3, 10), Fraction(1, 20)],
          [Fraction(9, 10), Fraction(1, 10), Fraction(5, 10), Fraction(3, 20)],
          [Fraction(2, 10), Fraction(8, 10), Fraction(1, 10), Fraction(1, 10)],
          [Fraction(5, 10), Fraction(5, 10), Fraction(9, 10), Fraction(7, 20)],
          [Fraction(3, 10), Fraction(4, 10), Fraction(6, 10), Fraction(1, 2)]]
    tf = np.array([[float(x) for x in row] for row in TF])
    r = oracle_lib.render(V, cam, tf, 0.0, 40.0, 0.5)
    pairs = [(0, Fraction(1, 4)), (0, Fraction(3, 4)), (1, Fraction(1, 4)), (1, Fraction(3, 4)),
             (2, Fraction(1, 4)), (2, Fraction(3, 4))]
    samples = []
    for i0, w in pairs:
        e = [(1 - w) * TF[i0][ch] + w * TF[i0 + 1][ch] for ch in range(4)]
        samples.append((e[:3], e[3]))
    np.testing.assert_allclose(r["rgba"][0, 0], _over(samples), atol=1e-15)


# ---------------------------------------------------------------------------
# Interpolation and lookup against closed forms and library routines
# ---------------------------------------------------------------------------

def test_trilinear_reproduces_multilinear_fields(oracle_lib):
    """Trilinear interpolation is exact for a + bx + cy + dz + e xyz + ..."""
    nx, ny, nz = 7, 5, 6
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    f = lambda x, y, z: 0.3 + 1.7 * x - 2.9 * y + 0.45 * z + 0.11 * x * y - 0.07 * y * z + 0.013 * x * y * z
    V = f(x, y, z).astype(np.float64)
    rng = np.random.default_rng(1)
    for _ in range(200):
        p = rng.uniform([0, 0, 0], [nx - 1, ny - 1, nz - 1])
        assert abs(oracle_lib.trilinear(V, p) - f(*p)) < 1e-11
    # the far faces (clamped cell origin) are still exact
    for p in ([nx - 1, 2.5, 3.25], [1.5, ny - 1, nz - 1], [nx - 1, ny - 1, nz - 1]):
        assert abs(oracle_lib.trilinear(V, p) - f(*p)) < 1e-11


def test_trilinear_matches_scipy(oracle_lib):
    from scipy.interpolate import RegularGridInterpolator
    rng = np.random.default_rng(2)
    V = rng.normal(size=(5, 6, 7)).astype(np.float32)
    ip = RegularGridInterpolator((np.arange(5), np.arange(6), np.arange(7)), V.astype(np.float64))
    for _ in range(200):
        p = rng.uniform([0, 0, 0], [6, 5, 4])
        assert abs(oracle_lib.trilinear(V, p) - ip([p[2], p[1], p[0]])[0]) < 1e-12


def test_tf_lookup_matches_np_interp(oracle_lib):
    rng = np.random.default_rng(3)
    K = 17
    tf = rng.uniform(size=(K, 4))
    vmin, vmax = -3.0, 50.0
    knots = np.linspace(vmin, vmax, K)
    for v in np.concatenate([rng.uniform(-10, 60, 300), knots]):
        got = oracle_lib.tf_lookup(tf, vmin, vmax, v)
        want = [np.interp(v, knots, tf[:, ch]) for ch in range(4)]   # clamps at both ends
        np.testing.assert_allclose(got, want, atol=1e-13)


def test_half_and_bfloat16_widening(oracle_lib):
    """Stored 16-bit voxels widen exactly (numpy float16 is IEEE binary16;
    bfloat16 is the upper half of a binary32)."""
    rng = np.random.default_rng(4)
    vals = np.concatenate([rng.normal(size=50) * 30, [0.0, -0.0, 6.1e-5, 5.96e-8, 65504.0]])
    h = vals.astype(np.float16)
    cube = np.zeros((2, 2, 2), np.float16)
    for v in h:
        cube[...] = v
        assert oracle_lib.trilinear(cube.view(np.uint16), [0.5, 0.5, 0.5], bits="f16") == float(v)
    f32 = vals.astype(np.float32)
    bf = (f32.view(np.uint32) >> 16).astype(np.uint16)
    for b in bf:
        cube16 = np.full((2, 2, 2), b, np.uint16)
        want = float(np.array([np.uint32(b) << np.uint32(16)], np.uint32).view(np.float32)[0])
        assert oracle_lib.trilinear(cube16, [0.0, 0.0, 0.0], bits="bf16") == want


# ---------------------------------------------------------------------------
# Brute force on tiny inputs
# ---------------------------------------------------------------------------

def test_brute_force_tiny_renders(oracle_lib):
    """8^3 random cubes, 4x4 images, random cameras: the oracle equals an
    independent evaluation (brute-force chord, scipy trilinear, np.interp
    table lookup, cumulative-product transmittance)."""
    from scipy.interpolate import RegularGridInterpolator
    rng = np.random.default_rng(5)
    for trial in range(6):
        V = (rng.normal(size=(8, 8, 8)) * 4 + 3).astype(np.float32)
        K = 8
        tf = rng.uniform(size=(K, 4))
        tf[:, 3] *= 0.3
        vmin, vmax = -4.0, 12.0
        knots = np.linspace(vmin, vmax, K)
        ip = RegularGridInterpolator((np.arange(8),) * 3, V.astype(np.float64))
        eye = rng.uniform(-6, 14, size=3)
        eye[2] = -8.0 if trial % 2 == 0 else 16.0
        target = rng.uniform(2, 5, size=3)
        fwd = target - eye
        if trial < 3:
            cam = cam_persp(tuple(eye), tuple(fwd), (0, 1, 0), 35.0, 4, 4)
        else:
            cam = cam_ortho(tuple(eye), tuple(fwd), (0.1, 1, 0), 6.0, 4, 4)
        thr = 0.6 if trial in (1, 4) else 2.0
        step = 0.45
        r = oracle_lib.render(V, cam, tf, vmin, vmax, step, ert=thr)
        for j in range(4):
            for i in range(4):
                n_o, ov, dv, tin = oracle_lib.ray(V.shape, cam, step, i, j)
                lo = -40.0 if cam["kind"] == 0 else 0.0
                ch = _chord_brute_force(ov, dv, (8, 8, 8), lo, 60.0)
                if ch is None or ch[1] - ch[0] < step / 2:
                    assert r["n_used"][j, i] == 0
                    continue
                ks = []
                k = 0
                while (k + 0.5) * step <= ch[1] - ch[0]:
                    ks.append(k)
                    k += 1
                t = ch[0] + (np.array(ks) + 0.5) * step
                P = ov[None, :] + t[:, None] * dv[None, :]
                v = ip(P[:, ::-1])
                rgba = np.stack([np.interp(v, knots, tf[:, c]) for c in range(4)], axis=1)
                a = rgba[:, 3]
                T_after = np.cumprod(1 - a)
                if thr <= 1:
                    stop = np.nonzero(1 - T_after >= thr)[0]
                    m = stop[0] + 1 if stop.size else len(a)
                else:
                    m = len(a)
                T_before = np.concatenate([[1.0], T_after[:-1]])[:m]
                C = (T_before[:, None] * a[:m, None] * rgba[:m, :3]).sum(0)
                want = np.concatenate([C, [1 - T_after[m - 1]]])
                assert r["n_used"][j, i] == m
                np.testing.assert_allclose(r["rgba"][j, i], want, atol=1e-8)


# ---------------------------------------------------------------------------
# Camera model pins
# ---------------------------------------------------------------------------

def test_perspective_silhouette(oracle_lib):
    """Face-on pinhole view of a box: a ray hits iff its direction passes
    through the front face.  With the eye on the axis at distance D in front
    of a face of half-width h, pixel (i, j) hits iff
    |sx| tan(fov/2) aspect <= h/D and |sy| tan(fov/2) <= h/D."""
    n = 11
    cube = np.full((n, n, n), 1.0, np.float32)
    tf = np.array([[1, 1, 1, 0.2]] * 2)
    W, H, fov = 16, 8, 30.0
    D = 17.3
    cx = (n - 1) / 2
    cam = cam_persp((cx, cx, -D), (0, 0, 1), (0, 1, 0), fov, W, H)
    r = oracle_lib.render(cube, cam, tf, 0.0, 2.0, 0.5)
    th = math.tan(math.radians(fov) / 2)
    h = (n - 1) / 2
    for j in range(H):
        for i in range(W):
            sx = (i + 0.5) / W * 2 - 1
            sy = 1 - (j + 0.5) / H * 2
            hit = abs(sx) * th * (W / H) <= h / D and abs(sy) * th <= h / D
            assert (r["rgba"][j, i, 3] > 0) == hit, (i, j)


def test_image_orientation_perspective(oracle_lib):
    """A bright octant at high x, high y seen along +z with up = +y appears
    top-left (r = f x up = -x points left on screen... i.e. +x is on the left)."""
    n = 16
    V = np.zeros((n, n, n), np.float32)
    V[:, n // 2:, n // 2:] = 10.0           # y >= 8, x >= 8
    tf = np.array([[0, 0, 0, 0], [1, 1, 1, 0.5]])
    cam = cam_persp((7.5, 7.5, -30.0), (0, 0, 1), (0, 1, 0), 30.0, 8, 8)
    r = oracle_lib.render(V, cam, tf, 0.0, 10.0, 0.5)
    A = r["rgba"][..., 3]
    assert A[1, 1] > 0.5 and A[6, 6] == 0.0 and A[1, 6] == 0.0 and A[6, 1] == 0.0


# ---------------------------------------------------------------------------
# Invariants
# ---------------------------------------------------------------------------

def test_translation_along_view_direction_ortho(oracle_lib):
    """Samples are anchored at the box entry, so sliding an orthographic eye
    along its view direction leaves the image unchanged."""
    rng = np.random.default_rng(6)
    V = (rng.normal(size=(9, 10, 11)) * 6).astype(np.float32)
    tf = rng.uniform(size=(32, 4)); tf[:, 3] *= 0.2
    fwd = np.array([0.3, -0.2, 1.0]); fwd /= np.linalg.norm(fwd)
    eye = np.array([5.0, 4.5, -10.0])
    base = oracle_lib.render(V, cam_ortho(tuple(eye), tuple(fwd), (0, 1, 0), 9.0, 12, 10), tf, -10, 10, 0.35)
    for s in (-3.7, 2.2, 11.0):
        r = oracle_lib.render(V, cam_ortho(tuple(eye + s * fwd), tuple(fwd), (0, 1, 0), 9.0, 12, 10), tf,
                              -10, 10, 0.35)
        np.testing.assert_allclose(r["rgba"], base["rgba"], atol=1e-12)
        assert (r["n_used"] == base["n_used"]).all()


def test_volume_translation_shifts_image(oracle_lib):
    """Moving the volume origin by one pixel pitch along the screen axes
    shifts the orthographic image by exactly one pixel."""
    rng = np.random.default_rng(7)
    V = (rng.normal(size=(8, 12, 12)) * 6).astype(np.float32)
    tf = rng.uniform(size=(16, 4)); tf[:, 3] *= 0.3
    W = H = 16
    cam = cam_ortho((5.5, 5.5, -10.0), (0, 0, 1), (0, 1, 0), float(H) * 1.0, W, H)   # pitch 1 voxel
    base = oracle_lib.render(V, cam, tf, -10, 10, 0.5)["rgba"]
    # r = -x: moving the volume by +1 in x moves it one pixel to the left
    sx = oracle_lib.render(V, cam, tf, -10, 10, 0.5, origin=(1.0, 0.0, 0.0))["rgba"]
    np.testing.assert_allclose(sx[:, :-1], base[:, 1:], atol=1e-12)
    # u = +y: moving the volume by +1 in y moves it one pixel up (toward row 0)
    sy = oracle_lib.render(V, cam, tf, -10, 10, 0.5, origin=(0.0, 1.0, 0.0))["rgba"]
    np.testing.assert_allclose(sy[:-1, :], base[1:, :], atol=1e-12)


def test_rotation_of_cube_and_camera(oracle_lib):
    """Rotating the data by 90 degrees about z and the camera with it leaves
    the image unchanged (catches axis transposes in the dense layout)."""
    rng = np.random.default_rng(8)
    n, nz = 10, 7
    V = (rng.normal(size=(nz, n, n)) * 6).astype(np.float32)
    # rotation R: (x, y) -> (n-1-y, x) about the box axis.  New[z, y', x'] = V[z, y, x]
    # with x' = n-1-y, y' = x, i.e. New[z, y', x'] = V[z, n-1-x', y'].
    Vr = np.empty_like(V)
    for yp in range(n):
        for xp in range(n):
            Vr[:, yp, xp] = V[:, n - 1 - xp, yp]
    tf = rng.uniform(size=(16, 4)); tf[:, 3] *= 0.3

    def R(p, is_dir):
        x, y, z = p
        if is_dir:
            return (-y, x, z)
        return (n - 1 - y, x, z)
    eye, fwd, up = (2.0, -14.0, -6.0), (0.25, 1.0, 0.45), (0.0, 0.2, 1.0)
    for kind in (0, 1):
        if kind:
            c0, c1 = cam_persp(eye, fwd, up, 40, 9, 7), cam_persp(R(eye, 0), R(fwd, 1), R(up, 1), 40, 9, 7)
        else:
            c0, c1 = cam_ortho(eye, fwd, up, 8, 9, 7), cam_ortho(R(eye, 0), R(fwd, 1), R(up, 1), 8, 9, 7)
        a = oracle_lib.render(V, c0, tf, -10, 10, 0.4)
        b = oracle_lib.render(Vr, c1, tf, -10, 10, 0.4)
        np.testing.assert_allclose(a["rgba"], b["rgba"], atol=1e-9)
        assert a["n_used"].sum() > 0


def test_early_termination_error_bound(oracle_lib):
    """ERT changes the image by at most 1 - thr (opacity and colour)."""
    rng = np.random.default_rng(9)
    V = (rng.normal(size=(20, 12, 12)) * 8 + 10).astype(np.float32)
    tf = rng.uniform(size=(32, 4)); tf[:, 3] *= 0.6
    cam = cam_persp((5.5, 5.5, -20.0), (0, 0, 1), (0, 1, 0), 30, 10, 10)
    full = oracle_lib.render(V, cam, tf, -10, 30, 0.5, ert=2.0)
    for thr in (0.9, 0.99):
        e = oracle_lib.render(V, cam, tf, -10, 30, 0.5, ert=thr)
        assert (e["n_used"] <= full["n_used"]).all() and (e["n_used"] < full["n_used"]).any()
        assert np.abs(e["rgba"] - full["rgba"]).max() <= 1 - thr + 1e-12


def test_mirror_symmetry_perspective(oracle_lib):
    """Data symmetric under x -> n-1-x and a camera in the symmetry plane give
    an image symmetric under column reversal."""
    rng = np.random.default_rng(10)
    n = 12
    V = (rng.normal(size=(n, n, n)) * 6).astype(np.float32)
    V = V + V[:, :, ::-1]
    tf = rng.uniform(size=(16, 4)); tf[:, 3] *= 0.3
    cam = cam_persp(((n - 1) / 2, 15.0, -18.0), (0.0, -0.5, 1.0), (0, 1, 0), 45, 10, 8)
    r = oracle_lib.render(V, cam, tf, -20, 20, 0.4)["rgba"]
    np.testing.assert_allclose(r, r[:, ::-1], atol=1e-12)
