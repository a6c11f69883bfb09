"""Pins for the oracle's backward pass: central finite differences of the
oracle's FORWARD render (a different computation from its store-all reverse
sweep) and a closed form for a constant slab.

The loss is L = sum over pixels and channels of (I - I_target)^2 unless a
test says otherwise; dL/dI = 2 (I - I_target).
"""
import numpy as np
import pytest


def cam_persp(eye, fwd, up, fov, W, H):
    return dict(kind=1, eye=eye, forward=fwd, up=up, ortho_height=0.0, fov_y_deg=fov, width=W, height=H)


def cam_ortho(eye, fwd, up, h, W, H):
    return dict(kind=0, eye=eye, forward=fwd, up=up, ortho_height=h, fov_y_deg=0.0, width=W, height=H)


def _setup(seed, ert=2.0, bg=(0.0, 0.0, 0.0, 0.0)):
    rng = np.random.default_rng(seed)
    V = (rng.normal(size=(8, 8, 8)) * 4 + 4).astype(np.float64)
    K = 12
    tf = rng.uniform(size=(K, 4))
    tf[:, 3] *= 0.35
    vmin, vmax = -6.0, 14.0
    cam = cam_persp((3.2, 4.1, -9.0), (0.05, -0.08, 1.0), (0, 1, 0), 38.0, 5, 4)
    target = rng.uniform(size=(4, 5, 4))
    return V, tf, vmin, vmax, cam, target, dict(ert=ert, bg=bg)


def _loss(orc, V, tf, vmin, vmax, cam, target, kw):
    I = orc.render(V, cam, tf, vmin, vmax, 0.45, nthreads=1, **kw)["rgba"]
    return float(((I - target) ** 2).sum()), I


def _fd_check(orc, seed, ert, bg):
    V, tf, vmin, vmax, cam, target, kw = _setup(seed, ert, bg)
    L0, I = _loss(orc, V, tf, vmin, vmax, cam, target, kw)
    gI = 2.0 * (I - target)
    gtf, gvox = orc.render_backward(V, cam, tf, vmin, vmax, 0.45, gI, nthreads=1, **kw)
    h = 1e-6
    checked = 0
    # every table entry
    for idx in np.ndindex(*tf.shape):
        tp, tm = tf.copy(), tf.copy()
        tp[idx] += h
        tm[idx] -= h
        Lp = _loss(orc, V, tp, vmin, vmax, cam, target, kw)[0]
        Lm = _loss(orc, V, tm, vmin, vmax, cam, target, kw)[0]
        fd = (Lp - Lm) / (2 * h)
        # the loss is polynomial in the table entries (no kinks): tight check
        assert abs(gtf[idx] - fd) <= 1e-6 * max(1.0, abs(fd)), (idx, gtf[idx], fd)
        checked += 1
    # a sample of voxels (kinks: table knots, cell faces -> compare one-sided FDs)
    rng = np.random.default_rng(seed + 100)
    flat = np.flatnonzero(np.abs(gvox) > 0)
    for q in rng.choice(flat, size=min(40, flat.size), replace=False):
        z, y, x = np.unravel_index(q, V.shape)
        Vp, Vm = V.copy(), V.copy()
        Vp[z, y, x] += h
        Vm[z, y, x] -= h
        Lp = _loss(orc, Vp, tf, vmin, vmax, cam, target, kw)[0]
        Lm = _loss(orc, Vm, tf, vmin, vmax, cam, target, kw)[0]
        right, left = (Lp - L0) / h, (L0 - Lm) / h
        if abs(right - left) > 1e-4 * max(1.0, abs(right)):
            continue                      # a kink within h: skip this voxel
        fd = (Lp - Lm) / (2 * h)
        assert abs(gvox[z, y, x] - fd) <= 1e-5 * max(1.0, abs(fd)), ((z, y, x), gvox[z, y, x], fd)
        checked += 1
    assert checked > tf.size + 20


@pytest.mark.parametrize("seed,ert,bg", [(0, 2.0, (0, 0, 0, 0)), (1, 0.7, (0, 0, 0, 0)),
                                         (2, 2.0, (0.2, 0.5, 0.1, 0.3))])
def test_backward_matches_central_differences(oracle_lib, seed, ert, bg):
    _fd_check(oracle_lib, seed, ert, bg)


def test_constant_slab_opacity_gradient(oracle_lib):
    """Constant density and table opacity a over n samples: the output opacity
    is 1-(1-a)^n, so with L = sum of output opacities, dL/da summed over the
    two table entries that each sample blends is n (1-a)^(n-1) per pixel."""
    cube = np.full((8, 8, 8), 10.0, np.float64)
    a = 0.05
    tf = np.array([[0.3, 0.3, 0.3, a]] * 2)
    cam = cam_ortho((3.5, 3.5, -10.0), (0, 0, 1), (0, 1, 0), 6.0, 4, 4)
    g = np.zeros((4, 4, 4))
    g[..., 3] = 1.0
    gtf, _ = oracle_lib.render_backward(cube, cam, tf, 0.0, 20.0, 0.5, g, want_vox=False)
    n = 14
    np.testing.assert_allclose(gtf[:, 3].sum(), 16 * n * (1 - a) ** (n - 1), rtol=1e-12)
    # colour entries: dL/dc = 0 for an opacity-only loss
    assert np.abs(gtf[:, :3]).max() == 0.0
    # value 10 sits exactly half way through the 2-entry table over [0, 20]
    np.testing.assert_allclose(gtf[0, 3], gtf[1, 3], rtol=1e-12)


def test_zero_opacity_table_has_zero_colour_gradient(oracle_lib):
    """With a = 0 everywhere nothing is emitted: dL/d(colour entries) = 0."""
    rng = np.random.default_rng(3)
    V = rng.normal(size=(6, 6, 6)) * 3
    tf = rng.uniform(size=(8, 4))
    tf[:, 3] = 0.0
    cam = cam_persp((2.5, 2.5, -8.0), (0, 0, 1), (0, 1, 0), 40, 4, 4)
    g = rng.normal(size=(4, 4, 4))
    gtf, _ = oracle_lib.render_backward(V, cam, tf, -5, 5, 0.5, g, want_vox=False)
    assert np.abs(gtf[:, :3]).max() == 0.0
    assert np.abs(gtf[:, 3]).max() > 0.0


# ---------------------------------------------------------------------------
# The kink bound of the voxel gradient (orc_render_backward_kinks)
# ---------------------------------------------------------------------------

def _kink_scene(value):
    """Constant cube along z with an opacity-only table of three entries over
    [0, 4] (u = v / 2), orthographic rays along z, loss L = sum of output
    opacity (dL/dI = (0, 0, 0, 1)): every sample's opacity term has the same
    sign, so the bound (a sum of magnitudes) equals the gap between the two
    one-sided derivatives."""
    V = np.full((10, 6, 6), value, np.float64)
    tf = np.array([[0.0, 0.0, 0.0, 0.05], [0.0, 0.0, 0.0, 0.2], [0.0, 0.0, 0.0, 0.1]])
    cam = cam_ortho((2.5, 2.5, -20.0), (0, 0, 1), (0, 1, 0), 4.0, 4, 4)
    g = np.zeros((4, 4, 4))
    g[..., 3] = 1.0
    return V, tf, cam, g


def _one_sided(orc, V, tf, cam, voxel, h=1e-6):
    def L(x):
        W = V.copy()
        W[voxel] = x
        return float(orc.render(W, cam, tf, 0.0, 4.0, 0.7, nthreads=1)["rgba"][..., 3].sum())
    x = V[voxel]
    return (L(x + h) - L(x)) / h, (L(x) - L(x - h)) / h


@pytest.mark.parametrize("value,end", [(2.0, 2.0), (4.0, 4.0), (2.6, None), (2.0 + 1e-3, 2.0)])
def test_kink_bound_is_the_gap_between_one_sided_derivatives(oracle_lib, value, end):
    """u = 1 is the end between the table's two intervals (opacity slopes
    +0.15 and -0.1 per entry, i.e. per 2 units of value): the voxel gradient
    there is either one-sided derivative, and the bound is their gap.  u = 2
    is vmax: one side has no slope at all.  u = 1.3 is inside an interval: no
    bound.  u = 1 + 5e-4 is within the 1e-3 tolerance of the end u = 1: its
    bound is the gap of the one-sided derivatives at that end."""
    V, tf, cam, g = _kink_scene(value)
    _, gvox, kink, mag = oracle_lib.render_backward(V, cam, tf, 0.0, 4.0, 0.7, g, nthreads=1, kink_eps=1e-3)
    kinked = end is not None
    for voxel in ((4, 2, 2), (7, 3, 2), (1, 2, 3)):
        Vk = _kink_scene(end)[0] if kinked else V
        d_plus, d_minus = _one_sided(oracle_lib, Vk, tf, cam, voxel)
        if kinked:
            assert abs(d_plus - d_minus) > 1e-2
            # near the end (not on it) the samples' weights differ from those at
            # the end by O(u - end) = 5e-4, and so does the bound
            np.testing.assert_allclose(kink[voxel], abs(d_plus - d_minus), rtol=1e-4 if value == end else 3e-3,
                                       atol=1e-9)
            if value == end:
                lo, hi = min(d_plus, d_minus), max(d_plus, d_minus)
                assert lo - 1e-5 <= gvox[voxel] <= hi + 1e-5
        else:
            assert kink[voxel] == 0.0
            np.testing.assert_allclose(gvox[voxel], d_plus, rtol=1e-4, atol=1e-9)
            np.testing.assert_allclose(d_plus, d_minus, rtol=1e-4, atol=1e-9)
            # one sign everywhere and no colour: no cancellation, the magnitude is the gradient's
            np.testing.assert_allclose(mag[voxel], abs(gvox[voxel]), rtol=1e-12)
    # a tolerance below the distance to the end finds no kink
    if value == 2.0 + 1e-3:
        _, _, kink, _ = oracle_lib.render_backward(V, cam, tf, 0.0, 4.0, 0.7, g, nthreads=1, kink_eps=1e-4)
        assert (kink == 0.0).all()


def test_kink_bound_leaves_gradients_unchanged(oracle_lib):
    """Asking for the bound does not change the gradients; random data with a
    wide tolerance flags only voxels that some sample near an interval end
    touches."""
    V, tf, vmin, vmax, cam, target, kw = _setup(4)
    _, I = _loss(oracle_lib, V, tf, vmin, vmax, cam, target, kw)
    gI = 2.0 * (I - target)
    a = oracle_lib.render_backward(V, cam, tf, vmin, vmax, 0.45, gI, nthreads=1, **kw)
    b = oracle_lib.render_backward(V, cam, tf, vmin, vmax, 0.45, gI, nthreads=1, kink_eps=0.05, **kw)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    assert (b[2] >= 0).all() and 0 < (b[2] > 0).sum() < (a[1] != 0).sum()
    # the magnitudes bound the gradient (triangle inequality), and cancel somewhere
    mag = b[3]
    assert (mag >= np.abs(a[1]) * (1 - 1e-12)).all()
    assert (mag > 2 * np.abs(a[1])).any()
