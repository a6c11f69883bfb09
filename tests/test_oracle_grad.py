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
