"""Pins for the oracle's sort-last building blocks (Sections 3.2 and 3.4):
sub-box renders composited in visibility order equal the whole render; a
constant slab split in two in closed form; the over operator's order."""
import numpy as np
import pytest


def cam_ortho(eye, fwd, up, h, W, H):
    return dict(kind=0, eye=eye, forward=fwd, up=up, ortho_height=h, fov_y_deg=0.0, width=W, height=H)


def cam_persp(eye, fwd, up, fov, W, H):
    return dict(kind=1, eye=eye, forward=fwd, up=up, ortho_height=0.0, fov_y_deg=fov, width=W, height=H)


def _boxes(cells, splits):
    """Partition of the cell index ranges [0, cells[a]) into splits[a] parts per axis."""
    edges = [np.linspace(0, n, s + 1).round().astype(int) for n, s in zip(cells, splits)]
    for i in range(splits[0]):
        for j in range(splits[1]):
            for k in range(splits[2]):
                yield ((edges[0][i], edges[1][j], edges[2][k]), (edges[0][i + 1], edges[1][j + 1], edges[2][k + 1]))


@pytest.mark.parametrize("splits", [(2, 2, 2), (3, 1, 2), (1, 4, 1)])
def test_subbox_composite_equals_whole_render(oracle_lib, splits):
    rng = np.random.default_rng(sum(splits))
    dims = (13, 11, 15)                                     # x, y, z voxels -> 12 x 10 x 14 cells
    cube = rng.standard_normal(dims[::-1]).astype(np.float32)
    tf = rng.uniform(0, 1, (12, 4)) * np.array([1, 1, 1, 0.35])
    bg = (0.1, 0.0, 0.2, 0.3)
    cams = [cam_persp((-14.0, 19.0, -16.0), (0.6, -0.6, 0.55), (0, 1, 0), 40.0, 14, 11),
            cam_persp((25.0, 4.0, 30.0), (-0.8, 0.1, -0.7), (0, 1, 0), 45.0, 12, 12),
            cam_ortho((6.0, 5.0, -20.0), (0.05, 0.02, 1.0), (0, 1, 0), 16.0, 10, 9)]
    cells = [d - 1 for d in dims]
    for cam in cams:
        whole = oracle_lib.render(cube, cam, tf, -3.0, 3.0, 0.37, ert=2.0, bg=bg)
        parts = [oracle_lib.render_subbox(cube, cam, tf, -3.0, 3.0, 0.37, lo, hi) for lo, hi in _boxes(cells, splits)]
        assert (sum(p["count"] for p in parts) == whole["n_used"]).all()    # each sample in one sub-box
        got = oracle_lib.composite([p["partial"] for p in parts], [p["depth"] for p in parts], bg=bg)
        np.testing.assert_allclose(got, whole["rgba"], atol=1e-12)
        assert whole["rgba"][..., 3].max() > 0.3


def test_split_slab_closed_form(oracle_lib):
    """A constant slab along z cut into the cells z < 3 and z >= 3: with samples
    at z = 0.25, 0.75, ... the front half holds 6 samples and the back 8, so
    T_front = (1-a)^6, C_front = c (1 - (1-a)^6), and the composite is the
    whole slab's 1 - (1-a)^14."""
    cube = np.full((8, 4, 4), 10.0, np.float32)
    c, a = np.array([0.3, 0.5, 0.7]), 0.1
    tf = np.array([[*c, a], [*c, a]])
    cam = cam_ortho((1.5, 1.5, -10.0), (0, 0, 1), (0, 1, 0), 2.0, 2, 2)
    front = oracle_lib.render_subbox(cube, cam, tf, 0.0, 20.0, 0.5, (0, 0, 0), (3, 3, 3))
    back = oracle_lib.render_subbox(cube, cam, tf, 0.0, 20.0, 0.5, (0, 0, 3), (3, 3, 7))
    assert (front["count"] == 6).all() and (back["count"] == 8).all()
    np.testing.assert_allclose(front["partial"][..., 3], 0.9 ** 6, atol=1e-15)
    np.testing.assert_allclose(front["partial"][..., :3], np.broadcast_to(c * (1 - 0.9 ** 6), (2, 2, 3)), atol=1e-15)
    np.testing.assert_allclose(front["depth"], 10.25, atol=1e-12)           # t of the sample at z = 0.25
    got = oracle_lib.composite([back["partial"], front["partial"]], [back["depth"], front["depth"]])
    np.testing.assert_allclose(got[..., 3], 1 - 0.9 ** 14, atol=1e-14)
    np.testing.assert_allclose(got[..., :3], np.broadcast_to(c * (1 - 0.9 ** 14), (2, 2, 3)), atol=1e-14)


def test_over_is_not_commutative(oracle_lib):
    """Two sub-images of different colours: front-to-back by depth differs from
    the swapped order, so the composite must follow the depths."""
    p1 = np.array([[[0.5, 0.0, 0.0, 0.5]]])
    p2 = np.array([[[0.0, 0.4, 0.0, 0.2]]])
    d1, d2 = np.array([[1.0]]), np.array([[2.0]])
    a = oracle_lib.composite([p1, p2], [d1, d2])
    b = oracle_lib.composite([p1, p2], [d2, d1])
    np.testing.assert_allclose(a[0, 0], [0.5, 0.2, 0.0, 0.9])
    np.testing.assert_allclose(b[0, 0], [0.1, 0.4, 0.0, 0.9])
    empty = np.array([[[0.0, 0.0, 0.0, 1.0]]])
    np.testing.assert_allclose(oracle_lib.composite([empty, p2], [np.array([[np.inf]]), d2])[0, 0], [0, 0.4, 0, 0.8])
