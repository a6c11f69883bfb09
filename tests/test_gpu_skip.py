"""Exact empty-space skipping: with skip_empty the forward render jumps over
bricks whose value range maps to zero-opacity table entries, and must give
bit for bit the image and sample counts of the plain march (skipped samples
add nothing and leave the transmittance unchanged); checked against the
oracle as well, on HI-like cubes where most bricks hold only noise."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import TOL_F32, compare, cuda_or_skip

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


@pytest.fixture(scope="module")
def P(torch):
    import paper_1211_4896_gb300 as P
    return P


def _threshold_table(K=64, v_on=6.0, vmin=-3.0, vmax=30.0, band=None):
    """Opacity 0 below v_on (and inside `band` if given), rising above."""
    v = vmin + (vmax - vmin) * np.arange(K) / (K - 1)
    t = (v - vmin) / (vmax - vmin)
    a = np.where(v < v_on, 0.0, 0.05 + 0.3 * (v - v_on) / (vmax - v_on))
    if band is not None:
        a = np.where((v > band[0]) & (v < band[1]), 0.0, a)
    return np.stack([t, t * t, 1 - t, a], axis=1).astype(np.float32)


CASES = [((64, 60, 72), 16, "f32", "persp", 2.0), ((80, 70, 66), 32, "f32", "ortho", 0.9),
         ((72, 72, 72), 16, "f16", "persp", 0.95), ((50, 45, 60), 64, "bf16", "persp", 2.0)]


@pytest.mark.parametrize("dims,brick,store,kind,ert", CASES)
def test_skip_is_bit_identical_and_matches_oracle(P, torch, dims, brick, store, kind, ert):
    cube = synth.hi_cube(dims, n_blobs=4, n_disks=1, seed=sum(dims)).numpy()
    t = torch.from_numpy(cube).cuda()
    vol = P.Volume(t, store, brick=brick)
    ref_cube = cube if store == "f32" else (t.half() if store == "f16" else t.bfloat16()).float().cpu().numpy()
    try:
        for tf_np in (_threshold_table(), _threshold_table(v_on=3.0, band=(8.0, 14.0))):
            tf = torch.from_numpy(tf_np).cuda()
            for view in range(3):
                cam = synth.camera_random_persp(dims, seed=13 * view + sum(dims), width=56, height=44,
                                                fov_y_deg=35.0)
                if kind == "ortho":
                    cam = dict(cam, kind=0, ortho_height=1.1 * max(dims), fov_y_deg=0.0)
                a, na = P.render(vol, cam, tf, -3.0, 30.0, 0.5, ert)
                b, nb = P.render(vol, cam, tf, -3.0, 30.0, 0.5, ert, skip_empty=True)
                assert torch.equal(a, b) and torch.equal(na, nb)
                if store == "f32" or view == 0:
                    compare(b.cpu().numpy(), nb.cpu().numpy(), oracle.render(ref_cube, cam, tf_np, -3.0, 30.0, 0.5,
                                                                             ert), TOL_F32)
        assert b[..., 3].max().item() > 0.05
    finally:
        vol.close()


def test_skip_with_null_voxels_and_after_update(P, torch):
    """Bricks holding NaN are never skipped (their samples take the table's
    low end); after vr_volume_update the brick ranges are rebuilt."""
    dims = (48, 40, 56)
    cube = synth.hi_cube(dims, n_blobs=3, n_disks=0, seed=4).numpy()
    cube[10:12, 5:9, 3:40] = np.nan
    vol = P.Volume(torch.from_numpy(cube).cuda(), "f32")
    tf_np = _threshold_table()
    tf_np[0, 3] = 0.2                                    # the low end (where NaN lands) is visible
    tf = torch.from_numpy(tf_np).cuda()
    try:
        cam = synth.camera_random_persp(dims, seed=3, width=48, height=40)
        a, na = P.render(vol, cam, tf, -3.0, 30.0, 0.5)
        b, nb = P.render(vol, cam, tf, -3.0, 30.0, 0.5, skip_empty=True)
        assert torch.equal(a, b) and torch.equal(na, nb)
        cube2 = np.ascontiguousarray(cube[::-1, ::-1, :]) * np.float32(2.0)
        vol.update(torch.from_numpy(cube2).cuda())
        a, na = P.render(vol, cam, tf, -3.0, 30.0, 0.5)
        b, nb = P.render(vol, cam, tf, -3.0, 30.0, 0.5, skip_empty=True)
        assert torch.equal(a, b) and torch.equal(na, nb)
        compare(b.cpu().numpy(), nb.cpu().numpy(), oracle.render(cube2, cam, tf_np, -3.0, 30.0, 0.5), TOL_F32)
    finally:
        vol.close()


def test_skip_only_on_the_composite_software_path(P, torch):
    from paper_1211_4896_gb300 import _lib as L
    vol = P.Volume(synth.hi_cube((20, 20, 20), 1, 0, 2).cuda(), "f32")
    tf = torch.from_numpy(_threshold_table(16)).cuda()
    cam = synth.camera_random_persp((20, 20, 20), seed=2, width=8, height=8)
    try:
        with pytest.raises(L.VRError) as e:
            P.render(vol, cam, tf, -3, 30, 1.0, mode=P.VR_MODE_MIP, skip_empty=True)
        assert e.value.status == L.VR_ERR_UNSUPPORTED
        with pytest.raises(L.VRError) as e:
            P.render(vol, cam, tf, -3, 30, 1.0, filter=L.VR_FILTER_SOFTWARE_STAGED, skip_empty=True)
        assert e.value.status == L.VR_ERR_UNSUPPORTED
    finally:
        vol.close()
