"""Sort-last rendering on the GPU (Sections 3.2 and 3.4): sub-box partial
images against the oracle's, and their depth-ordered composite against the
whole render (GPU and oracle), through the C ABI."""
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


def _boxes(cells, splits):
    edges = [np.linspace(0, n, s + 1).round().astype(int) for n, s in zip(cells, splits)]
    for i in range(splits[0]):
        for j in range(splits[1]):
            for k in range(splits[2]):
                yield ((int(edges[0][i]), int(edges[1][j]), int(edges[2][k])),
                       (int(edges[0][i + 1]), int(edges[1][j + 1]), int(edges[2][k + 1])))


CASES = [((33, 29, 41), "persp", 40, 34, 0.45, (2, 2, 2), 16, "f32"),
         ((48, 40, 36), "ortho", 36, 30, 0.6, (3, 1, 2), 32, "f32"),
         ((40, 36, 44), "persp", 32, 32, 0.5, (1, 4, 1), 16, "f16")]


@pytest.mark.parametrize("dims,kind,W,H,step,splits,brick,store", CASES)
def test_subboxes_composite_to_the_whole_render(P, torch, dims, kind, W, H, step, splits, brick, store):
    cube = synth.hi_cube(dims, n_blobs=6, n_disks=1, seed=sum(dims)).numpy()
    t = torch.from_numpy(cube).cuda()
    ref_cube = cube if store == "f32" else t.half().float().cpu().numpy()
    tf_np = synth.tf_random_pwl(seed=W * H, alpha_max=0.3)
    vol = P.Volume(t, store, brick=brick)
    tf = torch.from_numpy(tf_np).cuda()
    bg = (0.05, 0.1, 0.0, 0.2)
    cells = [d - 1 for d in dims]
    try:
        for view in range(2):
            cam = synth.camera_random_persp(dims, seed=31 * view + W, width=W, height=H, fov_y_deg=35.0)
            if kind == "ortho":
                cam = dict(cam, kind=0, ortho_height=1.1 * max(dims), fov_y_deg=0.0)
            whole, ns = P.render(vol, cam, tf, -3.0, 30.0, step, 2.0, bg=bg)
            parts, depths, counts = [], [], []
            for lo, hi in _boxes(cells, splits):
                part, depth, count = P.render_subbox(vol, cam, tf, -3.0, 30.0, step, lo, hi)
                parts.append(part)
                depths.append(depth)
                counts.append(count)
                ref = oracle.render_subbox(ref_cube, cam, tf_np, -3.0, 30.0, step, lo, hi)
                same = count.cpu().numpy() == ref["count"]
                assert same.mean() >= 0.995            # only samples on a cell boundary may move
                g = part.cpu().numpy().astype(np.float64)
                assert np.abs(g - ref["partial"])[same].max() <= TOL_F32
                d = depth.cpu().numpy().astype(np.float64)
                hit = same & (ref["count"] > 0)
                assert np.allclose(d[hit], ref["depth"][hit], rtol=1e-5, atol=1e-4)
                assert np.isinf(d[same & (ref["count"] == 0)]).all()
            # every sample lands in exactly one sub-box
            assert torch.equal(sum(counts), ns)
            got = P.composite(parts, depths, bg=bg)
            assert (got - whole).abs().max().item() <= 2e-6
            ref = oracle.render(ref_cube, cam, tf_np, -3.0, 30.0, step, 2.0, bg)
            compare(got.cpu().numpy(), ns.cpu().numpy(), ref, TOL_F32)
            assert ref["rgba"][..., 3].max() > 0.1
    finally:
        vol.close()


def test_composite_follows_depth_and_checks_arguments(P, torch):
    from paper_1211_4896_gb300 import _lib as L
    p1 = torch.tensor([[[0.5, 0.0, 0.0, 0.5]]], device="cuda")
    p2 = torch.tensor([[[0.0, 0.4, 0.0, 0.2]]], device="cuda")
    d1 = torch.tensor([[1.0]], device="cuda")
    d2 = torch.tensor([[2.0]], device="cuda")
    a = P.composite([p1, p2], [d1, d2]).cpu().numpy()[0, 0]
    b = P.composite([p1, p2], [d2, d1]).cpu().numpy()[0, 0]
    np.testing.assert_allclose(a, [0.5, 0.2, 0.0, 0.9], atol=1e-7)
    np.testing.assert_allclose(b, [0.1, 0.4, 0.0, 0.9], atol=1e-7)
    out = torch.empty((1, 1, 4), device="cuda")
    with pytest.raises(L.VRError) as e:
        L.vr_composite([], [], 1, 1, (0, 0, 0, 0), out.data_ptr())
    assert e.value.status == L.VR_ERR_INVALID_ARG
    vol = P.Volume(synth.hi_cube((12, 12, 12), 1, 0, 1).cuda(), "f32")
    tf = torch.from_numpy(synth.tf_ramp(8)).cuda()
    cam = synth.camera_random_persp((12, 12, 12), seed=1, width=8, height=8)
    try:
        with pytest.raises(L.VRError) as e:
            P.render_subbox(vol, cam, tf, -3, 50, 1.0, (3, 0, 0), (3, 11, 11))          # empty range
        assert e.value.status == L.VR_ERR_INVALID_ARG
        with pytest.raises(L.VRError) as e:
            P.render_subbox(vol, cam, tf, -3, 50, 1.0, (0, 0, 0), (12, 11, 11))         # beyond the 11 cells
        assert e.value.status == L.VR_ERR_INVALID_ARG
    finally:
        vol.close()


@pytest.mark.parametrize("store,parts,kind", [("f32", 2, "persp"), ("f32", 6, "ortho"), ("f16", 4, "persp")])
def test_sub_cube_volumes_give_the_whole_volume_partials(P, torch, store, parts, kind):
    """Object-space split as across GPUs (Section 3.2): each box of cells
    rendered from a volume holding only its sub-cube (voxels [lo, hi], origin
    at lo) with the whole grid's placement gives bit for bit the partial,
    depth and count of the same box rendered from the whole volume, and the
    depth-ordered composite of the pieces equals the whole render."""
    from paper_1211_4896_gb300.sortlast import split_cells, sub_cube
    dims = (45, 38, 52)
    cube = synth.hi_cube(dims, n_blobs=6, n_disks=1, seed=77).cuda()
    whole_vol = P.Volume(cube, store)
    tf_np = synth.tf_random_pwl(seed=12, alpha_max=0.3)
    tf = torch.from_numpy(tf_np).cuda()
    cam = synth.camera_random_persp(dims, seed=parts, width=44, height=36, fov_y_deg=35.0)
    if kind == "ortho":
        cam = dict(cam, kind=0, ortho_height=1.1 * max(dims), fov_y_deg=0.0)
    bg = (0.0, 0.05, 0.1, 0.2)
    vols = []
    try:
        whole, ns = P.render(whole_vol, cam, tf, -3.0, 30.0, 0.55, 2.0, bg=bg)
        pieces, depths, counts = [], [], []
        for lo, hi in split_cells([d - 1 for d in dims], parts):
            vol = P.Volume(sub_cube(cube, lo, hi), store, origin=tuple(float(x) for x in lo))
            vols.append(vol)
            part, depth, count = P.render_subbox(vol, cam, tf, -3.0, 30.0, 0.55, lo, hi, global_dims=dims, offset=lo)
            ref_p, ref_d, ref_c = P.render_subbox(whole_vol, cam, tf, -3.0, 30.0, 0.55, lo, hi)
            assert torch.equal(part, ref_p) and torch.equal(depth, ref_d) and torch.equal(count, ref_c)
            pieces.append(part)
            depths.append(depth)
            counts.append(count)
        assert torch.equal(sum(counts), ns)
        got = P.composite(pieces, depths, bg=bg)
        assert (got - whole).abs().max().item() <= 2e-6
        assert whole[..., 3].max().item() > 0.1
        from paper_1211_4896_gb300 import _lib as L
        with pytest.raises(L.VRError) as e:       # a box beyond the sub-cube's voxels
            P.render_subbox(vols[0], cam, tf, -3.0, 30.0, 0.55, (0, 0, 0), tuple(d - 1 for d in dims),
                            global_dims=dims, offset=(0, 0, 0))
        assert e.value.status == L.VR_ERR_INVALID_ARG
    finally:
        for v in vols:
            v.close()
        whole_vol.close()
