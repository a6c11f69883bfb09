"""Texture-layer copies of a float volume (the paper keeps its sub-cubes in
texture memory, Section 4.3): a dense view reads a 2D layered texture whose
layers cross the axis its rays run along most, gathering a cell's corners
with the texture unit's four-texel gather at the cell's exact integer corner
and interpolating them in software.  The values are the stored voxels, so
every result must equal the brick path's bit for bit (VR_TEX_LAYERS=0 turns
the layers off; the library reads it at each call): forward, batched and
allocation-free batched renders, and, up to FP32 summation order, the
backward.  Also covered: the copy bookkeeping, a voxel update, 16-bit
storage (no layers), a volume whose layer count exceeds the device limit
(falls back to the bricks), and the oracle."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import TOL_F32, compare, cuda_or_skip

pytestmark = pytest.mark.gpu

DIMS = (41, 37, 45)
VMIN, VMAX, STEP = -3.0, 30.0, 0.5


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


@pytest.fixture(scope="module")
def P(torch):
    import paper_1211_4896_gb300 as P
    return P


@pytest.fixture(scope="module")
def scene():
    cube = synth.hi_cube(DIMS, n_blobs=8, n_disks=1, seed=23).numpy()
    tf = synth.tf_random_pwl(seed=5, alpha_max=0.3)
    return cube, tf


def _cams(dims=DIMS):
    """Dense views (about one voxel per pixel) along each axis, both signs,
    oblique ones, ortho and perspective, ragged image sizes."""
    c = [0.5 * (d - 1) for d in dims]
    out = []
    dirs = [((0, 0, 1), (0, 1, 0)), ((0, 0, -1), (1, 0, 0)), ((1, 0, 0), (0, 1, 0)), ((-1, 0, 0), (0, 0, 1)),
            ((0, 1, 0), (0, 0, 1)), ((0, -1, 0), (1, 0, 0)), ((0.6, 0.2, 0.77), (0, 1, 0)),
            ((0.7, -0.5, 0.3), (0, 0, 1))]
    sizes = [(48, 40), (37, 29), (45, 51), (33, 33)]
    for q, (f, up) in enumerate(dirs):
        f = np.array(f, dtype=float) / np.linalg.norm(f)
        eye = [c[a] - 150.0 * f[a] for a in range(3)]
        W, H = sizes[q % len(sizes)]
        if q % 2:
            out.append(synth.camera_ortho(eye, tuple(f), up, 46.0, W, H))
        else:
            out.append(synth.camera_persp(eye, tuple(f), up, 18.0, W, H))
    return out


def _axis(cam):
    f = np.abs(np.asarray(cam["forward"], dtype=float))
    return int(np.argmax(f))


def _render(P, vol, cam, tf):
    return P.render(vol, cam, tf, VMIN, VMAX, STEP)


def test_forward_reads_layers_bit_identically(P, torch, scene, monkeypatch):
    cube, tf_np = scene
    from paper_1211_4896_gb300 import _lib as L
    vol = P.Volume(torch.from_numpy(cube).cuda(), "f32")
    tf = torch.from_numpy(tf_np).cuda()
    try:
        cams = _cams()
        monkeypatch.setenv("VR_TEX_LAYERS", "0")
        ref = [_render(P, vol, c, tf) for c in cams]
        assert L.vr_volume_info(vol.handle)["copies"] >> 9 == 0
        monkeypatch.delenv("VR_TEX_LAYERS")
        for c, (img0, ns0) in zip(cams, ref):
            img, ns = _render(P, vol, c, tf)
            torch.cuda.synchronize()
            assert L.vr_view_layout(vol.handle, L.make_camera(c)) == 9 + _axis(c)
            assert torch.equal(img, img0) and torch.equal(ns, ns0)
        info = L.vr_volume_info(vol.handle)
        assert info["copies"] >> 9 == 0b111
        assert info["copy_bytes"] >= 3 * 4 * int(np.prod(DIMS))
        for c, (img, ns) in list(zip(cams, ref))[:3]:
            compare(img.cpu().numpy(), ns.cpu().numpy(), oracle.render(cube, c, tf_np, VMIN, VMAX, STEP), TOL_F32)
        assert ref[0][0][..., 3].max().item() > 0.1
    finally:
        vol.close()


def test_batched_and_noalloc_read_layers(P, torch, scene):
    """One batch over views of every layer axis (one launch per layer copy)
    equals the single renders, replayed as a graph; the allocation-free batch
    reads the layers once they exist."""
    cube, tf_np = scene
    from paper_1211_4896_gb300 import _lib as L
    vol = P.Volume(torch.from_numpy(cube).cuda(), "f32")
    tf = torch.from_numpy(tf_np).cuda()
    try:
        cams = _cams()
        singles = [_render(P, vol, c, tf) for c in cams]
        jobs = [dict(vol=vol, cam=c, tf=tf, vmin=VMIN, vmax=VMAX, step=STEP,
                     out=torch.empty((c["height"], c["width"], 4), device="cuda"),
                     nsamples=torch.empty((c["height"], c["width"]), device="cuda", dtype=torch.int32))
                for c in cams]
        for _ in range(2):
            for j in jobs:
                j["out"].fill_(-1.0)
                j["nsamples"].fill_(-1)
            P.render_batched(jobs, use_graph=True)
            torch.cuda.synchronize()
            for j, (img, ns) in zip(jobs, singles):
                assert torch.equal(j["out"], img) and torch.equal(j["nsamples"], ns)
        s = int(torch.cuda.current_stream().cuda_stream)
        for c, (img, ns) in zip(cams, singles):
            out = torch.full_like(img, -1.0)
            n = torch.full_like(ns, -1)
            job = L.vr_job(vol.handle, L.make_camera(c), L.make_params(tf.data_ptr(), tf.shape[0], VMIN, VMAX, STEP,
                                                                        2.0), out.data_ptr(), n.data_ptr())
            L.vr_render_batched_noalloc([job], 8, 4, s)
            torch.cuda.synchronize()
            assert torch.equal(out, img) and torch.equal(n, ns)
    finally:
        vol.close()


def test_backward_reads_layers(P, torch, scene, monkeypatch):
    """Table and voxel gradients through the layers equal those through the
    bricks up to FP32 summation order, per view and in one multi-view call;
    the layer copy serves the backward of a view the forward never saw."""
    cube, tf_np = scene
    from paper_1211_4896_gb300 import _lib as L
    vol = P.Volume(torch.from_numpy(cube).cuda(), "f32")
    tf = torch.from_numpy(tf_np).cuda()
    try:
        cams = _cams()[:6]
        imgs, nss, gs = [], [], []
        monkeypatch.setenv("VR_TEX_LAYERS", "0")
        for q, c in enumerate(cams):
            img, ns = _render(P, vol, c, tf)
            imgs.append(img)
            nss.append(ns)
            gs.append(torch.randn(img.shape, device="cuda", generator=torch.Generator(device="cuda").manual_seed(q)))
        ref = [P.render_backward(vol, c, tf, VMIN, VMAX, STEP, i, n, g) for c, i, n, g in zip(cams, imgs, nss, gs)]
        ref_all = P.render_backward_views(vol, cams, tf, VMIN, VMAX, STEP, imgs, nss, gs)
        torch.cuda.synchronize()
        assert L.vr_volume_info(vol.handle)["copies"] >> 9 == 0
        monkeypatch.delenv("VR_TEX_LAYERS")
        got = [P.render_backward(vol, c, tf, VMIN, VMAX, STEP, i, n, g) for c, i, n, g in zip(cams, imgs, nss, gs)]
        got_all = P.render_backward_views(vol, cams, tf, VMIN, VMAX, STEP, imgs, nss, gs)
        torch.cuda.synchronize()
        assert L.vr_volume_info(vol.handle)["copies"] >> 9 == 0b111
        for (rt, rv), (gt, gv) in list(zip(ref, got)) + [(ref_all, got_all)]:
            assert (gt - rt).abs().max().item() <= 1e-5 * rt.abs().max().item()
            assert (gv - rv).abs().max().item() <= 1e-5 * rv.abs().max().item()
            assert rv.abs().max().item() > 0
    finally:
        vol.close()


def test_update_refreshes_layers(P, torch, scene):
    cube, tf_np = scene
    vol = P.Volume(torch.from_numpy(cube).cuda(), "f32")
    tf = torch.from_numpy(tf_np).cuda()
    try:
        cams = _cams()[:3]
        for c in cams:
            _render(P, vol, c, tf)
        cube2 = np.ascontiguousarray(cube[::-1, ::-1, :]) * np.float32(1.2)
        vol.update(torch.from_numpy(cube2).cuda())
        for c in cams:
            img, ns = _render(P, vol, c, tf)
            compare(img.cpu().numpy(), ns.cpu().numpy(), oracle.render(cube2, c, tf_np, VMIN, VMAX, STEP), TOL_F32)
    finally:
        vol.close()


@pytest.mark.parametrize("store", ["f16", "bf16"])
def test_half_storage_reads_no_layers(P, torch, scene, store):
    cube, tf_np = scene
    from paper_1211_4896_gb300 import _lib as L
    vol = P.Volume(torch.from_numpy(cube).cuda(), store)
    tf = torch.from_numpy(tf_np).cuda()
    try:
        for c in _cams()[:3]:
            _render(P, vol, c, tf)
        assert L.vr_volume_info(vol.handle)["copies"] >> 9 == 0
    finally:
        vol.close()


def test_layer_count_beyond_the_limit_falls_back(P, torch, monkeypatch):
    """A 12 x 10 x 4100 volume viewed along z would need 4100 layers (above
    the usual 2048-layer limit of 2D layered textures): the view reads the
    bricks, with the same result as with the layers turned off."""
    dims = (12, 10, 4100)
    cube = synth.hi_cube(dims, n_blobs=6, n_disks=0, seed=2).numpy()
    tf = torch.from_numpy(synth.tf_random_pwl(seed=5, alpha_max=0.05)).cuda()
    vol = P.Volume(torch.from_numpy(cube).cuda(), "f32")
    c = [0.5 * (d - 1) for d in dims]
    cam = synth.camera_ortho((c[0], c[1], -50.0), (0, 0, 1), (0, 1, 0), 13.0, 16, 16)
    try:
        a, na = _render(P, vol, cam, tf)
        monkeypatch.setenv("VR_TEX_LAYERS", "0")
        b, nb = _render(P, vol, cam, tf)
        torch.cuda.synchronize()
        assert torch.equal(a, b) and torch.equal(na, nb)
        assert int(na.sum()) > 0
    finally:
        vol.close()
