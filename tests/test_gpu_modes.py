"""GPU parity of the paper's other uses of the ray against the FP64 oracle:
maximum intensity projection (Section 3.3.1), the sigma-clipping transfer
function with its statistical mini-map (Section 4.5) and the 3D spectrum
tool (Section 4.4), through the C ABI; plus the mode checks of the paths
that do not implement them."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import TOL_F32, TOL_HALF, compare, cuda_or_skip

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


@pytest.fixture(scope="module")
def P(torch):
    import paper_1211_4896_gb300 as P
    return P


def _with_margins(ref, cube, cam, step):
    """Adds the sample-count decision margins of the same rays (the plain
    oracle render reports them); these modes have no early termination."""
    r = oracle.render(cube, cam, [[0, 0, 0, 0], [0, 0, 0, 0]], 0.0, 1.0, step)
    out = dict(ref)
    out["margin_n"] = r["margin_n"]
    out["margin_ert"] = np.full(r["margin_n"].shape, np.inf)
    return out


CASES = [
    # dims, camera kind, W, H, step, brick
    ((23, 17, 29), "persp", 37, 29, 0.37, 16),
    ((40, 33, 35), "ortho", 45, 31, 0.5, 32),
    ((70, 66, 80), "persp", 64, 48, 1.0, 16),
]


def _cams(dims, kind, W, H, n=3):
    for view in range(n):
        cam = synth.camera_random_persp(dims, seed=100 * view + W, width=W, height=H, fov_y_deg=35.0)
        if kind == "ortho":
            cam = dict(cam, kind=0, ortho_height=1.1 * max(dims), fov_y_deg=0.0)
        yield cam


@pytest.mark.parametrize("dims,kind,W,H,step,brick", CASES)
def test_mip_matches_oracle(P, torch, dims, kind, W, H, step, brick):
    cube = synth.hi_cube(dims, n_blobs=6, n_disks=1, seed=sum(dims)).numpy()
    tf_np = synth.tf_random_pwl(seed=W * H, alpha_max=0.6)
    vol = P.Volume(torch.from_numpy(cube).cuda(), "f32", brick=brick)
    tf = torch.from_numpy(tf_np).cuda()
    bg = (0.05, 0.1, 0.2, 0.3)
    try:
        for cam in _cams(dims, kind, W, H):
            img, ns = P.render(vol, cam, tf, -3.0, 30.0, step, bg=bg, mode=P.VR_MODE_MIP)
            ref = oracle.render_mip(cube, cam, tf_np, -3.0, 30.0, step, bg=bg)
            compare(img.cpu().numpy(), ns.cpu().numpy(), _with_margins(ref, cube, cam, step), TOL_F32)
            assert (ref["n_used"] > 0).any()
    finally:
        vol.close()


@pytest.mark.parametrize("store", ["f16", "bf16"])
def test_mip_half_storage_on_the_rounded_cube(P, torch, store):
    """16-bit storage: against the oracle on the stored (rounded) values at
    the float32 tolerance, and on the float32 cube within 2e-3."""
    dims = (33, 41, 27)
    cube = synth.hi_cube(dims, n_blobs=5, n_disks=1, seed=7).numpy()
    t = torch.from_numpy(cube).cuda()
    rounded = (t.half() if store == "f16" else t.bfloat16()).float().cpu().numpy()
    tf_np = synth.tf_random_pwl(seed=5, alpha_max=0.5)
    vol = P.Volume(t, store)
    tf = torch.from_numpy(tf_np).cuda()
    try:
        cam = next(_cams(dims, "persp", 40, 36, 1))
        img, ns = P.render(vol, cam, tf, -3.0, 30.0, 0.6, mode=P.VR_MODE_MIP)
        img, ns = img.cpu().numpy(), ns.cpu().numpy()
        compare(img, ns, _with_margins(oracle.render_mip(rounded, cam, tf_np, -3.0, 30.0, 0.6), rounded, cam, 0.6),
                TOL_F32)
        compare(img, ns, _with_margins(oracle.render_mip(cube, cam, tf_np, -3.0, 30.0, 0.6), cube, cam, 0.6),
                TOL_HALF)
    finally:
        vol.close()


def test_mip_rolled_view_reads_a_copy_bit_identically(P, torch, monkeypatch):
    """A view and its 90-degree roll about the view axis (square image, eye on
    the axis) read different brick layouts and give transposed images (the
    brick copies: texture layers off)."""
    monkeypatch.setenv("VR_TEX_LAYERS", "0")
    dims = (40, 36, 44)
    cube = synth.hi_cube(dims, n_blobs=8, n_disks=1, seed=7).numpy()
    vol = P.Volume(torch.from_numpy(cube).cuda(), "f32")
    tf = torch.from_numpy(synth.tf_random_pwl(seed=3, alpha_max=0.5)).cuda()
    n = 48
    c = [0.5 * (d - 1) for d in dims]
    eye = (c[0], c[1], c[2] - 180.0)
    try:
        a, na = P.render(vol, synth.camera_persp(eye, (0, 0, 1), (0, 1, 0), 20.0, n, n), tf, -3, 30, 0.5,
                         mode=P.VR_MODE_MIP)
        b, nb = P.render(vol, synth.camera_persp(eye, (0, 0, 1), (1, 0, 0), 20.0, n, n), tf, -3, 30, 0.5,
                         mode=P.VR_MODE_MIP)
        assert P._lib.vr_volume_info(vol.handle)["copies"] == 0b10
        i, j = np.arange(n)[None, :], np.arange(n)[:, None]
        assert np.array_equal(b.cpu().numpy(), a.cpu().numpy()[n - 1 - i, j])
        assert np.array_equal(nb.cpu().numpy(), na.cpu().numpy()[n - 1 - i, j])
        # MIP and sigma clipping through the texture layers (across z for both
        # views): the images of the bricks, bit for bit
        mm = P.minimap(vol, (8, 8, 8))
        for up in ((0, 1, 0), (1, 0, 0)):
            cam = synth.camera_persp(eye, (0, 0, 1), up, 20.0, n, n)
            for kw in (dict(mode=P.VR_MODE_MIP), dict(mode=P.VR_MODE_SIGMA, minimap=mm, region=(8, 8, 8))):
                monkeypatch.setenv("VR_TEX_LAYERS", "0")
                ref, rn = P.render(vol, cam, tf, -3, 30, 0.5, **kw)
                monkeypatch.delenv("VR_TEX_LAYERS")
                got, gn = P.render(vol, cam, tf, -3, 30, 0.5, **kw)
                torch.cuda.synchronize()
                assert torch.equal(got, ref) and torch.equal(gn, rn)
        assert P._lib.vr_volume_info(vol.handle)["copies"] >> 9 == 0b100
    finally:
        vol.close()


@pytest.mark.parametrize("store", ["f32", "f16"])
def test_minimap_matches_oracle(P, torch, store):
    """Region means and standard deviations (FP64 sums on the GPU, rounded to
    float32) against the oracle's, with short last regions on every axis."""
    dims = (37, 29, 41)
    cube = synth.hi_cube(dims, n_blobs=6, n_disks=1, seed=21).numpy()
    t = torch.from_numpy(cube).cuda()
    stored = t if store == "f32" else t.half().float()
    vol = P.Volume(t, store)
    try:
        for region in ((8, 8, 8), (5, 7, 16), (37, 29, 41), (1, 29, 3)):
            got = P.minimap(vol, region).cpu().numpy().astype(np.float64)
            ref = oracle.minimap(stored.cpu().numpy(), region)
            assert got.shape == ref.shape
            np.testing.assert_allclose(got, ref, rtol=2e-7, atol=1e-6)
    finally:
        vol.close()


@pytest.mark.parametrize("dims,kind,W,H,step,brick", CASES)
def test_sigma_clipping_matches_oracle(P, torch, dims, kind, W, H, step, brick):
    """The sigma-clipped render with the GPU's mini-map against the oracle's
    render with its own FP64 mini-map; table range [-1, 6] sigma."""
    cube = synth.hi_cube(dims, n_blobs=6, n_disks=1, seed=sum(dims)).numpy()
    cube[:, :, dims[0] // 2:] = 3.0 * cube[:, :, dims[0] // 2:] + 5.0      # a louder, offset half
    tf_np = synth.tf_random_pwl(seed=W + H, alpha_max=0.4)
    vol = P.Volume(torch.from_numpy(cube).cuda(), "f32", brick=brick)
    tf = torch.from_numpy(tf_np).cuda()
    region = (11, 8, 13)
    try:
        mm = P.minimap(vol, region)
        stats = oracle.minimap(cube, region)
        for cam in _cams(dims, kind, W, H):
            img, ns = P.render(vol, cam, tf, -1.0, 6.0, step, mode=P.VR_MODE_SIGMA, minimap=mm, region=region)
            ref = oracle.render_sigma(cube, cam, tf_np, -1.0, 6.0, step, stats, region)
            compare(img.cpu().numpy(), ns.cpu().numpy(), _with_margins(ref, cube, cam, step), TOL_F32)
            assert ref["rgba"][..., 3].max() > 0.05
    finally:
        vol.close()


def test_sigma_with_one_region_equals_rescaled_composite(P, torch):
    """One region: the sigma render equals the composite render over
    [mu + vmin sd, mu + vmax sd] up to FP32 rounding of the rescale."""
    dims = (30, 26, 34)
    cube = synth.hi_cube(dims, n_blobs=5, n_disks=1, seed=31).numpy()
    vol = P.Volume(torch.from_numpy(cube).cuda(), "f32")
    tf_np = synth.tf_random_pwl(seed=9, alpha_max=0.3)
    tf = torch.from_numpy(tf_np).cuda()
    try:
        mm = P.minimap(vol, dims)
        mu, sd = (float(x) for x in mm.cpu().numpy().reshape(2))
        cam = next(_cams(dims, "persp", 32, 30, 1))
        a, na = P.render(vol, cam, tf, -1.0, 4.0, 0.5, 0.95, mode=P.VR_MODE_SIGMA, minimap=mm, region=dims)
        b, nb = P.render(vol, cam, tf, mu - sd, mu + 4.0 * sd, 0.5, 0.95)
        assert np.abs(a.cpu().numpy() - b.cpu().numpy()).max() <= 1e-4
    finally:
        vol.close()


@pytest.mark.parametrize("store", ["f32", "bf16"])
def test_profile_matches_oracle(P, torch, store):
    """3D spectrum tool: every sample value of several rays (axis-parallel,
    oblique, perspective), including a truncated read and a miss."""
    dims = (45, 38, 52)
    cube = synth.hi_cube(dims, n_blobs=6, n_disks=2, seed=41).numpy()
    t = torch.from_numpy(cube).cuda()
    stored = (t if store == "f32" else t.bfloat16().float()).cpu().numpy()
    vol = P.Volume(t, store)
    try:
        cams = [synth.camera_ortho((22.0, 18.5, -30.0), (0, 0, 1), (0, 1, 0), 40.0, 24, 20)]
        cams += list(_cams(dims, "persp", 31, 27, 2))
        for cam in cams:
            for (i, j) in ((0, 0), (cam["width"] // 2, cam["height"] // 2), (cam["width"] - 3, 4)):
                got = P.profile(vol, cam, 0.45, i, j).cpu().numpy().astype(np.float64)
                ref = oracle.profile(stored, cam, 0.45, i, j)
                n_ray, *_ = oracle.ray(dims[::-1], cam, 0.45, i, j)
                if got.shape != ref.shape:          # only on a sample-count tie
                    assert abs(got.size - ref.size) == 1
                    m = min(got.size, ref.size)
                    got, ref = got[:m], ref[:m]
                np.testing.assert_allclose(got, ref, atol=2e-5 * max(1.0, np.abs(ref).max(initial=0.0)))
        cam = cams[1]
        full = P.profile(vol, cam, 0.45, 15, 13).cpu().numpy()
        part = P.profile(vol, cam, 0.45, 15, 13, max_values=7).cpu().numpy()
        assert part.size == min(7, full.size) and np.array_equal(part, full[:part.size])
        miss = synth.camera_ortho((500.0, 500.0, -30.0), (0, 0, 1), (0, 1, 0), 4.0, 4, 4)
        assert P.profile(vol, miss, 0.45, 1, 1).numel() == 0
    finally:
        vol.close()


def test_modes_checked_on_paths_without_them(P, torch):
    """Sigma clipping without a mini-map is an invalid argument; the backward,
    the batched call and the texture filter refuse MIP (unsupported)."""
    from paper_1211_4896_gb300 import _lib as L
    dims = (20, 20, 20)
    vol = P.Volume(synth.hi_cube(dims, 2, 0, 3).cuda(), "f32")
    tf = torch.from_numpy(synth.tf_ramp(16)).cuda()
    cam = next(_cams(dims, "persp", 16, 16, 1))
    out = torch.empty((16, 16, 4), device="cuda")
    ns = torch.empty((16, 16), device="cuda", dtype=torch.int32)
    s = int(torch.cuda.current_stream().cuda_stream)
    try:
        with pytest.raises(L.VRError) as e:
            L.vr_render(vol.handle, L.make_camera(cam), L.make_params(tf.data_ptr(), 16, -3, 50, 1.0, mode=L.VR_MODE_SIGMA),
                        out.data_ptr(), ns.data_ptr(), s)
        assert e.value.status == L.VR_ERR_INVALID_ARG
        mip = L.make_params(tf.data_ptr(), 16, -3, 50, 1.0, mode=L.VR_MODE_MIP)
        L.vr_render(vol.handle, L.make_camera(cam), mip, out.data_ptr(), ns.data_ptr(), s)
        gtf = torch.empty((16, 4), device="cuda", dtype=torch.float64)
        with pytest.raises(L.VRError) as e:
            L.vr_render_backward(vol.handle, L.make_camera(cam), mip, out.data_ptr(), ns.data_ptr(), out.data_ptr(),
                                 gtf.data_ptr(), None, 0, s)
        assert e.value.status == L.VR_ERR_UNSUPPORTED
        with pytest.raises(L.VRError) as e:
            L.vr_render_batched([L.vr_job(vol.handle, L.make_camera(cam), mip, out.data_ptr(), ns.data_ptr())],
                                L.vr_batch_opts(0, 8, 4, 0), s)
        assert e.value.status == L.VR_ERR_UNSUPPORTED
        tex = L.make_params(tf.data_ptr(), 16, -3, 50, 1.0, filter=L.VR_FILTER_TEXTURE, mode=L.VR_MODE_MIP)
        with pytest.raises(L.VRError) as e:
            L.vr_render(vol.handle, L.make_camera(cam), tex, out.data_ptr(), ns.data_ptr(), s)
        assert e.value.status == L.VR_ERR_UNSUPPORTED
    finally:
        torch.cuda.synchronize()
        vol.close()
