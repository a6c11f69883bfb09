"""Host-side fault injection: one of the library's device allocations is made
to fail (vr_debug_fail_alloc) and every entry point must report VR_ERR_OOM or
fall back as documented, leave its handle usable, and give the same results
once memory is available again.  Nothing on the device faults."""
import numpy as np
import pytest

import synth
from tests.helpers import cuda_or_skip

pytestmark = pytest.mark.gpu

DIMS = (30, 26, 34)


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


@pytest.fixture(scope="module")
def P(torch):
    import paper_1211_4896_gb300 as P
    return P


@pytest.fixture
def L(P):
    from paper_1211_4896_gb300 import _lib as L
    yield L
    L.vr_debug_fail_alloc(-1)


def _cam(forward, up, size=48):
    c = [0.5 * (d - 1) for d in DIMS]
    eye = [c[a] - 120.0 * forward[a] for a in range(3)]
    return synth.camera_persp(eye, forward, up, 25.0, size, size)


def _tf(torch):
    return torch.from_numpy(synth.tf_random_pwl(seed=8, alpha_max=0.3)).cuda()


def _cube(torch):
    return synth.hi_cube(DIMS, n_blobs=4, n_disks=1, seed=19).cuda()


def test_volume_create_reports_oom_and_recovers(P, torch, L):
    cube = _cube(torch)
    for after in (0, 1):                     # the bricks, then the work counters
        L.vr_debug_fail_alloc(after)
        with pytest.raises(L.VRError) as e:
            P.Volume(cube, "f32")
        assert e.value.status == L.VR_ERR_OOM
    vol = P.Volume(cube, "f32")
    vol.close()


def test_brick_copy_that_cannot_be_allocated_is_not_used(P, torch, L, monkeypatch):
    monkeypatch.setenv("VR_TEX_LAYERS", "0")          # the brick copies only
    vol = P.Volume(_cube(torch), "f32")
    tf = _tf(torch)
    cam = _cam((0, 0, 1), (1, 0, 0))         # image rows along +y: prefers the y-fastest copy
    try:
        L.vr_debug_fail_alloc(0)
        a, na = P.render(vol, cam, tf, -3.0, 30.0, 0.5)
        assert L.vr_volume_info(vol.handle)["copies"] == 0
        assert L.vr_view_layout(vol.handle, L.make_camera(cam)) == -1
        b, nb = P.render(vol, cam, tf, -3.0, 30.0, 0.5)   # now the copy is built and read
        assert L.vr_volume_info(vol.handle)["copies"] == 1 << 1
        assert torch.equal(a, b) and torch.equal(na, nb)
        assert a[..., 3].max().item() > 0.05
    finally:
        vol.close()


def test_texture_layers_that_cannot_be_allocated_are_not_used(P, torch, L):
    """The layered array's allocation fails: the view falls back to its brick
    copy (built by the same call); the next call builds the layers and reads
    them; the images agree bit for bit."""
    vol = P.Volume(_cube(torch), "f32")
    tf = _tf(torch)
    cam = _cam((0, 0, 1), (1, 0, 0))         # along z, rows along +y: layers across z, else the y-fastest copy
    try:
        L.vr_debug_fail_alloc(0)
        a, na = P.render(vol, cam, tf, -3.0, 30.0, 0.5)
        assert L.vr_volume_info(vol.handle)["copies"] == 1 << 1
        b, nb = P.render(vol, cam, tf, -3.0, 30.0, 0.5)
        assert L.vr_volume_info(vol.handle)["copies"] == (1 << 1) | (1 << 11)
        assert L.vr_view_layout(vol.handle, L.make_camera(cam)) == 11
        assert torch.equal(a, b) and torch.equal(na, nb)
        assert a[..., 3].max().item() > 0.05
    finally:
        vol.close()


def test_backward_without_quad_scratch_falls_back_to_direct(P, torch, L):
    vol = P.Volume(_cube(torch), "f32")
    tf = _tf(torch)
    cam = _cam((0, 0, 1), (0, 1, 0), size=64)     # dense rays: prefers the quad scratch
    nvox = int(np.prod(DIMS))
    try:
        img, ns = P.render(vol, cam, tf, -3.0, 30.0, 0.5)
        g = torch.randn(img.shape, device="cuda", generator=torch.Generator(device="cuda").manual_seed(3))
        ref_tf, ref_vox = P.render_backward(vol, cam, tf, -3.0, 30.0, 0.5, img, ns, g, vox_reduce="direct")
        rows = L.vr_volume_info(vol.handle)["scratch_bytes"]       # the table rows only
        L.vr_debug_fail_alloc(0)                 # the quad scratch
        got_tf, got_vox = P.render_backward(vol, cam, tf, -3.0, 30.0, 0.5, img, ns, g)
        torch.cuda.synchronize()
        assert L.vr_volume_info(vol.handle)["scratch_bytes"] == rows
        assert (got_vox - ref_vox).abs().max().item() <= 1e-4 * ref_vox.abs().max().item()
        assert (got_tf - ref_tf).abs().max().item() <= 1e-5 * ref_tf.abs().max().item()
        P.render_backward(vol, cam, tf, -3.0, 30.0, 0.5, img, ns, g)          # now it is allocated
        assert L.vr_volume_info(vol.handle)["scratch_bytes"] == rows + 16 * nvox
    finally:
        vol.close()


def test_scratch_allocations_report_oom_and_recover(P, torch, L):
    tf = _tf(torch)
    cam = _cam((0, 0, 1), (0, 1, 0))         # rows along -x: reads the bricks, no copy needed
    for what in ("table rows", "brick ranges", "statistics", "batch plan"):
        vol = P.Volume(_cube(torch), "f32")
        try:
            img, ns = P.render(vol, cam, tf, -3.0, 30.0, 0.5)
            g = torch.randn_like(img)
            job = [dict(vol=vol, cam=cam, tf=tf, vmin=-3.0, vmax=30.0, step=0.5, out=torch.empty_like(img))]
            calls = {"table rows": lambda: P.render_backward(vol, cam, tf, -3.0, 30.0, 0.5, img, ns, g,
                                                             vox_reduce="direct"),
                     "brick ranges": lambda: P.render(vol, cam, tf, -3.0, 30.0, 0.5, skip_empty=True),
                     "statistics": lambda: P.moments(vol),
                     "batch plan": lambda: P.render_batched(job, use_graph=False)}
            L.vr_debug_fail_alloc(0)
            with pytest.raises(L.VRError) as e:
                calls[what]()
            assert e.value.status == L.VR_ERR_OOM, what
            calls[what]()                                          # memory is back: it works
            torch.cuda.synchronize()
            L.vr_check(vol.handle, int(torch.cuda.current_stream().cuda_stream))
        finally:
            vol.close()
    # and the results are right after a failed first attempt
    vol = P.Volume(_cube(torch), "f32")
    try:
        a, na = P.render(vol, cam, tf, -3.0, 30.0, 0.5)
        L.vr_debug_fail_alloc(0)
        with pytest.raises(L.VRError):
            P.render(vol, cam, tf, -3.0, 30.0, 0.5, skip_empty=True)
        b, nb = P.render(vol, cam, tf, -3.0, 30.0, 0.5, skip_empty=True)
        assert torch.equal(a, b) and torch.equal(na, nb)
    finally:
        vol.close()
