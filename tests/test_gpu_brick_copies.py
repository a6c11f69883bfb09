"""Brick copies.  A software-filter view whose image rows run closest to the
y (z) axis reads a copy of the bricks stored with that axis fastest, so that
the rays of one warp read neighbouring elements; for 16-bit storage the copy
is paired (each element holds its own value and the next one along that
axis, four loads per cell) and exists for the x axis too.  The arithmetic of
a sample does not depend on where its corners are stored, so a view and the
same view rolled by 90 degrees about its forward axis (same rays, image
transposed; square image, the eye on the axis) agree bit for bit although
they read different layouts; so do a render from the bricks themselves and
one from a copy.  Views whose rays are far apart read blocked copies
(2 x 2 x BW blocks of one sector, deep along the rays' main axis).  Covered:
single renders, one batch reading every layout, the allocation-free batch,
the backward, and a voxel update that must refresh the copies.  Both views
are also checked against the oracle."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import TOL_F32, compare, cuda_or_skip

pytestmark = pytest.mark.gpu

DIMS = (40, 36, 44)
W = 48
VMIN, VMAX, STEP = -3.0, 30.0, 0.5


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


@pytest.fixture(autouse=True)
def _brick_copies_only(monkeypatch):
    """Dense float views would read texture-layer copies
    (tests/test_gpu_tex_layers.py); these tests are about the brick copies."""
    monkeypatch.setenv("VR_TEX_LAYERS", "0")


@pytest.fixture(scope="module")
def P(torch):
    import paper_1211_4896_gb300 as P
    return P


def _cam(forward, up, kind, size=W):
    c = [0.5 * (d - 1) for d in DIMS]
    eye = [c[a] - 180.0 * forward[a] for a in range(3)]
    if kind == "ortho":
        return synth.camera_ortho(eye, forward, up, 50.0, size, size)
    return synth.camera_persp(eye, forward, up, 20.0, size, size)


# (camera reading x-fastest bricks, its roll reading order `order`, map from
#  the x-order image to the rolled one: rolled[j, i] = base[rows, cols])
_I = np.arange(W)[None, :]
_J = np.arange(W)[:, None]
PAIRS = [
    # forward +z: up +y gives rows along -x; up +x gives rows along +y
    (((0, 0, 1), (0, 1, 0)), ((0, 0, 1), (1, 0, 0)), 1, (W - 1 - _I, _J)),
    # forward +y: up +z gives rows along +x; up +x gives rows along -z
    (((0, 1, 0), (0, 0, 1)), ((0, 1, 0), (1, 0, 0)), 2, (_I, W - 1 - _J)),
]


@pytest.fixture(scope="module")
def scene():
    cube = synth.hi_cube(DIMS, n_blobs=8, n_disks=1, seed=7).numpy()
    tf = synth.tf_random_pwl(seed=3, alpha_max=0.3)
    return cube, tf


def _volume(P, torch, cube, store="f32"):
    return P.Volume(torch.from_numpy(np.ascontiguousarray(cube)).cuda(), store)


def _noalloc(P, torch, vol, cam, tf):
    """Render through the allocation-free batch (reads whatever copy exists)."""
    from paper_1211_4896_gb300 import _lib as L
    out = torch.full((W, W, 4), -1.0, device="cuda")
    ns = torch.full((W, W), -1, device="cuda", dtype=torch.int32)
    job = L.vr_job(vol.handle, L.make_camera(cam), L.make_params(tf.data_ptr(), tf.shape[0], VMIN, VMAX, STEP, 2.0),
                   out.data_ptr(), ns.data_ptr())
    L.vr_render_batched_noalloc([job], 8, 4, int(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return out, ns


def _copies(P, vol):
    return P._lib.vr_volume_info(vol.handle)["copies"]


@pytest.mark.parametrize("store", ["f32", "f16"])
@pytest.mark.parametrize("kind", ["ortho", "persp"])
@pytest.mark.parametrize("pair", range(len(PAIRS)))
def test_rolled_view_reads_a_copy_bit_identically(P, torch, scene, kind, pair, store):
    cube, tf_np = scene
    (fa, ua), (fb, ub), order, (rows, cols) = PAIRS[pair]
    vol = _volume(P, torch, cube, store)
    tf = torch.from_numpy(tf_np).cuda()
    # copy ids: 1, 2 plain y / z; 3, 4, 5 paired x / y / z (16-bit, dense rays: ~1 voxel per pixel here)
    x_copy = 0 if store == "f32" else 1 << 3
    b_copy = 1 << order if store == "f32" else 1 << (3 + order)
    try:
        assert _copies(P, vol) == 0
        camA, camB = _cam(fa, ua, kind), _cam(fb, ub, kind)
        L = P._lib
        layout = lambda cam: L.vr_view_layout(vol.handle, L.make_camera(cam))   # noqa: E731
        assert layout(camA) == -1 and layout(camB) == -1          # nothing built yet
        a, na = P.render(vol, camA, tf, VMIN, VMAX, STEP)
        assert _copies(P, vol) == x_copy
        assert layout(camA) == (-1 if store == "f32" else 3)
        b, nb = P.render(vol, camB, tf, VMIN, VMAX, STEP)
        torch.cuda.synchronize()
        assert layout(camB) == (order if store == "f32" else 3 + order)
        info = P._lib.vr_volume_info(vol.handle)
        assert info["copies"] == x_copy | b_copy
        per_copy = info["bytes"] * (1 if store == "f32" else 2)
        assert info["copy_bytes"] == per_copy * bin(info["copies"]).count("1")
        a, na, b, nb = a.cpu().numpy(), na.cpu().numpy(), b.cpu().numpy(), nb.cpu().numpy()
        assert np.array_equal(b, a[rows, cols]) and np.array_equal(nb, na[rows, cols])
        if store == "f32":
            for cam, img, ns in ((camA, a, na), (camB, b, nb)):
                compare(img, ns, oracle.render(cube, cam, tf_np, VMIN, VMAX, STEP), TOL_F32)
        assert a[..., 3].max() > 0.1
    finally:
        vol.close()


def test_batch_with_every_order_matches_single_renders(P, torch, scene):
    """One batch holding views of all three axes (one launch per layout, in
    one graph) equals the single renders bit for bit, replayed."""
    cube, tf_np = scene
    vol = _volume(P, torch, cube)
    tf = torch.from_numpy(tf_np).cuda()
    try:
        cams = [_cam(f, u, k) for k in ("persp", "ortho") for (f, u) in
                [PAIRS[0][0], PAIRS[0][1], PAIRS[1][1], PAIRS[1][0]]]
        singles = [P.render(vol, c, tf, VMIN, VMAX, STEP) for c in cams]
        jobs = [dict(vol=vol, cam=c, tf=tf, vmin=VMIN, vmax=VMAX, step=STEP,
                     out=torch.empty((W, W, 4), device="cuda"),
                     nsamples=torch.empty((W, W), device="cuda", dtype=torch.int32)) for c in cams]
        for _ in range(2):
            for j in jobs:
                j["out"].fill_(-1.0)
                j["nsamples"].fill_(-1)
            P.render_batched(jobs, use_graph=True)
            torch.cuda.synchronize()
            for j, (img, ns) in zip(jobs, singles):
                assert torch.equal(j["out"], img) and torch.equal(j["nsamples"], ns)
        assert _copies(P, vol) == 0b110
    finally:
        vol.close()


def test_noalloc_batch_uses_only_existing_copies(P, torch, scene):
    """The allocation-free batch never builds a copy (it reads the bricks
    themselves); once a render has built one it reads it.  Either way the
    images equal the single render bit for bit."""
    cube, tf_np = scene
    vol = _volume(P, torch, cube)
    tf = torch.from_numpy(tf_np).cuda()
    try:
        camB = _cam(*PAIRS[0][1], "persp")
        first, ns_first = _noalloc(P, torch, vol, camB, tf)
        assert _copies(P, vol) == 0
        img, ns = P.render(vol, camB, tf, VMIN, VMAX, STEP)
        torch.cuda.synchronize()
        assert _copies(P, vol) == 0b10
        assert torch.equal(first, img) and torch.equal(ns_first, ns)
        again, ns_again = _noalloc(P, torch, vol, camB, tf)
        assert torch.equal(again, img) and torch.equal(ns_again, ns)
    finally:
        vol.close()


@pytest.mark.parametrize("store", ["f16", "bf16"])
def test_half_paired_copies_match_bricks(P, torch, scene, store):
    """16-bit storage: paired copies (two halves per load) render exactly what
    the bricks themselves render, for an x-, y- and z-copy view."""
    cube, tf_np = scene
    vol = _volume(P, torch, cube, store)
    tf = torch.from_numpy(tf_np).cuda()
    try:
        cams = [_cam(*PAIRS[0][0], "persp"), _cam(*PAIRS[0][1], "persp"), _cam(*PAIRS[1][1], "ortho")]
        plain = [_noalloc(P, torch, vol, c, tf) for c in cams]
        assert _copies(P, vol) == 0
        for c, (img0, ns0) in zip(cams, plain):
            img, ns = P.render(vol, c, tf, VMIN, VMAX, STEP)
            torch.cuda.synchronize()
            assert torch.equal(img, img0) and torch.equal(ns, ns0)
        assert _copies(P, vol) == 0b111000
        (fa, ua), (fb, ub), order, (rows, cols) = PAIRS[0]
        a = plain[0][0].cpu().numpy()
        b = plain[1][0].cpu().numpy()
        assert np.array_equal(b, a[rows, cols])
    finally:
        vol.close()


def _sparse_blocked_case(P, torch, scene, store, brick):
    """Rays about 3-4 voxels apart (16x16 images of the 40x36x44 cube): the
    forward reads a blocked copy (2 x 2 x 2 float or 2 x 2 x 4 16-bit blocks
    of one 32-byte sector, deep along the axis the rays advance along), bit
    for bit the result of the bricks themselves (read by the allocation-free
    batch, which builds no copy); a rolled view matches; a batch of these
    views reads the same copies and equals the single renders."""
    cube, tf_np = scene
    vol = P.Volume(torch.from_numpy(np.ascontiguousarray(cube)).cuda(), store, brick=brick)
    tf = torch.from_numpy(tf_np).cuda()
    n = 16
    i, j = np.arange(n)[None, :], np.arange(n)[:, None]
    from paper_1211_4896_gb300 import _lib as L
    try:
        cams = [_cam(*PAIRS[0][0], "persp", n), _cam(*PAIRS[0][1], "persp", n), _cam(*PAIRS[1][1], "ortho", n),
                _cam((1, 0, 0), (0, 1, 0), "persp", n)]
        plain = []
        for c in cams:
            out = torch.full((n, n, 4), -1.0, device="cuda")
            ns = torch.full((n, n), -1, device="cuda", dtype=torch.int32)
            job = L.vr_job(vol.handle, L.make_camera(c),
                           L.make_params(tf.data_ptr(), tf.shape[0], VMIN, VMAX, STEP, 2.0), out.data_ptr(),
                           ns.data_ptr())
            L.vr_render_batched_noalloc([job], 8, 4, int(torch.cuda.current_stream().cuda_stream))
            torch.cuda.synchronize()
            plain.append((out, ns))
        assert _copies(P, vol) == 0
        for c, (img0, ns0) in zip(cams, plain):
            img, ns = P.render(vol, c, tf, VMIN, VMAX, STEP)
            torch.cuda.synchronize()
            assert torch.equal(img, img0) and torch.equal(ns, ns0)
        # blocked copies deep along z (views along z), y and x: ids 8, 7, 6
        assert _copies(P, vol) == (1 << 8) | (1 << 7) | (1 << 6)
        assert [L.vr_view_layout(vol.handle, L.make_camera(c)) for c in cams] == [8, 8, 7, 6]
        info = L.vr_volume_info(vol.handle)
        eb = 4 if store == "f32" else 2
        bw = 2 if eb == 4 else 4
        per = (brick + 2) ** 2 * ((brick + bw) // bw * bw) * eb * int(np.prod(info["bricks"]))
        assert info["copy_bytes"] == 3 * per
        a = plain[0][0].cpu().numpy()
        b, _ = P.render(vol, cams[1], tf, VMIN, VMAX, STEP)
        assert np.array_equal(b.cpu().numpy(), a[n - 1 - i, j])
        assert a[..., 3].max() > 0.1
        jobs = [dict(vol=vol, cam=c, tf=tf, vmin=VMIN, vmax=VMAX, step=STEP,
                     out=torch.empty((n, n, 4), device="cuda"),
                     nsamples=torch.empty((n, n), device="cuda", dtype=torch.int32)) for c in cams]
        P.render_batched(jobs, use_graph=True)
        torch.cuda.synchronize()
        for jb, (img0, ns0) in zip(jobs, plain):
            assert torch.equal(jb["out"], img0) and torch.equal(jb["nsamples"], ns0)
        if store == "f32":
            for c, (img, ns) in zip(cams, plain):
                compare(img.cpu().numpy(), ns.cpu().numpy(), oracle.render(cube, c, tf_np, VMIN, VMAX, STEP), TOL_F32)
    finally:
        vol.close()


@pytest.mark.parametrize("store,brick", [("f16", 16), ("bf16", 16), ("f16", 32)])
def test_sparse_rays_read_blocked_copies(P, torch, scene, store, brick):
    """16-bit storage: sparse views read blocked copies by default."""
    _sparse_blocked_case(P, torch, scene, store, brick)


def test_sparse_rays_in_64_bricks_read_row_copies(P, torch, scene):
    """16-bit storage in 64^3 bricks (the default for large volumes): sparse
    views read the bricks and the row copies (the image rows' axis fastest),
    which measured faster there than blocked copies; bit for bit the result
    of the bricks themselves, and no blocked copy is built."""
    cube, tf_np = scene
    vol = P.Volume(torch.from_numpy(np.ascontiguousarray(cube)).cuda(), "f16", brick=64)
    tf = torch.from_numpy(tf_np).cuda()
    n = 16
    from paper_1211_4896_gb300 import _lib as L
    try:
        cams = [_cam(*PAIRS[0][0], "persp", n), _cam(*PAIRS[0][1], "persp", n), _cam(*PAIRS[1][1], "ortho", n),
                _cam((1, 0, 0), (0, 1, 0), "persp", n)]
        for c in cams:
            out = torch.full((n, n, 4), -1.0, device="cuda")
            ns = torch.full((n, n), -1, device="cuda", dtype=torch.int32)
            job = L.vr_job(vol.handle, L.make_camera(c),
                           L.make_params(tf.data_ptr(), tf.shape[0], VMIN, VMAX, STEP, 2.0), out.data_ptr(),
                           ns.data_ptr())
            L.vr_render_batched_noalloc([job], 8, 4, int(torch.cuda.current_stream().cuda_stream))
            img, ns1 = P.render(vol, c, tf, VMIN, VMAX, STEP)
            torch.cuda.synchronize()
            assert torch.equal(img, out) and torch.equal(ns1, ns)
            assert L.vr_view_layout(vol.handle, L.make_camera(c)) in (-1, 1, 2)
        assert _copies(P, vol) & ((1 << 6) | (1 << 7) | (1 << 8)) == 0
        assert _copies(P, vol) != 0                       # at least one row copy was taken
    finally:
        vol.close()


@pytest.mark.parametrize("brick", [16, 32])
def test_float_sparse_rays_read_blocked_copies_when_asked(brick):
    """Float storage reads blocked copies for sparse views when
    VR_SPARSE_LAYOUT=b (a separate process: the library reads the variable
    once)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, VR_SPARSE_LAYOUT="b",
               PYTHONPATH=root + os.pathsep + os.environ.get("PYTHONPATH", ""))
    code = ("import torch, tests.test_gpu_brick_copies as t, paper_1211_4896_gb300 as P, synth\n"
            "cube = synth.hi_cube(t.DIMS, n_blobs=8, n_disks=1, seed=7).numpy()\n"
            "tf = synth.tf_random_pwl(seed=3, alpha_max=0.3)\n"
            "t._sparse_blocked_case(P, torch, (cube, tf), 'f32', %d)\nprint('ok')\n" % brick)
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]


@pytest.mark.parametrize("pair", range(len(PAIRS)))
def test_backward_of_rolled_view_matches(P, torch, scene, pair):
    """Adjoint of the rolled view with the rolled output gradient: the same
    table and voxel gradients up to FP32 summation order."""
    cube, tf_np = scene
    (fa, ua), (fb, ub), order, (rows, cols) = PAIRS[pair]
    vol = _volume(P, torch, cube)
    tf = torch.from_numpy(tf_np).cuda()
    try:
        camA, camB = _cam(fa, ua, "persp"), _cam(fb, ub, "persp")
        gA = np.random.default_rng(11).standard_normal((W, W, 4)).astype(np.float32)
        gB = np.ascontiguousarray(gA[rows, cols])
        out = []
        for cam, g in ((camA, gA), (camB, gB)):
            img, ns = P.render(vol, cam, tf, VMIN, VMAX, STEP)
            gt, gv = P.render_backward(vol, cam, tf, VMIN, VMAX, STEP, img, ns, torch.from_numpy(g).cuda())
            torch.cuda.synchronize()
            out.append((gt.cpu().numpy(), gv.cpu().numpy()))
        assert _copies(P, vol) == 1 << order
        (tA, vA), (tB, vB) = out
        assert np.abs(tA - tB).max() <= 1e-5 * np.abs(tA).max()
        assert np.abs(vA - vB).max() <= 1e-5 * np.abs(vA).max()
        assert np.abs(vA).max() > 0
    finally:
        vol.close()


def test_update_refreshes_reordered_copies(P, torch, scene):
    """After vr_volume_update a view reading a reordered copy sees the new
    voxels: it still equals its x-order roll and the oracle on the new cube."""
    cube, tf_np = scene
    vol = _volume(P, torch, cube)
    tf = torch.from_numpy(tf_np).cuda()
    try:
        (fa, ua), (fb, ub), order, (rows, cols) = PAIRS[1]
        camA, camB = _cam(fa, ua, "ortho"), _cam(fb, ub, "ortho")
        P.render(vol, camB, tf, VMIN, VMAX, STEP)
        torch.cuda.synchronize()
        assert _copies(P, vol) == 1 << order
        cube2 = np.ascontiguousarray(cube[::-1, :, ::-1]) * np.float32(1.3)
        vol.update(torch.from_numpy(cube2).cuda())
        a, na = P.render(vol, camA, tf, VMIN, VMAX, STEP)
        b, nb = P.render(vol, camB, tf, VMIN, VMAX, STEP)
        torch.cuda.synchronize()
        a, b = a.cpu().numpy(), b.cpu().numpy()
        assert np.array_equal(b, a[rows, cols])
        compare(b, nb.cpu().numpy(), oracle.render(cube2, camB, tf_np, VMIN, VMAX, STEP), TOL_F32)
    finally:
        vol.close()


def test_auto_brick_size_follows_volume_bytes(P, torch):
    """brick = 0 picks 16^3 bricks, and 64^3 once 16^3 bricks (with their
    +1 apron) would take more than 16 GiB: a 2048 x 2048 x 1024 16-bit cube
    needs about 10 GB of 16^3 bricks, a 4096 x 2048 x 1024 one about 21 GB."""
    for (nz, ny, nx), want in (((1024, 2048, 2048), 16), ((1024, 2048, 4096), 64)):
        cube = torch.zeros((nz, ny, nx), device="cuda", dtype=torch.float16)
        vol = P.Volume(cube, "f16")
        try:
            assert vol.info["brick"] == want, (nx, ny, nz, vol.info["brick"])
        finally:
            vol.close()
            del cube
            torch.cuda.empty_cache()
