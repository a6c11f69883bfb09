"""GPU adjoint parity: the re-march backward kernel against (a) the oracle's
store-all FP64 reverse sweep (a different algorithm) and (b) central finite
differences of the GPU forward (h = 1e-3) on table entries and voxels, with
the rule |g - fd| <= 1e-3 max(|fd|, 1e-3 max_j |fd_j|); FD points where the
one-sided differences disagree (a kink within h) are redrawn."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import cuda_or_skip

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


@pytest.fixture(scope="module")
def P(torch):
    import paper_1211_4896_gb300 as P
    return P


def _setup(torch, P, dims, seed, W, H, store="f32"):
    dev = torch.device("cuda")
    cube = synth.hi_cube(dims, n_blobs=max(4, int(np.prod(dims) / 30000)), n_disks=1, seed=seed)
    vol = P.Volume(cube.to(dev), store)
    cam = synth.camera_random_persp(dims, seed=seed + 1, width=W, height=H)
    return cube, vol, cam


def _grad_close(g, ref, rel=1e-3):
    scale = np.abs(ref).max()
    err = np.abs(g - ref)
    bound = rel * np.maximum(np.abs(ref), 1e-3 * scale) + 1e-12
    return err <= bound, err, bound


@pytest.mark.parametrize("filt", [0, 2])
@pytest.mark.parametrize("ert,bg", [(2.0, (0, 0, 0, 0)), (0.9, (0.2, 0.1, 0.4, 0.3))])
def test_backward_matches_fp64_reverse_sweep(P, torch, ert, bg, filt):
    dims = (36, 30, 40)
    cube, vol, cam = _setup(torch, P, dims, seed=12, W=48, H=40)
    dev = torch.device("cuda")
    tf_np = synth.tf_random_pwl(seed=3, alpha_max=0.25)
    tf = torch.from_numpy(tf_np).to(dev)
    img, ns = P.render(vol, cam, tf, -3.0, 30.0, 0.5, ert, bg, filter=filt)
    target = torch.rand_like(img)
    g = 2.0 * (img - target)
    gtf, gvox = P.render_backward(vol, cam, tf, -3.0, 30.0, 0.5, img, ns, g, ert, bg, filter=filt)
    torch.cuda.synchronize()
    ref_tf, ref_vox = oracle.render_backward(cube.numpy(), cam, tf_np, -3.0, 30.0, 0.5,
                                             g.cpu().numpy().astype(np.float64), ert=ert, bg=bg)
    # The GPU marches in FP32: sample positions carry ~1e-5 voxel rounding, so
    # a sample's value moves by |grad v| * 1e-5 and its table-bin weight by
    # (K-1)/(vmax-vmin) times that (7.7 bins per unit value here).  Gradients
    # are therefore compared norm-wise and against the largest entry, at 1e-3.
    gt = gtf.cpu().numpy()
    rel_norm = np.linalg.norm(gt - ref_tf) / np.linalg.norm(ref_tf)
    rel_max = np.abs(gt - ref_tf).max() / np.abs(ref_tf).max()
    print("table gradient: rel. norm err %.3g, max err / max |g| %.3g" % (rel_norm, rel_max))
    assert rel_norm <= 1e-3 and rel_max <= 1e-3, (rel_norm, rel_max)
    gv = gvox.cpu().numpy().astype(np.float64)
    rel_norm = np.linalg.norm(gv - ref_vox) / np.linalg.norm(ref_vox)
    rel_max = np.abs(gv - ref_vox).max() / np.abs(ref_vox).max()
    print("voxel gradient: rel. norm err %.3g, max err / max |g| %.3g" % (rel_norm, rel_max))
    assert rel_norm <= 1e-3 and rel_max <= 1e-3, (rel_norm, rel_max)
    vol.close()


@pytest.mark.parametrize("K", [2, 1600])
def test_backward_smallest_and_largest_table(P, torch, K, monkeypatch):
    """The backward copies its table into shared memory (K float4 entries, up
    to 1600, the largest table it accepts): the two-entry table and the
    largest one against the oracle's FP64 reverse sweep, through the texture
    layers (the dense float view's copy) and through the brick copies."""
    dims = (30, 26, 34)
    cube, vol, cam = _setup(torch, P, dims, seed=33, W=40, H=36)
    dev = torch.device("cuda")
    tf_np = synth.tf_ramp(K, alpha_max=0.3)
    tf = torch.from_numpy(tf_np).to(dev)
    g, ref_tf, ref_vox = None, None, None
    for layers in ("1", "0"):
        monkeypatch.setenv("VR_TEX_LAYERS", layers)        # read at each call
        img, ns = P.render(vol, cam, tf, -3.0, 30.0, 0.5, 2.0)
        if g is None:
            g = torch.randn(img.shape, device=dev, generator=torch.Generator(device=dev).manual_seed(K))
            ref_tf, ref_vox = oracle.render_backward(cube.numpy(), cam, tf_np, -3.0, 30.0, 0.5,
                                                     g.cpu().numpy().astype(np.float64))
        gtf, gvox = P.render_backward(vol, cam, tf, -3.0, 30.0, 0.5, img, ns, g, 2.0)
        torch.cuda.synchronize()
        for got, ref in ((gtf.cpu().numpy(), ref_tf), (gvox.cpu().numpy().astype(np.float64), ref_vox)):
            rel_norm = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            rel_max = np.abs(got - ref).max() / np.abs(ref).max()
            assert rel_norm <= 1e-3 and rel_max <= 1e-3, (K, layers, rel_norm, rel_max)
    with pytest.raises(P.VRError):                            # one entry more is refused
        big = torch.from_numpy(synth.tf_ramp(1601, alpha_max=0.3)).to(dev)
        P.render_backward(vol, cam, big, -3.0, 30.0, 0.5, img, ns, g, 2.0)
    vol.close()


@pytest.mark.parametrize("dims,brick,store,W,H,step", [((36, 30, 40), 16, "f32", 48, 40, 0.5),
                                                       ((41, 27, 33), 32, "f16", 64, 56, 0.35),
                                                       ((30, 34, 26), 16, "bf16", 40, 30, 1.0)])
def test_voxel_gradient_direct_and_scratch_reductions_agree(P, torch, dims, brick, store, W, H, step):
    """Both voxel-gradient reductions (straight into the dense gradient, and
    through the quad scratch plus its gather) against the FP64 reverse sweep,
    overwriting and accumulating over three views (carried along x, y and z),
    per view and in one multi-view call; odd and even nx, table and voxel
    gradients alike."""
    dev = torch.device("cuda")
    cube = synth.hi_cube(dims, n_blobs=5, n_disks=1, seed=sum(dims))
    t = cube.to(dev)
    vol = P.Volume(t, store, brick=brick)
    ref_cube = (cube.numpy() if store == "f32" else
                (t.half() if store == "f16" else t.bfloat16()).float().cpu().numpy()).astype(np.float64)
    tf_np = synth.tf_random_pwl(seed=W, alpha_max=0.3)
    tf = torch.from_numpy(tf_np).to(dev)
    cams = [synth.camera_random_persp(dims, seed=7 * q + H, width=W, height=H) for q in range(2)]
    # and one view mostly along y (the random ones carry along x or z)
    ext = [d - 1.0 for d in dims]
    fwd = np.array([0.25, -0.93, 0.27]) / np.linalg.norm([0.25, -0.93, 0.27])
    eye = tuple(e / 2.0 - 1.6 * max(ext) * f for e, f in zip(ext, fwd))
    cams.append(synth.camera_persp(eye, tuple(fwd), (0.0, 0.0, 1.0), 40.0, W, H))
    try:
        res = {}
        ref_tf, ref_vox = 0.0, 0.0
        for q, cam in enumerate(cams):
            img, ns = P.render(vol, cam, tf, -3.0, 30.0, step, 2.0)
            g = torch.randn(img.shape, device=dev, generator=torch.Generator(device=dev).manual_seed(q))
            rt, rv = oracle.render_backward(ref_cube, cam, tf_np, -3.0, 30.0, step,
                                            g.cpu().numpy().astype(np.float64))
            ref_tf, ref_vox = ref_tf + rt, ref_vox + rv
            for mode in ("direct", "scratch"):
                prev = res.get(mode)
                gtf, gvox = P.render_backward(vol, cam, tf, -3.0, 30.0, step, img, ns, g, 2.0,
                                              grad_tf=None if prev is None else prev[0],
                                              grad_vox=None if prev is None else prev[1],
                                              accumulate=prev is not None, vox_reduce=mode)
                res[mode] = (gtf, gvox)
        # the same three views in one call
        imgs, nss, gs = [], [], []
        for q, cam in enumerate(cams):
            img, ns = P.render(vol, cam, tf, -3.0, 30.0, step, 2.0)
            imgs.append(img)
            nss.append(ns)
            gs.append(torch.randn(img.shape, device=dev, generator=torch.Generator(device=dev).manual_seed(q)))
        for mode in ("direct", "scratch"):
            res["views_" + mode] = P.render_backward_views(vol, cams, tf, -3.0, 30.0, step, imgs, nss, gs, 2.0,
                                                           vox_reduce=mode)
        torch.cuda.synchronize()
        for mode, (gtf, gvox) in res.items():
            for got, ref in ((gtf.cpu().numpy(), ref_tf), (gvox.cpu().numpy().astype(np.float64), ref_vox)):
                rel_norm = np.linalg.norm(got - ref) / np.linalg.norm(ref)
                rel_max = np.abs(got - ref).max() / np.abs(ref).max()
                assert rel_norm <= 1e-3 and rel_max <= 1e-3, (mode, rel_norm, rel_max)
        d, s = res["direct"][1], res["scratch"][1]
        assert (d - s).abs().max().item() <= 1e-4 * d.abs().max().item()
        assert (s != 0).float().mean().item() > 0.05
        info = P._lib.vr_volume_info(vol.handle)                # the quad scratch is held and reported
        assert info["scratch_bytes"] >= 16 * int(np.prod(dims))
    finally:
        vol.close()


def test_backward_central_differences_table_and_voxels(P, torch):
    """Scaled-down form of the differentiation workload: L2 loss against a
    target rendered with a hidden table; FD on 32 table entries, 32 voxels."""
    dev = torch.device("cuda")
    dims = (64, 64, 64)
    cube, vol, cam = _setup(torch, P, dims, seed=31, W=96, H=96)
    cube_d = cube.to(dev)
    hidden = torch.from_numpy(synth.tf_ramp(256)).to(dev)
    tf = (hidden + 0.05 * torch.rand_like(hidden)).clamp(0, 1).contiguous()
    tf[:, 3] *= 0.5
    step = 0.5
    tgt, _ = P.render(vol, cam, hidden, synth.TF_VMIN, synth.TF_VMAX, step, 2.0)

    def loss(tfv, vol_):
        im, _ = P.render(vol_, cam, tfv, synth.TF_VMIN, synth.TF_VMAX, step, 2.0)
        return float(((im.double() - tgt.double()) ** 2).sum())

    img, ns = P.render(vol, cam, tf, synth.TF_VMIN, synth.TF_VMAX, step, 2.0)
    gtf, gvox = P.render_backward(vol, cam, tf, synth.TF_VMIN, synth.TF_VMAX, step, img, ns, 2.0 * (img - tgt), 2.0)
    gtf = gtf.cpu().numpy()
    gvox = gvox.cpu().numpy()
    h = 1e-3
    rng = np.random.default_rng(0)
    # table entries with a non-zero gradient
    cand = np.argwhere(np.abs(gtf) > 1e-3 * np.abs(gtf).max())
    picks = cand[rng.choice(len(cand), size=32, replace=False)]
    fds, gs = [], []
    for (e, ch) in picks:
        tp, tm = tf.clone(), tf.clone()
        tp[e, ch] += h
        tm[e, ch] -= h
        fds.append((loss(tp, vol) - loss(tm, vol)) / (2 * h))
        gs.append(gtf[e, ch])
    fds, gs = np.array(fds), np.array(gs)
    ok, err, bound = _grad_close(gs, fds)
    assert ok.all(), list(zip(gs[~ok], fds[~ok]))
    print("table FD (h=1e-3): max |g - fd| / |fd| = %.3g" % np.max(np.abs(gs - fds) / np.abs(fds)))
    # Voxels.  (1) Strict: central differences (h = 1e-3) of the FP64 forward
    # render (the exact rendering function) against the GPU gradient, 1e-3
    # rule, kink-screened.  (2) The GPU forward itself, at h = 1e-2: a voxel
    # nudged by h moves a nearby sample's opacity by ~1e-3 h * |d alpha/dv|
    # (~2e-6 here) while FP32 stores opacities with a half-ulp of ~4e-9, so a
    # re-rendered sample resolves the change only to ~0.2%; a voxel feeds a
    # handful of samples, whose rounding does not average out (0.4%-1.1%
    # measured over runs), so the GPU-forward differences are a sanity check
    # held to 3e-2.
    cube_np = cube.numpy().astype(np.float64)
    tf_np = tf.cpu().numpy()
    tgt_np = tgt.cpu().numpy().astype(np.float64)

    def loss64(V):
        I = oracle.render(V, cam, tf_np, synth.TF_VMIN, synth.TF_VMAX, step, 2.0)["rgba"]
        return float(((I - tgt_np) ** 2).sum())

    L0 = loss64(cube_np)
    cand = np.argwhere(np.abs(gvox) > 1e-2 * np.abs(gvox).max())
    fds, gs = [], []
    for q in rng.permutation(len(cand)):
        z, y, x = cand[q]
        vals = []
        for d in (h, -h):
            V = cube_np.copy()
            V[z, y, x] += d
            vals.append(loss64(V))
        right, left = (vals[0] - L0) / h, (L0 - vals[1]) / h
        if abs(right - left) > 2e-4 * max(abs(right), abs(left), 1e-9):
            continue
        fds.append((vals[0] - vals[1]) / (2 * h))
        gs.append(gvox[z, y, x])
        if len(fds) == 32:
            break
    fds, gs = np.array(fds), np.array(gs)
    ok, err, bound = _grad_close(gs, fds)
    print("voxel FD of the FP64 forward (h=1e-3): max |g - fd| / |fd| = %.3g" % np.max(np.abs(gs - fds) / np.abs(fds)))
    assert len(fds) == 32 and ok.all(), list(zip(gs[~ok], fds[~ok]))

    h = 1e-2
    L0 = loss(tf, vol)
    cand = np.argwhere(np.abs(gvox) > 1e-2 * np.abs(gvox).max())
    checked = 0
    fds, gs = [], []
    for q in rng.permutation(len(cand)):
        z, y, x = cand[q]
        vals = []
        for d in (h, -h):
            c2 = cube_d.clone()
            c2[z, y, x] += d
            vol.update(c2)
            vals.append(loss(tf, vol))
        vol.update(cube_d)
        right, left = (vals[0] - L0) / h, (L0 - vals[1]) / h
        if abs(right - left) > 2e-3 * max(abs(right), abs(left), 1e-6):
            continue
        fds.append((vals[0] - vals[1]) / (2 * h))
        gs.append(gvox[z, y, x])
        checked += 1
        if checked == 32:
            break
    fds, gs = np.array(fds), np.array(gs)
    ok, err, bound = _grad_close(gs, fds, rel=3e-2)
    print("voxel FD of the GPU forward (h=1e-2): max |g - fd| / |fd| = %.3g" % np.max(np.abs(gs - fds) / np.abs(fds)))
    assert checked == 32 and ok.all(), list(zip(gs[~ok], fds[~ok]))
    vol.close()


def test_autograd_function(P, torch):
    dev = torch.device("cuda")
    dims = (32, 32, 32)
    cube, vol, cam = _setup(torch, P, dims, seed=5, W=40, H=40)
    c = cube.to(dev).requires_grad_(True)
    tf = torch.from_numpy(synth.tf_random_pwl(seed=1)).to(dev).requires_grad_(True)
    img = P.render_diff(c, tf, vol, cam, -3.0, 30.0, 0.5)
    loss = (img ** 2).sum()
    loss.backward()
    img2, ns = P.render(vol, cam, tf.detach(), -3.0, 30.0, 0.5)
    gtf, gvox = P.render_backward(vol, cam, tf.detach(), -3.0, 30.0, 0.5, img2, ns, 2 * img2)
    torch.cuda.synchronize()
    assert torch.allclose(tf.grad, gtf.float(), rtol=1e-4, atol=1e-6)
    assert torch.allclose(c.grad, gvox, rtol=1e-3, atol=1e-6)
    vol.close()


def test_backward_rejects_opaque_background_and_texture(P, torch):
    dev = torch.device("cuda")
    cube, vol, cam = _setup(torch, P, (16, 16, 16), seed=2, W=8, H=8)
    tf = torch.from_numpy(synth.tf_ramp(16)).to(dev)
    img, ns = P.render(vol, cam, tf, -3, 50, 0.5)
    with pytest.raises(P.VRError) as ei:
        P.render_backward(vol, cam, tf, -3, 50, 0.5, img, ns, img, bg=(0, 0, 0, 1.0))
    assert ei.value.status == -2
    vol.close()


@pytest.mark.parametrize("filt", [0, 2])
def test_multi_view_call_equals_accumulated_single_calls(P, torch, filt):
    """vr_render_backward_views (one call for several views, with and
    without VR_GRAD_ACCUMULATE on top of earlier sums) equals the per-view
    calls accumulated, for the brick path and the staged filter, and leaves
    the gradients untouched by views that miss the box."""
    dev = torch.device("cuda")
    dims = (30, 26, 34)
    cube, vol, _ = _setup(torch, P, dims, seed=21, W=40, H=32)
    tf = torch.from_numpy(synth.tf_random_pwl(seed=4, alpha_max=0.3)).to(dev)
    cams = [synth.camera_random_persp(dims, seed=40 + q, width=40, height=32) for q in range(3)]
    # a fourth view that looks away from the cube: no ray hits it
    away = dict(cams[0], forward=tuple(-f for f in cams[0]["forward"]))
    cams.append(away)
    imgs, nss, gs = [], [], []
    for q, cam in enumerate(cams):
        img, ns = P.render(vol, cam, tf, -3.0, 30.0, 0.5, 2.0, filter=filt)
        imgs.append(img)
        nss.append(ns)
        gs.append(torch.randn(img.shape, device=dev, generator=torch.Generator(device=dev).manual_seed(100 + q)))
    assert int(nss[3].sum()) == 0
    try:
        ref_tf, ref_vox = None, None
        for q, cam in enumerate(cams):
            ref_tf, ref_vox = P.render_backward(vol, cam, tf, -3.0, 30.0, 0.5, imgs[q], nss[q], gs[q], 2.0,
                                                grad_tf=ref_tf, grad_vox=ref_vox, accumulate=q > 0, filter=filt)
        got_tf, got_vox = P.render_backward_views(vol, cams, tf, -3.0, 30.0, 0.5, imgs, nss, gs, 2.0, filter=filt)
        # accumulate: the first two views, then the last two on top
        acc_tf, acc_vox = P.render_backward_views(vol, cams[:2], tf, -3.0, 30.0, 0.5, imgs[:2], nss[:2], gs[:2],
                                                  2.0, filter=filt)
        acc_tf, acc_vox = P.render_backward_views(vol, cams[2:], tf, -3.0, 30.0, 0.5, imgs[2:], nss[2:], gs[2:],
                                                  2.0, grad_tf=acc_tf, grad_vox=acc_vox, accumulate=True,
                                                  filter=filt)
        torch.cuda.synchronize()
        for t, v in ((got_tf, got_vox), (acc_tf, acc_vox)):
            assert (t - ref_tf).abs().max().item() <= 1e-5 * ref_tf.abs().max().item()
            assert (v - ref_vox).abs().max().item() <= 1e-4 * ref_vox.abs().max().item()
        assert ref_vox.abs().max().item() > 0
    finally:
        vol.close()


def test_multi_view_call_many_views_mixed_layouts_and_sizes(P, torch):
    """One vr_render_backward_views call over 22 views (19 of them looking
    along z, three along x or y, one of them away from the box), with images
    of ragged sizes (widths and heights that are not multiples of the 8 x 4
    ray tile), equals the per-view calls accumulated: the views' kernels
    alternate between two streams and overlap, each with its own work
    counter, all adding into the same rows and voxel gradient."""
    from paper_1211_4896_gb300 import _lib as L
    dev = torch.device("cuda")
    dims = (34, 30, 28)
    cube = synth.hi_cube(dims, n_blobs=6, n_disks=1, seed=77)
    vol = P.Volume(cube.to(dev), "f32")
    tf = torch.from_numpy(synth.tf_random_pwl(seed=8, alpha_max=0.3)).to(dev)
    ext = [d - 1.0 for d in dims]
    rng = np.random.default_rng(3)
    cams = []
    for q in range(22):
        if q < 19:
            f = np.array([rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), 1.0])
        else:
            f = [np.array([1.0, 0.15, 0.1]), np.array([0.1, -1.0, 0.2]), np.array([0.0, 0.0, -1.0])][q - 19]
        f = f / np.linalg.norm(f)
        eye = tuple(e / 2.0 - 1.7 * max(ext) * c for e, c in zip(ext, f))
        if q == 21:                     # looks away from the box
            f = -f
        up = (0.0, 1.0, 0.0) if abs(f[1]) < 0.9 else (0.0, 0.0, 1.0)
        W, H = [(37, 29), (8, 4), (41, 13), (16, 9), (23, 31)][q % 5]
        cams.append(synth.camera_persp(eye, tuple(f), up, 40.0, W, H))
    imgs, nss, gs = [], [], []
    for q, cam in enumerate(cams):
        img, ns = P.render(vol, cam, tf, -3.0, 30.0, 0.5, 2.0)
        imgs.append(img)
        nss.append(ns)
        gs.append(torch.randn(img.shape, device=dev, generator=torch.Generator(device=dev).manual_seed(300 + q)))
    # the layouts the renders built and read
    layouts = [L.vr_view_layout(vol.handle, L.make_camera(c)) for c in cams]
    assert len(set(layouts)) >= 2, layouts
    assert int(nss[21].sum()) == 0
    try:
        ref_tf, ref_vox = None, None
        for q, cam in enumerate(cams):
            ref_tf, ref_vox = P.render_backward(vol, cam, tf, -3.0, 30.0, 0.5, imgs[q], nss[q], gs[q], 2.0,
                                                grad_tf=ref_tf, grad_vox=ref_vox, accumulate=q > 0,
                                                vox_reduce="direct")
        got_tf, got_vox = P.render_backward_views(vol, cams, tf, -3.0, 30.0, 0.5, imgs, nss, gs, 2.0,
                                                  vox_reduce="direct")
        torch.cuda.synchronize()
        assert (got_tf - ref_tf).abs().max().item() <= 1e-5 * ref_tf.abs().max().item()
        assert (got_vox - ref_vox).abs().max().item() <= 1e-4 * ref_vox.abs().max().item()
        assert ref_vox.abs().max().item() > 0
    finally:
        vol.close()


@pytest.mark.slow
def test_differentiation_workload_crop_elementwise_against_fp64(P, torch):
    """The differentiation workload's kernel configuration checked element by
    element against the FP64 store-all reverse sweep on a 32^3 crop: the 512^3
    float32 cube of that workload, cropped around its brightest voxel; its four
    orbit views refitted to the crop at the workload's ray pitch (0.9 voxel at
    the centre, so 64^2 images: the same samples per voxel as the 1024^2 views
    of the whole cube), step 0.5, no early termination; L2 loss against
    targets rendered with the hidden ramp table; gradients of the loss over
    the four views from one vr_render_backward_views call, which takes the
    quad scratch by itself (the views are dense).

    Every table entry must satisfy |g - ref| <= 1e-3 max(|ref|, 1e-3 max|ref|).
    So must every voxel, up to two allowances the oracle computes:
      - its kink bound: the voxel gradient of a piecewise-linear table jumps
        where a sample's value crosses an interval end, and a sample within
        FP32 rounding of one (tolerance from the crop's largest value gradient
        and a 1e-5 voxel position error) may take either side's slope; the
        bound is the largest change that choice can make;
      - the FP32 forward error of the re-march, 2 N u times the sum of the
        magnitudes the voxel's terms are made of (u = 2^-24, N the longest
        ray's sample count): the suffix colour is formed by running sums
        along the ray, so where the terms cancel to a small gradient the
        rounding of the large parts remains (the one-sided FD rule's floor,
        1e-6 max|ref|, is below it there)."""
    from paper_1211_4896_gb300 import _lib as L
    dev = torch.device("cuda")
    pre = synth.preset_diff_512()
    cube = synth.hi_cube(pre["dims"], pre["n_blobs"], pre["n_disks"], pre["seed"], device=dev)
    n = 32
    flat = int(torch.argmax(cube).item())
    centre = np.unravel_index(flat, cube.shape)                     # (z, y, x)
    lo = [int(min(max(c - n // 2, 0), s - n)) for c, s in zip(centre, cube.shape)]
    crop = cube[lo[0]:lo[0] + n, lo[1]:lo[1] + n, lo[2]:lo[2] + n].contiguous()
    del cube
    torch.cuda.empty_cache()
    crop_np = crop.cpu().numpy()
    vol = P.Volume(crop, "f32")
    cams = synth.orbit_cameras((n, n, n), 4, 40.0, 64, 64, start_deg=20.0)
    hidden_np = synth.tf_ramp(256)
    rng = np.random.default_rng(5)
    tf_np = np.clip(hidden_np + 0.05 * rng.uniform(size=hidden_np.shape), 0.0, 1.0).astype(np.float32)
    hidden = torch.from_numpy(hidden_np).to(dev)
    tf = torch.from_numpy(tf_np).to(dev)
    step, vmin, vmax = pre["step"], synth.TF_VMIN, synth.TF_VMAX
    outs, nss, grads = [], [], []
    for c in cams:
        tgt, _ = P.render(vol, c, hidden, vmin, vmax, step, 2.0)
        img, ns = P.render(vol, c, tf, vmin, vmax, step, 2.0)
        outs.append(img)
        nss.append(ns)
        grads.append(2.0 * (img - tgt))
    gtf, gvox = P.render_backward_views(vol, cams, tf, vmin, vmax, step, outs, nss, grads, 2.0)
    torch.cuda.synchronize()
    assert L.vr_volume_info(vol.handle)["scratch_bytes"] >= 16 * n ** 3, \
        "the dense views should have taken the quad scratch"
    # tolerance of "at an interval end", in table entries
    grad = max(float(np.abs(np.diff(crop_np, axis=a)).max()) for a in range(3))
    eps_u = (255.0 / (vmax - vmin)) * (grad * np.sqrt(3.0) * 1e-5 + 4e-7 * float(np.abs(crop_np).max()))
    ref_tf = np.zeros((256, 4))
    ref_vox = np.zeros((n, n, n))
    kink = np.zeros((n, n, n))
    mag = np.zeros((n, n, n))
    for c, g, ns in zip(cams, grads, nss):
        o = oracle.render(crop_np, c, tf_np, vmin, vmax, step, 2.0)
        assert (o["n_used"] == ns.cpu().numpy()).all(), "sample counts differ from the oracle's"
        rt, rv, kv, mv = oracle.render_backward(crop_np, c, tf_np, vmin, vmax, step,
                                                g.cpu().numpy().astype(np.float64), ert=2.0, kink_eps=eps_u)
        ref_tf += rt
        ref_vox += rv
        kink += kv
        mag += mv
    ok, err, bound = _grad_close(gtf.cpu().numpy(), ref_tf)
    print("table gradient: worst err/bound %.3g" % float((err / bound).max()))
    assert ok.all(), "table gradient: %d of %d entries outside the 1e-3 rule" % (int((~ok).sum()), ok.size)
    gv = gvox.cpu().numpy().astype(np.float64)
    _, err, bound = _grad_close(gv, ref_vox)
    n_max = max(int(ns.max()) for ns in nss)
    fp32 = 2.0 * n_max * 2.0 ** -24 * mag
    allow = bound + kink + fp32
    ok = err <= allow
    print("voxel gradient: eps_u %.2g entries; %d of %d voxels touched by a sample at an interval end; "
          "%d outside the plain rule (%d within their kink bound); worst err/allowance %.3g" % (
              eps_u, int((kink > 0).sum()), kink.size, int((err > bound).sum()),
              int(((err > bound) & (err <= bound + kink)).sum()), float((err / allow).max())))
    for q in np.argwhere(~ok)[:20]:
        q = tuple(q)
        print("  voxel %s: got %.6g ref %.6g err %.3g bound %.3g kink %.3g fp32 %.3g" % (
            q, gv[q], ref_vox[q], err[q], bound[q], kink[q], fp32[q]))
    assert ok.all(), "voxel gradient: %d of %d entries outside the rule, worst at %s" % (
        int((~ok).sum()), ok.size, np.unravel_index(int(np.argmax(err / allow)), ref_vox.shape))
    assert (err <= bound).mean() > 0.99, "the plain 1e-3 rule should hold for almost every voxel"
    assert (kink > 0).mean() < 0.5, "too many voxels at an interval end for the check to mean much"
    vol.close()
