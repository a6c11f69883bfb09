"""Run by tests/test_gpu_bounds_check.py in a child process whose
VR_LIBRARY points at the bounds-check build: every kind of call on small
ragged volumes (three storage types, three brick sizes, rays that enter,
graze, start inside or miss the box, views that read every brick layout),
then vr_check on every volume must find no index outside its buffer."""
import sys

import numpy as np


def main():
    import torch
    import oracle
    import synth
    import paper_1211_4896_gb300 as P
    from paper_1211_4896_gb300 import _lib as L
    assert L.vr_bounds_checked(), "not the bounds-check build"
    dev = torch.device("cuda")
    s = int(torch.cuda.current_stream().cuda_stream)
    tf_np = synth.tf_random_pwl(seed=5, alpha_max=0.3)
    tf = torch.from_numpy(tf_np).to(dev)
    vols, calls = [], 0
    for dims, brick, store in [((23, 19, 30), 16, "f32"), ((40, 33, 17), 32, "f16"), ((35, 70, 21), 64, "bf16"),
                               ((66, 40, 52), 16, "f16"), ((2, 2, 2), 16, "f32")]:
        cube = synth.hi_cube(dims, n_blobs=3, n_disks=1, seed=sum(dims)).to(dev)
        vol = P.Volume(cube, store, brick=brick)
        vols.append(vol)
        cams = [synth.camera_random_persp(dims, seed=q, width=37, height=29) for q in range(4)]
        c = [0.5 * (d - 1) for d in dims]
        for f, u in (((0, 0, 1), (0, 1, 0)), ((0, 0, 1), (1, 0, 0)), ((0, 1, 0), (0, 0, 1)), ((1, 0, 0), (0, 0, 1))):
            eye = [c[a] - 3.0 * max(dims) * f[a] for a in range(3)]
            cams.append(synth.camera_ortho(eye, f, u, 1.2 * max(dims), 33, 31))
        cams.append(synth.camera_persp(tuple(c), (0.3, -0.2, 0.93), (0, 1, 0), 70.0, 24, 20))     # eye inside
        cams.append(synth.camera_ortho((c[0], c[1], -50.0), (0, 0, 1), (0, 1, 0), 0.01, 8, 8))  # one column
        graze = [c[0], float(dims[1] - 1), -40.0]
        cams.append(synth.camera_persp(graze, (0, 0, 1), (0, 1, 0), 10.0, 16, 16))              # grazing top face
        for cam in cams:
            for ert in (2.0, 0.9):
                img, ns = P.render(vol, cam, tf, -3.0, 30.0, 0.6, ert, (0.1, 0.2, 0.0, 0.3))
                calls += 1
            P.render(vol, cam, tf, -3.0, 30.0, 0.6, mode=P.VR_MODE_MIP)
            mm = P.minimap(vol, (5, 6, 7))
            P.render(vol, cam, tf, 0.0, 6.0, 0.6, 0.95, mode=P.VR_MODE_SIGMA, minimap=mm, region=(5, 6, 7))
            P.render(vol, cam, tf, -3.0, 30.0, 0.6, 0.95, skip_empty=True)
            g = torch.randn(img.shape, device=dev)
            for mode in ("direct", "scratch"):
                P.render_backward(vol, cam, tf, -3.0, 30.0, 0.6, img, ns, g, 0.9, (0.1, 0.2, 0.0, 0.3),
                                  vox_reduce=mode)
            P.profile(vol, cam, 0.6, cam["width"] // 2, cam["height"] // 2)
            calls += 6
        # staged filter and multi-view backward
        if store == "f32":
            img, ns = P.render(vol, cams[0], tf, -3.0, 30.0, 0.6, 2.0, filter=L.VR_FILTER_SOFTWARE_STAGED)
            P.render_backward(vol, cams[0], tf, -3.0, 30.0, 0.6, img, ns, torch.randn_like(img), 2.0,
                              filter=L.VR_FILTER_SOFTWARE_STAGED)
        imgs, nss = zip(*[P.render(vol, cam, tf, -3.0, 30.0, 0.6, 2.0) for cam in cams[:5]])
        P.render_backward_views(vol, cams[:5], tf, -3.0, 30.0, 0.6, list(imgs), list(nss),
                                [torch.randn_like(i) for i in imgs], 2.0)
        # sort-last: whole volume and sub-cube volumes
        cells = [d - 1 for d in dims]
        from paper_1211_4896_gb300.sortlast import split_cells, sub_cube
        parts = min(4, min(cells))
        boxes = split_cells(cells, parts) if parts >= 1 else []
        pieces, depths = [], []
        for lo, hi in boxes:
            part, depth, _ = P.render_subbox(vol, cams[1], tf, -3.0, 30.0, 0.6, lo, hi)
            sv = P.Volume(sub_cube(cube, lo, hi), store, brick=brick, origin=tuple(float(q) for q in lo))
            vols.append(sv)
            P.render_subbox(sv, cams[1], tf, -3.0, 30.0, 0.6, lo, hi, global_dims=dims, offset=lo)
            pieces.append(part)
            depths.append(depth)
        if pieces:
            P.composite(pieces, depths)
        # batched (graph) over every view, and the allocation-free form
        jobs = [dict(vol=vol, cam=cam, tf=tf, vmin=-3.0, vmax=30.0, step=0.6, ert=0.95,
                     out=torch.empty((cam["height"], cam["width"], 4), device=dev),
                     nsamples=torch.empty((cam["height"], cam["width"]), device=dev, dtype=torch.int32))
                for cam in cams]
        P.render_batched(jobs, use_graph=True)
        P.render_batched(jobs, use_graph=True)
        cj = P.render_batched(jobs, use_graph=False)
        L.vr_render_batched_noalloc(cj, 8, 4, s)
        P.moments(vol)
        P.histogram(vol, -3.0, 30.0, 64)
        P.median(vol)
        calls += 8
        # the checked build still renders correctly
        if store == "f32" and dims[0] > 2:
            img, ns = P.render(vol, cams[0], tf, -3.0, 30.0, 0.6, 2.0)
            ref = oracle.render(cube.cpu().numpy(), cams[0], tf_np, -3.0, 30.0, 0.6, 2.0)
            assert np.abs(img.cpu().numpy() - ref["rgba"]).max() <= 1e-4
    torch.cuda.synchronize()
    for v in vols:
        L.vr_check(v.handle, s)          # raises VRError on a caught out-of-range index
    for v in vols:
        v.close()
    print("bounds-check ok: %d volumes, %d+ calls" % (len(vols), calls))


if __name__ == "__main__":
    sys.exit(main())
