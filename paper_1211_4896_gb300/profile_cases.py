"""Small, self-contained cases for profiling one kernel launch with ncu
(inputs larger than L2, a few GB on the device at most):

  python -m paper_1211_4896_gb300.profile_cases fwd    # 512^3 f32, 4 orbit views at 960x540, step 1, ERT 0.99
  python -m paper_1211_4896_gb300.profile_cases fwd16  # the same views of the cube stored as f16
  python -m paper_1211_4896_gb300.profile_cases views16 # 512^3 f16 at 1920x1080: an axis view (0 deg) and an
                                                       # oblique one (45 deg), forward only, each rendered twice
  python -m paper_1211_4896_gb300.profile_cases views32 # the same views of the cube stored f32
  python -m paper_1211_4896_gb300.profile_cases bat    # the same 4 views in one batched call, f32
  python -m paper_1211_4896_gb300.profile_cases bwd    # 256^3 f32, 2 views at 512^2, step 0.5, table = ramp + 5% noise
  python -m paper_1211_4896_gb300.profile_cases bwd512 # the 512^3 differentiation workload (1024^2, step 0.5):
                                                       # backward of a z-view and an x-view, direct reductions
                                                       # then through the quad scratch (4 bwd launches, 2 gathers)
  python -m paper_1211_4896_gb300.profile_cases stats  # 512^3 f32: moments, 256-bin histogram, median (twice)
  python -m paper_1211_4896_gb300.profile_cases skip   # the fwd views with a table transparent below v = 6,
                                                       # plain then with empty-space skipping

The fwd/fwd16/bwd cases render each view forward then backward on cuda:0,
so capture the kernel of interest with -k and -c.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def case_fwd(store="f32"):
    import torch
    import synth
    import paper_1211_4896_gb300 as P
    dev = torch.device("cuda")
    dims = (512, 512, 512)
    vol = P.Volume(synth.hi_cube(dims, 250, 25, 9, device=dev), store)
    tf = torch.from_numpy(synth.tf_ramp(256)).to(dev)
    ns = None
    for c in synth.orbit_cameras(dims, 4, 40.0, 960, 540, start_deg=20.0):
        img, ns = P.render(vol, c, tf, -3.0, 50.0, 1.0, 0.99)
        P.render_backward(vol, c, tf, -3.0, 50.0, 1.0, img, ns, torch.randn_like(img), 0.99)
    torch.cuda.synchronize()
    print("ok", int(ns.sum()))


def case_views(store="f16"):
    import torch
    import synth
    import paper_1211_4896_gb300 as P
    dev = torch.device("cuda")
    dims = (512, 512, 512)
    vol = P.Volume(synth.hi_cube(dims, 250, 25, 9, device=dev), store)
    tf = torch.from_numpy(synth.tf_ramp(256)).to(dev)
    ns = None
    total = 0
    for c in synth.orbit_cameras(dims, 8, 40.0, 1920, 1080)[:2]:       # 0 and 45 degrees
        P.render(vol, c, tf, -3.0, 50.0, 1.0, 0.99)                       # builds the copy it reads
        img, ns = P.render(vol, c, tf, -3.0, 50.0, 1.0, 0.99)
        total += int(ns.sum())
    torch.cuda.synchronize()
    print("ok", total)


def case_bat():
    import torch
    import synth
    import paper_1211_4896_gb300 as P
    dev = torch.device("cuda")
    dims = (512, 512, 512)
    vol = P.Volume(synth.hi_cube(dims, 250, 25, 9, device=dev), "f32")
    tf = torch.from_numpy(synth.tf_ramp(256)).to(dev)
    jobs = [dict(vol=vol, cam=c, tf=tf, vmin=-3.0, vmax=50.0, step=1.0, ert=0.99,
                 out=torch.empty((540, 960, 4), device=dev),
                 nsamples=torch.empty((540, 960), device=dev, dtype=torch.int32))
            for c in synth.orbit_cameras(dims, 4, 40.0, 960, 540, start_deg=20.0)]
    for _ in range(2):
        P.render_batched(jobs)
    torch.cuda.synchronize()
    print("ok", sum(int(j["nsamples"].sum()) for j in jobs))


def case_bwd():
    import torch
    import synth
    import paper_1211_4896_gb300 as P
    dev = torch.device("cuda")
    dims = (256, 256, 256)
    vol = P.Volume(synth.hi_cube(dims, 160, 0, 5, device=dev), "f32")
    hidden = torch.from_numpy(synth.tf_ramp(256)).to(dev)
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    tf = (hidden + 0.05 * torch.rand(hidden.shape, device=dev, generator=g)).clamp(0, 1).contiguous()
    ns = None
    for c in synth.orbit_cameras(dims, 2, 40.0, 512, 512, start_deg=20.0):
        img, ns = P.render(vol, c, tf, -3.0, 50.0, 0.5, 2.0)
        P.render_backward(vol, c, tf, -3.0, 50.0, 0.5, img, ns, torch.randn_like(img), 2.0)
    torch.cuda.synchronize()
    print("ok", int(ns.sum()))


def case_bwd512():
    import torch
    import synth
    import paper_1211_4896_gb300 as P
    dev = torch.device("cuda")
    pre = synth.preset_diff_512()
    vol = P.Volume(synth.hi_cube(pre["dims"], pre["n_blobs"], pre["n_disks"], pre["seed"], device=dev), "f32")
    torch.cuda.empty_cache()
    hidden = torch.from_numpy(synth.tf_ramp(256)).to(dev)
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    tf = (hidden + 0.05 * torch.rand(hidden.shape, device=dev, generator=g)).clamp(0, 1).contiguous()
    views = []
    for c in pre["cameras"][:2]:              # 0 deg (along z) and 90 deg (along x)
        img, ns = P.render(vol, c, tf, synth.TF_VMIN, synth.TF_VMAX, pre["step"], 2.0)
        views.append((c, img, ns, torch.randn_like(img)))
    gvox = torch.empty(vol.shape, device=dev)
    for mode in ("direct", "scratch"):
        for c, img, ns, gr in views:
            P.render_backward(vol, c, tf, synth.TF_VMIN, synth.TF_VMAX, pre["step"], img, ns, gr, 2.0,
                              grad_vox=gvox, vox_reduce=mode)
    torch.cuda.synchronize()
    print("ok", sum(int(v[2].sum()) for v in views))


def case_skip():
    import numpy as np
    import torch
    import synth
    import paper_1211_4896_gb300 as P
    dev = torch.device("cuda")
    dims = (512, 512, 512)
    vol = P.Volume(synth.hi_cube(dims, 250, 25, 9, device=dev), "f32")
    v = -3.0 + 53.0 * np.arange(256) / 255
    t = (v + 3.0) / 53.0
    a = np.where(v < 6.0, 0.0, 0.02 + 0.2 * (v - 6.0) / 44.0)
    tf = torch.from_numpy(np.stack([t, t * t, 1 - t, a], 1).astype(np.float32)).to(dev)
    for flag in (False, True):
        for c in synth.orbit_cameras(dims, 4, 40.0, 960, 540, start_deg=20.0):
            img, ns = P.render(vol, c, tf, -3.0, 50.0, 1.0, 0.99, skip_empty=flag)
    torch.cuda.synchronize()
    print("ok", int(ns.sum()))


def case_stats():
    import torch
    import synth
    import paper_1211_4896_gb300 as P
    dev = torch.device("cuda")
    vol = P.Volume(synth.hi_cube((512, 512, 512), 250, 25, 9, device=dev), "f32")
    for _ in range(2):
        m = P.moments(vol)
        h = P.histogram(vol, m["min"], m["max"], 256)
        med = P.median(vol)
    torch.cuda.synchronize()
    print("ok", m["count"], int(h.sum()), med)


if __name__ == "__main__":
    from paper_1211_4896_gb300 import build
    build.build()
    {"fwd": case_fwd, "fwd16": lambda: case_fwd("f16"), "bat": case_bat, "bwd": case_bwd, "bwd512": case_bwd512, "views16": case_views, "views32": lambda: case_views("f32"),
     "stats": case_stats, "skip": case_skip}[sys.argv[1] if len(sys.argv) > 1 else "fwd"]()
