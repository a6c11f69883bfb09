"""The allocation-free batched entry point, vr_render_batched_noalloc.

Some callers cannot allocate device memory while they render: a service that
runs inside a fixed device-memory budget, a process whose device memory is
handed out by another allocator's pool, or a frame loop that cannot take the
synchronisation a cudaMalloc may cause.  For them the library keeps the batch
descriptors and the work counters in one static device array instead of
allocating them per job list.  This file checks that the variant renders
exactly what vr_render_batched renders (the same kernels, so the same bits),
on two calls in a row (the second call finds the first call's contents in the
shared array), that a warmed-up call makes no library allocation at all, and
that it refuses more jobs than the array holds.  It is collected last so that
a failure here cannot hide others.
"""
import numpy as np
import pytest

import synth
from tests.helpers import cuda_or_skip

pytestmark = pytest.mark.gpu


def _jobs(torch, P, L, dev):
    rng = np.random.default_rng(7)
    vols, jobs_a, jobs_b, outs_a, outs_b = [], [], [], [], []
    for q in range(5):
        dims = tuple(int(x) for x in rng.integers(16, 48, size=3))
        vol = P.Volume(synth.hi_cube(dims, n_blobs=3, n_disks=1, seed=50 + q).to(dev), "f32")
        W, H = int(rng.integers(8, 60)), int(rng.integers(8, 50))
        cam = synth.camera_random_persp(dims, seed=60 + q, width=W, height=H)
        tf = torch.from_numpy(synth.tf_random_pwl(seed=70 + q)).to(dev)
        vols.append((vol, tf))
        for outs, jobs in ((outs_a, jobs_a), (outs_b, jobs_b)):
            img = torch.full((H, W, 4), -1.0, device=dev)
            ns = torch.full((H, W), -1, dtype=torch.int32, device=dev)
            outs.append((img, ns))
            jobs.append(L.vr_job(vol.handle, L.make_camera(cam),
                                 L.make_params(tf.data_ptr(), tf.shape[0], -3.0, 30.0, 0.6, 0.99 if q % 2 else 2.0),
                                 img.data_ptr(), ns.data_ptr()))
    return vols, jobs_a, jobs_b, outs_a, outs_b


def test_noalloc_batched_matches_vr_render_batched_twice():
    torch = cuda_or_skip()
    import paper_1211_4896_gb300 as P
    from paper_1211_4896_gb300 import _lib as L

    dev = torch.device("cuda")
    vols, jobs_a, jobs_b, outs_a, outs_b = _jobs(torch, P, L, dev)
    stream = int(torch.cuda.current_stream().cuda_stream)
    L.vr_render_batched(jobs_a, L.vr_batch_opts(0, 8, 4, 0), stream)
    for call in range(2):
        for img, ns in outs_b:
            img.fill_(-1.0)
            ns.fill_(-1)
        L.vr_render_batched_noalloc(jobs_b, 8, 4, stream)
        torch.cuda.synchronize()
        for (ia, na), (ib, nb) in zip(outs_a, outs_b):
            assert torch.equal(na, nb), "sample counts differ on call %d" % call
            assert torch.equal(ia, ib), "call %d: images differ (max abs %.3g)" % (call, (ia - ib).abs().max().item())

    too_many = [jobs_b[0]] * (L.VR_NOALLOC_MAX_JOBS + 1)
    with pytest.raises(L.VRError) as ei:
        L.vr_render_batched_noalloc(too_many, 8, 4, stream)
    assert ei.value.status == L.VR_ERR_INVALID_ARG and "exceeds the maximum" in str(ei.value)
    for vol, _ in vols:
        vol.close()


def test_noalloc_call_makes_no_library_allocation():
    """Every device allocation of the library goes through one function that
    vr_debug_fail_alloc(0) arms to fail the next time.  A warmed-up
    allocation-free call with the injection armed must succeed with the same
    bits, and leave the injection armed: the next allocating call (a volume
    creation) is the one that fails."""
    torch = cuda_or_skip()
    import paper_1211_4896_gb300 as P
    from paper_1211_4896_gb300 import _lib as L

    dev = torch.device("cuda")
    vols, jobs_a, jobs_b, outs_a, outs_b = _jobs(torch, P, L, dev)
    stream = int(torch.cuda.current_stream().cuda_stream)
    L.vr_render_batched(jobs_a, L.vr_batch_opts(0, 8, 4, 0), stream)
    L.vr_render_batched_noalloc(jobs_b, 8, 4, stream)          # first call: looks up the scratch address
    cube = synth.hi_cube((20, 20, 20), n_blobs=2, n_disks=0, seed=3).to(dev)
    torch.cuda.synchronize()
    try:
        L.vr_debug_fail_alloc(0)
        for img, ns in outs_b:
            img.fill_(-1.0)
            ns.fill_(-1)
        L.vr_render_batched_noalloc(jobs_b, 8, 4, stream)
        torch.cuda.synchronize()
        for (ia, na), (ib, nb) in zip(outs_a, outs_b):
            assert torch.equal(na, nb) and torch.equal(ia, ib)
        with pytest.raises(L.VRError) as ei:                   # the armed failure is still pending
            P.Volume(cube, "f32")
        assert ei.value.status == L.VR_ERR_OOM
    finally:
        L.vr_debug_fail_alloc(-1)
    for vol, _ in vols:
        vol.close()
