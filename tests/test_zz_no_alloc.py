"""The allocation-free batched entry point, vr_render_batched_noalloc.

Some callers cannot allocate device memory while they render: work recorded
into a CUDA stream capture (a cudaMalloc would invalidate the capture), or a
service that runs inside a fixed device-memory budget owned by another
allocator.  For them the library keeps the batch descriptors and the work
counter in one static device array instead of allocating them per job list.
This file checks that the variant renders exactly what vr_render_batched
renders, on two calls in a row (the second call finds the first call's
contents in the shared array), and that it refuses more jobs than the array
holds.  It is collected last so that a failure here cannot hide others.
"""
import numpy as np
import pytest

import synth
from tests.helpers import TOL_F32, cuda_or_skip

pytestmark = pytest.mark.gpu


def test_noalloc_batched_matches_vr_render_batched_twice():
    torch = cuda_or_skip()
    import paper_1211_4896_gb300 as P
    from paper_1211_4896_gb300 import _lib as L

    dev = torch.device("cuda")
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
            err = (ia - ib).abs().max().item()
            assert err <= TOL_F32, "call %d: max abs difference %.3g" % (call, err)

    too_many = [jobs_b[0]] * (L.VR_NOALLOC_MAX_JOBS + 1)
    with pytest.raises(L.VRError) as ei:
        L.vr_render_batched_noalloc(too_many, 8, 4, stream)
    assert ei.value.status == L.VR_ERR_INVALID_ARG and "exceeds the maximum" in str(ei.value)
    for vol, _ in vols:
        vol.close()
