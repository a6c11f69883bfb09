"""Failure detection without a GPU fault: a bounded device-side wait that runs
out (a barrier that nothing completes) records a timeout in the volume's
status word; vr_check reports it once (VR_ERR_TIMEOUT) and clears it, and
the device and the volume stay usable.  Host-side validation errors are
covered without a GPU in test_abi.py."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import TOL_F32, compare, cuda_or_skip

pytestmark = pytest.mark.gpu


def test_bounded_wait_timeout_is_reported_once_and_the_device_stays_usable():
    torch = cuda_or_skip()
    import paper_1211_4896_gb300 as P
    from paper_1211_4896_gb300 import _lib as L
    dims = (24, 20, 28)
    cube = synth.hi_cube(dims, 3, 0, 5).numpy()
    vol = P.Volume(torch.from_numpy(cube).cuda(), "f32")
    s = int(torch.cuda.current_stream().cuda_stream)
    tf_np = synth.tf_random_pwl(seed=2, alpha_max=0.3)
    tf = torch.from_numpy(tf_np).cuda()
    try:
        L.vr_check(vol.handle, s)                                # clean
        L.vr_selftest_timeout(vol.handle, s)
        with pytest.raises(L.VRError) as e:
            L.vr_check(vol.handle, s)
        assert e.value.status == L.VR_ERR_TIMEOUT
        L.vr_check(vol.handle, s)                                # reported once, then cleared
        cam = synth.camera_random_persp(dims, seed=4, width=32, height=24)
        img, ns = P.render(vol, cam, tf, -3.0, 30.0, 0.5)        # the context is intact
        torch.cuda.synchronize()
        compare(img.cpu().numpy(), ns.cpu().numpy(), oracle.render(cube, cam, tf_np, -3.0, 30.0, 0.5), TOL_F32)
        # a timeout on one volume does not touch another volume's status
        other = P.Volume(torch.from_numpy(cube).cuda(), "f32")
        try:
            L.vr_selftest_timeout(vol.handle, s)
            L.vr_check(other.handle, s)
            with pytest.raises(L.VRError):
                L.vr_check(vol.handle, s)
        finally:
            other.close()
    finally:
        vol.close()
