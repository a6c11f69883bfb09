"""Bounds checking in the kernels (a stand-in for a memory checker): the
self-test's caught index is reported by vr_check once, in the normal build;
and the bounds-check build (-DVR_BOUNDS_CHECK, every gather, scatter,
table-bin, per-brick and mini-map index tested before the access) runs every
kind of call on ragged volumes without catching an index outside its
buffer."""
import os
import subprocess
import sys

import pytest

from tests.helpers import cuda_or_skip

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_caught_index_is_reported_once():
    torch = cuda_or_skip()
    import synth
    import paper_1211_4896_gb300 as P
    from paper_1211_4896_gb300 import _lib as L
    vol = P.Volume(synth.hi_cube((12, 12, 12), 1, 0, 3).cuda(), "f32")
    s = int(torch.cuda.current_stream().cuda_stream)
    try:
        L.vr_check(vol.handle, s)
        L.vr_selftest_bounds(vol.handle, s)
        with pytest.raises(L.VRError) as e:
            L.vr_check(vol.handle, s)
        assert e.value.status == L.VR_ERR_INTERNAL
        L.vr_check(vol.handle, s)
    finally:
        vol.close()


def test_bounds_check_build_finds_nothing():
    cuda_or_skip()
    from paper_1211_4896_gb300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, VR_LIBRARY=lib, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-m", "tests._bounds_cases"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "bounds-check ok" in r.stdout
