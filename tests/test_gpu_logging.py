"""VR_LOG=1: the library writes one line on stderr per launch decision (the
layout a view reads and when a brick or texture-layer copy is built, the forward's grid, the
batch's layout groups and grids, the backward's voxel-gradient form);
without it, nothing."""
import os
import subprocess
import sys

import pytest

from tests.helpers import cuda_or_skip

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import torch, synth, paper_1211_4896_gb300 as P
dims = (40, 36, 44)
vol = P.Volume(synth.hi_cube(dims, 3, 0, 1).cuda(), "f32")
tf = torch.from_numpy(synth.tf_ramp(64)).cuda()
c = [0.5 * (d - 1) for d in dims]
cams = [synth.camera_persp([c[0], c[1], c[2] - 150], (0, 0, 1), up, 25.0, 64, 64) for up in ((0, 1, 0), (1, 0, 0))]
img, ns = P.render(vol, cams[1], tf, -3.0, 30.0, 0.5)
P.render_backward(vol, cams[1], tf, -3.0, 30.0, 0.5, img, ns, torch.randn_like(img))
P.render_batched([dict(vol=vol, cam=cam, tf=tf, vmin=-3.0, vmax=30.0, step=0.5, out=torch.empty_like(img))
                  for cam in cams], use_graph=False)
import os
os.environ["VR_TEX_LAYERS"] = "0"          # the brick copies
P.render(vol, cams[1], tf, -3.0, 30.0, 0.5)
torch.cuda.synchronize()
vol.close()
print("done")
"""


def _run(log):
    env = dict(os.environ, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    env.pop("VR_LOG", None)
    env.pop("VR_TEX_LAYERS", None)
    if log:
        env["VR_LOG"] = "1"
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "done" in r.stdout, r.stderr[-2000:]
    return [line for line in r.stderr.splitlines() if line.startswith("vr: ")]


def test_log_lines_only_with_vr_log():
    cuda_or_skip()
    lines = _run(True)
    text = "\n".join(lines)
    assert "prefers texture layers across axis 2; building them" in text
    assert "forward 64x64: layout order 2 texture layers" in text
    assert "backward of 1 view(s): voxel gradient through the quad scratch" in text
    assert "batch, brick layout 11: 2 job(s)" in text
    assert "prefers brick copy 1 (plain); building it" in text
    assert "forward 64x64: layout order 1," in text
    assert _run(False) == []
