"""The compulsory-traffic ceiling of the benchmark counts the distinct voxels
that the trilinear footprints of a view's composited samples touch
(bench.footprint_voxels).  Checked here on the CPU against a brute-force
count built from the oracle's own ray set-up (its voxel-space origin,
direction and entry parameter per pixel, and its per-pixel sample counts):
every sample's cell and its eight corners go into a Python set.  Covers a
perspective and an orthographic view, early termination (rays stopped
part-way), anisotropic sizes, and the slab-by-slab count the function uses
for grids too large for one bitmap."""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")


def _brute_force(dims, cam, step, n_used):
    nx, ny, nz = dims
    seen = set()
    H, W = n_used.shape
    for j in range(H):
        for i in range(W):
            n = int(n_used[j, i])
            if n == 0:
                continue
            _, ov, dv, tin = oracle.ray((nz, ny, nx), cam, step, i, j)
            for k in range(n):
                p = ov + (tin + (k + 0.5) * step) * dv
                x0 = min(max(math.floor(p[0]), 0), nx - 2)
                y0 = min(max(math.floor(p[1]), 0), ny - 2)
                z0 = min(max(math.floor(p[2]), 0), nz - 2)
                for q in range(8):
                    seen.add((x0 + (q & 1), y0 + ((q >> 1) & 1), z0 + (q >> 2)))
    return len(seen)


@pytest.mark.parametrize("kind,ert", [("persp", 2.0), ("persp", 0.9), ("ortho", 2.0)])
def test_footprint_voxels_matches_brute_force(oracle_lib, kind, ert):
    import bench
    dims = (21, 17, 24)                                   # nx, ny, nz
    cube = synth.hi_cube(dims, n_blobs=4, n_disks=1, seed=5).numpy()
    tf = synth.tf_ramp(64, alpha_max=0.3)
    step = 0.7
    if kind == "persp":
        cam = synth.camera_random_persp(dims, seed=9, width=23, height=19)
    else:
        c = [0.5 * (d - 1) for d in dims]
        f = np.array([0.3, -0.2, 0.93])
        f = f / np.linalg.norm(f)
        eye = tuple(c[a] - 60.0 * f[a] for a in range(3))
        cam = synth.camera_ortho(eye, tuple(f), (0.0, 1.0, 0.0), 30.0, 22, 18)
    ref = oracle.render(cube, cam, tf, -3.0, 30.0, step, ert)
    n_used = ref["n_used"].astype(np.int32)
    assert n_used.max() > 0
    if ert < 1.0:                                         # some rays stop part-way
        full = np.array([[oracle.ray((dims[2], dims[1], dims[0]), cam, step, i, j)[0]
                          for i in range(n_used.shape[1])] for j in range(n_used.shape[0])])
        assert (n_used < full).any()
    want = _brute_force(dims, cam, step, n_used)
    ns = torch.from_numpy(n_used)
    assert bench.footprint_voxels(torch, dims, cam, step, ns) == want
    # counted in slabs of a few cell layers along z (the large-grid path)
    small = (dims[0] - 1) * (dims[1] - 1) * 3
    assert bench.footprint_voxels(torch, dims, cam, step, ns, max_bitmap_bytes=small) == want
