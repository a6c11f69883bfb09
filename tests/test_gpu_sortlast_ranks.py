"""Sort-last across ranks with the GPU kernels (Sections 3.2 and 3.4): two
processes share the one GPU, each holding only its sub-cube of the volume
(its cells' voxels plus the one-voxel overlap) as a volume of its own, and
call the product's render_sortlast: each renders the partial image of its
cells, the gloo all-to-all (staged through host memory) hands band b of
every partial to rank b, each rank composites its band in depth order, and
the all-gather assembles the image on both ranks.  The image must equal the
FP64 oracle's whole render within 1e-4.  The two processes exchange only
through gloo on the host; no kernel of one waits on the other."""
import os
import socket
import sys

import numpy as np
import pytest

from tests.helpers import TOL_F32, cuda_or_skip

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _scene():
    import synth
    dims = (61, 47, 55)
    cube = synth.hi_cube(dims, n_blobs=6, n_disks=1, seed=23)
    cam = synth.camera_random_persp(dims, seed=31, width=70, height=53)
    tf = synth.tf_random_pwl(seed=12, alpha_max=0.3)
    return dims, cube, cam, tf


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist
    import paper_1211_4896_gb300 as P
    from paper_1211_4896_gb300 import sortlast
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dims, cube, cam, tf_np = _scene()
        lo, hi = sortlast.split_cells(tuple(d - 1 for d in dims), world)[rank]
        vol = P.Volume(sortlast.sub_cube(cube, lo, hi).to(dev), "f32", origin=tuple(float(q) for q in lo))
        tf = torch.from_numpy(tf_np).to(dev)
        image = sortlast.render_sortlast(vol, dims, lo, lo, hi, cam, tf, -3.0, 30.0, 0.6, bg=(0.1, 0.0, 0.2, 0.25))
        torch.cuda.synchronize()
        out[rank] = (image.device.type, image.cpu().numpy())
        vol.close()
    finally:
        dist.destroy_process_group()


def test_render_sortlast_two_ranks_on_gpu():
    cuda_or_skip()
    import torch.multiprocessing as mp
    import oracle
    from oracle.parity import MARGIN_N
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    dims, cube, cam, tf = _scene()
    ref = oracle.render(cube.numpy(), cam, tf, -3.0, 30.0, 0.6, 2.0, (0.1, 0.0, 0.2, 0.25))
    whole = ref["rgba"]
    assert whole[..., 3].max() > 0.1
    keep = ref["margin_n"] >= MARGIN_N          # a sample-count tie may move one sample between FP32 and FP64
    assert keep.mean() > 0.99
    for rank in range(world):
        kind, image = res[rank]
        assert kind == "cuda" and image.shape == whole.shape
        err = np.abs(image.astype(np.float64) - whole)[keep].max()
        assert err <= TOL_F32, "rank %d: max abs error %.3g" % (rank, err)
        np.testing.assert_array_equal(image, res[0][1])
