"""Sort-last across ranks, host side (Sections 3.2 and 3.4), on CPU with
gloo: every rank renders the partial image of its own box of cells (here
with the FP64 oracle, standing in for the GPU sub-box kernel), the
all-to-all exchange hands band b of every partial to rank b, each rank
composites its band in depth order (the oracle's composite), and the
all-gather assembles the image, which must equal the oracle's whole render.
Also the partition helpers: the boxes tile the grid of cells exactly."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _scene(world):
    import oracle
    import synth
    dims = (26, 22, 30)
    cube = synth.hi_cube(dims, n_blobs=4, n_disks=1, seed=11).numpy()
    cam = synth.camera_random_persp(dims, seed=3 + world, width=28, height=23)
    tf = synth.tf_random_pwl(seed=9, alpha_max=0.35)
    return oracle, cube, cam, tf


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist
    from paper_1211_4896_gb300 import sortlast
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        oracle, cube, cam, tf = _scene(world)
        nz, ny, nx = cube.shape
        lo, hi = sortlast.split_cells((nx - 1, ny - 1, nz - 1), world)[rank]
        ref = oracle.render_subbox(cube, cam, tf, -3.0, 30.0, 0.6, lo, hi)
        partial = torch.from_numpy(ref["partial"])
        depth = torch.from_numpy(ref["depth"])
        parts, depths = sortlast.exchange_bands(partial, depth)
        # the pieces are the other ranks' rows of this band, bit for bit
        mine = dist.get_rank()
        r0, r1 = sortlast.band_rows(cam["height"], world)[mine]
        everyone = [torch.empty_like(partial) for _ in range(world)]
        dist.all_gather(everyone, partial)
        ok = all(torch.equal(parts[q], everyone[q][r0:r1]) for q in range(world))
        band = torch.from_numpy(oracle.composite([p.numpy() for p in parts], [d.numpy() for d in depths],
                                                 bg=(0.1, 0.0, 0.2, 0.25)))
        image = sortlast.gather_bands(band, cam["height"])
        out[rank] = (ok, image.numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sortlast_exchange_gloo(world):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    oracle, cube, cam, tf = _scene(world)
    whole = oracle.render(cube, cam, tf, -3.0, 30.0, 0.6, 2.0, (0.1, 0.0, 0.2, 0.25))["rgba"]
    assert whole[..., 3].max() > 0.1
    for rank in range(world):
        ok, image = res[rank]
        assert ok
        assert image.shape == whole.shape
        np.testing.assert_allclose(image, whole, rtol=0, atol=1e-12)
        np.testing.assert_array_equal(image, res[0][1])


@pytest.mark.parametrize("cells,parts", [((25, 21, 29), 1), ((25, 21, 29), 2), ((25, 21, 29), 6),
                                         ((1023, 1023, 1023), 8), ((40, 7, 9), 12)])
def test_split_cells_tiles_the_grid(cells, parts):
    sys.path.insert(0, ROOT)
    from paper_1211_4896_gb300.sortlast import split_cells
    boxes = split_cells(cells, parts)
    assert len(boxes) == parts
    if np.prod(cells) <= 10 ** 6:
        owner = np.zeros(cells[::-1], dtype=np.int32)
        for lo, hi in boxes:
            assert all(0 <= l < h <= c for l, h, c in zip(lo, hi, cells))
            owner[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] += 1
        assert (owner == 1).all()
    else:
        assert sum(np.prod([h - l for l, h in zip(lo, hi)]) for lo, hi in boxes) == np.prod(cells)


def test_band_rows_and_sub_cube():
    pytest.importorskip("torch")
    import torch
    sys.path.insert(0, ROOT)
    from paper_1211_4896_gb300.sortlast import band_rows, sub_cube
    rows = band_rows(1080, 7)
    assert rows[0][0] == 0 and rows[-1][1] == 1080
    assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))
    assert max(r1 - r0 for r0, r1 in rows) - min(r1 - r0 for r0, r1 in rows) <= 1
    cube = torch.arange(5 * 6 * 7, dtype=torch.float32).reshape(5, 6, 7)
    sc = sub_cube(cube, (2, 1, 0), (5, 4, 3))
    assert tuple(sc.shape) == (4, 4, 4)                # cells [lo, hi) need voxels [lo, hi]
    assert torch.equal(sc, cube[0:4, 1:5, 2:6])
