"""Sort-last rendering over several GPUs (Sections 3.2 and 3.4): the cube is
split into sub-boxes of cells, one per rank; each rank keeps only its
sub-cube (its cells' voxels plus the one-voxel overlap the far cells need)
and renders the partial image of its cells at the whole render's sample
positions (`render_subbox` with `global_dims` / `offset`); one all-to-all
exchange then sends horizontal band b of every partial image (premultiplied
colour and transmittance, and the depth of its first sample) to rank b; each
rank over-composites the pieces of its band in per-pixel depth order
(`composite`), and an all-gather assembles the image on every rank.

One process per GPU; torch.distributed carries the exchange (NCCL between
GPUs).  The partition, the exchange and the gather take and return plain
tensors, so they run on any backend and device (with a backend whose
collectives take host tensors only, such as gloo, device tensors are staged
through host memory); the compositing arithmetic is `composite`'s."""
from __future__ import annotations

import torch
import torch.distributed as dist


def split_cells(cells, parts: int):
    """Splits the cell grid cells = (cx, cy, cz) into `parts` boxes [lo, hi)
    (x, y, z order): the factors of `parts` are spread over the axes, largest
    factor first to the longest remaining axis, and each axis is cut into
    near-equal runs.  Returns the boxes in x-fastest order of their grid
    position."""
    cells = [int(c) for c in cells]
    if parts < 1:
        raise ValueError("parts must be >= 1")
    factors, n, f = [], parts, 2
    while n > 1:
        while n % f == 0:
            factors.append(f)
            n //= f
        f += 1
    grid = [1, 1, 1]
    for f in sorted(factors, reverse=True):
        a = max(range(3), key=lambda q: cells[q] / grid[q])
        grid[a] *= f
    if any(g > c for g, c in zip(grid, cells)):
        raise ValueError("more parts than cells along an axis")
    edges = [[round(c * i / g) for i in range(g + 1)] for c, g in zip(cells, grid)]
    boxes = []
    for k in range(grid[2]):
        for j in range(grid[1]):
            for i in range(grid[0]):
                boxes.append(((edges[0][i], edges[1][j], edges[2][k]),
                              (edges[0][i + 1], edges[1][j + 1], edges[2][k + 1])))
    return boxes


def sub_cube(cube: torch.Tensor, lo, hi) -> torch.Tensor:
    """The voxels a box of cells [lo, hi) needs: [lo, hi] per axis (the
    cube is indexed (z, y, x))."""
    return cube[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1].contiguous()


def band_rows(height: int, parts: int):
    """Rows [r0, r1) of the `parts` horizontal bands of an image (near-equal)."""
    return [(height * b // parts, height * (b + 1) // parts) for b in range(parts)]


def _host_staged(group) -> bool:
    """True when the group's backend takes host tensors only (gloo)."""
    return dist.get_backend(group) == "gloo"


def exchange_bands(partial: torch.Tensor, depth: torch.Tensor, group=None):
    """All-to-all of horizontal bands: this rank sends band b of its partial
    image (H, W, 4) and depth (H, W) to rank b and receives its own band from
    every rank.  Returns (partials, depths): lists in rank order of
    (h, W, 4) and (h, W) tensors, h = this rank's band height."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    H, W = depth.shape
    rows = band_rows(H, world)
    sizes = [r1 - r0 for r0, r1 in rows]
    h = sizes[rank]
    dev = partial.device
    cdev = torch.device("cpu") if _host_staged(group) else dev
    out_p = torch.empty((world * h, W, 4), dtype=partial.dtype, device=cdev)
    out_d = torch.empty((world * h, W), dtype=depth.dtype, device=cdev)
    dist.all_to_all_single(out_p, partial.contiguous().to(cdev), [h] * world, sizes, group=group)
    dist.all_to_all_single(out_d, depth.contiguous().to(cdev), [h] * world, sizes, group=group)
    return list(out_p.to(dev).split(h)), list(out_d.to(dev).split(h))


def gather_bands(band: torch.Tensor, height: int, group=None) -> torch.Tensor:
    """All-gather of every rank's composited band (h_r, W, 4) into the
    (height, W, 4) image, on every rank."""
    world = dist.get_world_size(group)
    rows = band_rows(height, world)
    hmax = max(r1 - r0 for r0, r1 in rows)
    cdev = torch.device("cpu") if _host_staged(group) else band.device
    pad = torch.zeros((hmax,) + tuple(band.shape[1:]), dtype=band.dtype, device=cdev)
    pad[:band.shape[0]] = band.to(cdev)
    got = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(got, pad, group=group)
    return torch.cat([g[:r1 - r0] for g, (r0, r1) in zip(got, rows)]).to(band.device)


def render_sortlast(vol, global_dims, offset, cell_lo, cell_hi, cam: dict, tf: torch.Tensor, vmin: float,
                    vmax: float, step: float, bg=(0.0, 0.0, 0.0, 0.0), group=None) -> torch.Tensor:
    """One view rendered by all ranks of `group`: this rank's volume `vol`
    holds the voxels [offset, offset + dims) of the global_dims grid and
    renders the cells [cell_lo, cell_hi); the ranks' boxes must partition the
    grid's cells.  Returns the (H, W, 4) image on every rank."""
    from .api import composite, render_subbox
    partial, depth, _ = render_subbox(vol, cam, tf, vmin, vmax, step, cell_lo, cell_hi, global_dims=global_dims,
                                      offset=offset)
    parts, depths = exchange_bands(partial, depth, group)
    band = composite(parts, depths, bg=bg)
    return gather_bands(band, int(cam["height"]), group)
