"""Torch-facing helpers over the C ABI: device memory and streams come from
PyTorch, the work is done by libvr.so.  Tensors must live on a CUDA device;
nothing here computes on the CPU."""
from __future__ import annotations

import numpy as np
import torch

from . import _lib as L

_DTYPES = {torch.float32: L.VR_F32, torch.float16: L.VR_F16, torch.bfloat16: L.VR_BF16}
_NAMES = {"f32": L.VR_F32, "f16": L.VR_F16, "bf16": L.VR_BF16}


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _need_cuda(t: torch.Tensor, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor (there is no CPU path)" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)


def _need(t: torch.Tensor, name: str, shape, dtype, device):
    """A caller-provided buffer the library reads or writes through a raw
    pointer: it must have exactly this shape and dtype and live on the
    volume's device (the C ABI cannot check sizes)."""
    _need_cuda(t, name)
    if tuple(t.shape) != tuple(shape) or t.dtype != dtype:
        raise ValueError("%s must be a %s tensor of shape %s (got %s %s)" % (name, dtype, tuple(shape), t.dtype,
                                                                            tuple(t.shape)))
    if t.device != torch.device(device):
        raise ValueError("%s must be on %s (got %s)" % (name, device, t.device))


class Volume:
    """A bricked, device-resident copy of a dense cube (nz, ny, nx), x fastest."""

    def __init__(self, cube: torch.Tensor, store_dtype="f32", brick: int = 0, origin=None, spacing=None,
                 stream=None):
        _need_cuda(cube, "cube")
        if cube.dim() != 3 or cube.dtype not in _DTYPES:
            raise ValueError("cube must be a 3D float32/float16/bfloat16 tensor (nz, ny, nx)")
        self.src_dtype = _DTYPES[cube.dtype]
        self.store_dtype = _NAMES[store_dtype] if isinstance(store_dtype, str) else int(store_dtype)
        nz, ny, nx = cube.shape
        self.dims = (nx, ny, nz)
        self.shape = (nz, ny, nx)
        self.device = cube.device
        self.origin = tuple(origin) if origin is not None else (0.0, 0.0, 0.0)
        self.spacing = tuple(spacing) if spacing is not None else (1.0, 1.0, 1.0)
        with torch.cuda.device(cube.device):
            self.handle = L.vr_volume_create(cube.data_ptr(), self.src_dtype, self.store_dtype, self.dims,
                                             self.origin, self.spacing, brick, _stream(stream))
        self.info = L.vr_volume_info(self.handle)

    def rebrick(self, brick: int, stream=None) -> "Volume":
        """A new Volume with the same voxels in bricks of `brick` (16, 32 or
        64), built on the device from this one's bricks."""
        out = Volume.__new__(Volume)
        for k in ("src_dtype", "store_dtype", "dims", "shape", "device", "origin", "spacing"):
            setattr(out, k, getattr(self, k))
        with torch.cuda.device(self.device):
            out.handle = L.vr_volume_rebrick(self.handle, int(brick), _stream(stream))
        out.info = L.vr_volume_info(out.handle)
        return out

    def update(self, cube: torch.Tensor, stream=None):
        _need_cuda(cube, "cube")
        if tuple(cube.shape) != self.shape or _DTYPES.get(cube.dtype) != self.src_dtype:
            raise ValueError("update needs the same shape and dtype as at creation")
        L.vr_volume_update(self.handle, cube.data_ptr(), self.src_dtype, _stream(stream))

    def close(self):
        if getattr(self, "handle", None):
            L.vr_volume_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _params(tf: torch.Tensor, vmin, vmax, step, ert, bg, filter, mode=L.VR_MODE_COMPOSITE, minimap=None,
            region=(1, 1, 1), skip_empty=False):
    _need_cuda(tf, "tf")
    if tf.dtype != torch.float32 or tf.dim() != 2 or tf.shape[1] != 4:
        raise ValueError("tf must be a (K, 4) float32 CUDA tensor")
    mm = None
    if mode == L.VR_MODE_SIGMA:
        if minimap is None:
            raise ValueError("mode VR_MODE_SIGMA needs the volume's minimap (see minimap())")
        _need_cuda(minimap, "minimap")
        if minimap.dtype != torch.float32 or minimap.dim() != 4 or minimap.shape[3] != 2:
            raise ValueError("minimap must be the (mz, my, mx, 2) float32 tensor of minimap()")
        mm = minimap.data_ptr()
    return L.make_params(tf.data_ptr(), tf.shape[0], vmin, vmax, step, ert, bg, filter, mode, mm, region,
                         skip_empty)


def render(vol: Volume, cam: dict, tf: torch.Tensor, vmin: float, vmax: float, step: float, ert: float = 2.0,
           bg=(0.0, 0.0, 0.0, 0.0), filter: int = L.VR_FILTER_SOFTWARE, want_nsamples: bool = True,
           out: torch.Tensor | None = None, nsamples: torch.Tensor | None = None, stream=None,
           mode: int = L.VR_MODE_COMPOSITE, minimap: torch.Tensor | None = None, region=(1, 1, 1),
           skip_empty: bool = False):
    """Forward render; returns (rgba (H, W, 4) float32, nsamples (H, W) int32 or None).
    mode: VR_MODE_COMPOSITE, VR_MODE_MIP, or VR_MODE_SIGMA with the volume's
    `minimap` (from minimap(vol, region)) and its `region`.  skip_empty: skip
    bricks that the table makes fully transparent (same result)."""
    H, W = int(cam["height"]), int(cam["width"])
    if out is None:
        out = torch.empty((H, W, 4), device=vol.device, dtype=torch.float32)
    _need(out, "out", (H, W, 4), torch.float32, vol.device)
    if want_nsamples and nsamples is None:
        nsamples = torch.empty((H, W), device=vol.device, dtype=torch.int32)
    if want_nsamples:
        _need(nsamples, "nsamples", (H, W), torch.int32, vol.device)
    if mode == L.VR_MODE_SIGMA and minimap is not None:
        nz, ny, nx = vol.shape
        m = [-(-n // int(r)) for n, r in zip((nx, ny, nz), region)]
        _need(minimap, "minimap", (m[2], m[1], m[0], 2), torch.float32, vol.device)
    p = _params(tf, vmin, vmax, step, ert, bg, filter, mode, minimap, region, skip_empty)
    L.vr_render(vol.handle, L.make_camera(cam), p, out.data_ptr(),
                nsamples.data_ptr() if (want_nsamples and nsamples is not None) else None, _stream(stream))
    return out, (nsamples if want_nsamples else None)


def render_backward(vol: Volume, cam: dict, tf: torch.Tensor, vmin, vmax, step, rgba, nsamples, grad_rgba,
                    ert: float = 2.0, bg=(0.0, 0.0, 0.0, 0.0), want_vox: bool = True, grad_tf=None, grad_vox=None,
                    accumulate: bool = False, filter: int = L.VR_FILTER_SOFTWARE, stream=None,
                    vox_reduce: str | None = None):
    """Adjoint: returns (grad_tf (K, 4) float64, grad_vox (nz, ny, nx) float32 or None).
    vox_reduce: None (the library picks), "direct" (reductions straight into
    grad_vox) or "scratch" (through the 16-byte-per-voxel quad scratch)."""
    H, W = int(cam["height"]), int(cam["width"])
    _need(rgba, "rgba", (H, W, 4), torch.float32, vol.device)
    _need(nsamples, "nsamples", (H, W), torch.int32, vol.device)
    _need(grad_rgba, "grad_rgba", (H, W, 4), torch.float32, vol.device)
    grad_tf, grad_vox = _grad_outputs(vol, tf, want_vox, grad_tf, grad_vox)
    p = _params(tf, vmin, vmax, step, ert, bg, filter)
    L.vr_render_backward(vol.handle, L.make_camera(cam), p, rgba.data_ptr(), nsamples.data_ptr(),
                         grad_rgba.data_ptr(), grad_tf.data_ptr(), grad_vox.data_ptr() if want_vox else None,
                         (L.VR_GRAD_ACCUMULATE if accumulate else 0) | _VOX_REDUCE[vox_reduce], _stream(stream))
    return grad_tf, (grad_vox if want_vox else None)


_VOX_REDUCE = {None: 0, "direct": L.VR_GRAD_DIRECT, "scratch": L.VR_GRAD_SCRATCH}


def _grad_outputs(vol: Volume, tf: torch.Tensor, want_vox: bool, grad_tf, grad_vox):
    if grad_tf is None:
        grad_tf = torch.empty(tuple(tf.shape), device=vol.device, dtype=torch.float64)
    _need(grad_tf, "grad_tf", tuple(tf.shape), torch.float64, vol.device)
    if want_vox:
        if grad_vox is None:
            grad_vox = torch.empty(vol.shape, device=vol.device, dtype=torch.float32)
        _need(grad_vox, "grad_vox", vol.shape, torch.float32, vol.device)
    return grad_tf, grad_vox


def render_backward_views(vol: Volume, cams, tf: torch.Tensor, vmin, vmax, step, rgbas, nsamples, grad_rgbas,
                          ert: float = 2.0, bg=(0.0, 0.0, 0.0, 0.0), want_vox: bool = True, grad_tf=None,
                          grad_vox=None, accumulate: bool = False, filter: int = L.VR_FILTER_SOFTWARE, stream=None,
                          vox_reduce: str | None = None):
    """Adjoint of a loss summed over several views in one call: returns
    (grad_tf (K, 4) float64, grad_vox (nz, ny, nx) float32 or None), equal to
    render_backward per view with accumulate after the first."""
    if not (len(cams) == len(rgbas) == len(nsamples) == len(grad_rgbas)) or not cams:
        raise ValueError("cams, rgbas, nsamples and grad_rgbas must be non-empty and of equal length")
    for q, cam in enumerate(cams):
        H, W = int(cam["height"]), int(cam["width"])
        _need(rgbas[q], "rgbas[%d]" % q, (H, W, 4), torch.float32, vol.device)
        _need(nsamples[q], "nsamples[%d]" % q, (H, W), torch.int32, vol.device)
        _need(grad_rgbas[q], "grad_rgbas[%d]" % q, (H, W, 4), torch.float32, vol.device)
    grad_tf, grad_vox = _grad_outputs(vol, tf, want_vox, grad_tf, grad_vox)
    views = [L.vr_grad_view(L.make_camera(c), r.data_ptr(), n.data_ptr(), g.data_ptr())
             for c, r, n, g in zip(cams, rgbas, nsamples, grad_rgbas)]
    p = _params(tf, vmin, vmax, step, ert, bg, filter)
    L.vr_render_backward_views(vol.handle, views, p, grad_tf.data_ptr(), grad_vox.data_ptr() if want_vox else None,
                               (L.VR_GRAD_ACCUMULATE if accumulate else 0) | _VOX_REDUCE[vox_reduce],
                               _stream(stream))
    return grad_tf, (grad_vox if want_vox else None)


def minimap(vol: Volume, region, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Statistical mini-map of the sigma-clipping transfer function: an
    (mz, my, mx, 2) float32 tensor of each region's mean and standard
    deviation (regions of region = (rx, ry, rz) voxels)."""
    nz, ny, nx = vol.shape
    m = [-(-n // int(r)) for n, r in zip((nx, ny, nz), region)]
    if out is None:
        out = torch.empty((m[2], m[1], m[0], 2), device=vol.device, dtype=torch.float32)
    _need(out, "out", (m[2], m[1], m[0], 2), torch.float32, vol.device)
    L.vr_minimap(vol.handle, region, out.data_ptr(), _stream(stream))
    return out


def profile(vol: Volume, cam: dict, step: float, i: int, j: int, max_values: int | None = None, stream=None):
    """3D spectrum tool: the values of the samples along pixel (i, j)'s ray.
    Returns a float32 CUDA tensor of the first min(n, max_values) values
    (max_values defaults to a bound on any ray's sample count)."""
    if max_values is None:
        nz, ny, nx = vol.shape
        diag = float(np.sqrt(sum(((n - 1) * s) ** 2 for n, s in zip((nx, ny, nz), vol.spacing))))
        max_values = int(diag / step) + 2
    values = torch.empty(max(1, max_values), device=vol.device, dtype=torch.float32)
    count = torch.zeros(1, device=vol.device, dtype=torch.int32)
    L.vr_profile(vol.handle, L.make_camera(cam), step, i, j, values.data_ptr(), max_values, count.data_ptr(),
                 _stream(stream))
    n = min(int(count.item()), max_values)
    return values[:n]


def render_subbox(vol: Volume, cam: dict, tf: torch.Tensor, vmin: float, vmax: float, step: float, cell_lo, cell_hi,
                  stream=None, global_dims=None, offset=None):
    """Sort-last partial render of the cells [cell_lo, cell_hi) (x, y, z):
    returns (partial (H, W, 4): premultiplied colour and transmittance,
    depth (H, W): distance of the first sample from the eye or inf, count
    (H, W)).  With global_dims and offset the volume holds the voxels
    [offset, offset + dims) of a grid of global_dims voxels (its origin is
    that of its own first voxel) and the cells are the whole grid's."""
    H, W = int(cam["height"]), int(cam["width"])
    partial = torch.empty((H, W, 4), device=vol.device, dtype=torch.float32)
    depth = torch.empty((H, W), device=vol.device, dtype=torch.float32)
    count = torch.empty((H, W), device=vol.device, dtype=torch.int32)
    p = _params(tf, vmin, vmax, step, 2.0, (0.0, 0.0, 0.0, 0.0), L.VR_FILTER_SOFTWARE)
    if global_dims is None and offset is None:
        L.vr_render_subbox(vol.handle, L.make_camera(cam), p, cell_lo, cell_hi, partial.data_ptr(), depth.data_ptr(),
                           count.data_ptr(), _stream(stream))
    else:
        L.vr_render_subbox_of(vol.handle, global_dims, offset, L.make_camera(cam), p, cell_lo, cell_hi,
                              partial.data_ptr(), depth.data_ptr(), count.data_ptr(), _stream(stream))
    return partial, depth, count


def composite(partials, depths, bg=(0.0, 0.0, 0.0, 0.0), stream=None) -> torch.Tensor:
    """Over-composite of partial images (from render_subbox) in per-pixel depth order."""
    if not partials or len(partials) != len(depths):
        raise ValueError("partials and depths must be non-empty and of equal length")
    H, W = depths[0].shape
    for q, (pt, d) in enumerate(zip(partials, depths)):
        _need(pt, "partials[%d]" % q, (H, W, 4), torch.float32, depths[0].device)
        _need(d, "depths[%d]" % q, (H, W), torch.float32, depths[0].device)
    out = torch.empty((H, W, 4), device=depths[0].device, dtype=torch.float32)
    L.vr_composite([p.data_ptr() for p in partials], [d.data_ptr() for d in depths], W, H, bg, out.data_ptr(),
                   _stream(stream))
    return out


def moments(vol: Volume, stream=None) -> dict:
    """Count, mean, population standard deviation, minimum and maximum of the
    non-NaN voxels (Section 4.2)."""
    out = torch.empty(5, device=vol.device, dtype=torch.float64)
    L.vr_moments(vol.handle, out.data_ptr(), _stream(stream))
    v = out.cpu().tolist()
    return dict(count=int(v[0]), mean=v[1], sd=v[2], min=v[3], max=v[4])


def histogram(vol: Volume, lo: float, hi: float, nbins: int, stream=None) -> torch.Tensor:
    """Counts of the voxel values in [lo, hi] in nbins equal bins (Section 4.1)."""
    counts = torch.empty(int(nbins), device=vol.device, dtype=torch.int64)
    L.vr_histogram(vol.handle, lo, hi, nbins, counts.data_ptr(), _stream(stream))
    return counts


def median(vol: Volume, stream=None) -> float:
    """The value of rank (n + 1) // 2 among the n non-NaN voxels (Section 4.3)."""
    out = torch.empty(1, device=vol.device, dtype=torch.float64)
    L.vr_median(vol.handle, out.data_ptr(), _stream(stream))
    return float(out.item())


class RenderFunction(torch.autograd.Function):
    """Differentiable render: inputs (cube, tf), output the RGBA image.  The
    volume handle must hold the bricked copy of ``cube`` (call vol.update
    after changing it).  Gradients come from the adjoint kernel."""

    @staticmethod
    def forward(ctx, cube, tf, vol, cam, vmin, vmax, step, ert, bg):
        img, ns = render(vol, cam, tf.detach().contiguous(), vmin, vmax, step, ert, bg)
        ctx.vol, ctx.cam, ctx.args = vol, cam, (vmin, vmax, step, ert, bg)
        ctx.want_vox = cube.requires_grad
        ctx.save_for_backward(tf.detach().contiguous(), img, ns)
        return img

    @staticmethod
    def backward(ctx, grad_img):
        tf, img, ns = ctx.saved_tensors
        vmin, vmax, step, ert, bg = ctx.args
        gtf, gvox = render_backward(ctx.vol, ctx.cam, tf, vmin, vmax, step, img, ns, grad_img.contiguous(),
                                    ert, bg, want_vox=ctx.want_vox)
        return (gvox if ctx.want_vox else None), gtf.to(tf.dtype), None, None, None, None, None, None, None


def render_diff(cube, tf, vol, cam, vmin, vmax, step, ert=2.0, bg=(0.0, 0.0, 0.0, 0.0)):
    return RenderFunction.apply(cube, tf, vol, cam, vmin, vmax, step, ert, bg)


def autotune_key(jobs) -> str:
    """Cache key of a job list for the batched autotuner: the device, the
    storage type and brick size, and every job's volume and image size."""
    import hashlib
    dev = torch.cuda.get_device_name(jobs[0]["vol"].device) if torch.cuda.is_available() else "cpu"
    parts = [dev, str(jobs[0]["vol"].store_dtype), str(jobs[0]["vol"].info["brick"])]
    for j in jobs:
        parts.append("%s:%dx%d" % ("x".join(map(str, j["vol"].shape[::-1])), int(j["cam"]["width"]),
                                   int(j["cam"]["height"])))
    return hashlib.sha1("|".join(parts).encode()).hexdigest()


def cached_tuning(key: str, tune, cache_path=None) -> dict:
    """Looks `key` up in the JSON file cache_path (else $VR_AUTOTUNE_CACHE;
    no cache when neither is set); on a miss calls tune() -> dict and stores
    its result (written to a temporary file, then renamed)."""
    import json
    import os
    path = cache_path or os.environ.get("VR_AUTOTUNE_CACHE")
    table = {}
    if path and os.path.exists(path):
        with open(path) as f:
            table = json.load(f)
        if key in table:
            return dict(table[key])
    best = dict(tune())
    if path:
        table[key] = best
        tmp = "%s.tmp%d" % (path, os.getpid())
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    return best


def autotune_batched(jobs, cache_path=None, stream=None) -> L.vr_batch_opts:
    """Ray-tile shape, CTAs per SM and warps per tile for this job list
    (vr_autotune_batched tries each and keeps the fastest), remembered across
    processes in the autotune cache (cache_path or $VR_AUTOTUNE_CACHE) under
    autotune_key; the entry records the volumes' brick size too."""
    def tune():
        cj = render_batched(jobs, use_graph=False, stream=stream)
        best = L.vr_autotune_batched(cj, L.vr_batch_opts(0, 0, 0, 0), _stream(stream))
        return {"tile_w": best.tile_w, "tile_h": best.tile_h, "ctas_per_sm": best.ctas_per_sm,
                "warps_per_tile": best.warps_per_tile, "brick": int(jobs[0]["vol"].info["brick"])}
    b = cached_tuning(autotune_key(jobs), tune, cache_path)
    return L.vr_batch_opts(1, b["tile_w"], b["tile_h"], b["ctas_per_sm"], b.get("warps_per_tile", 1))


def autotune_batched_bricks(jobs, brick_sizes=(16, 32, 64), cache_path=None, stream=None, reps: int = 3):
    """The batched autotuner over brick sizes as well: for each size the job
    list's volumes are re-bricked once (Volume.rebrick, kept on the source
    Volume for later calls), autotune_batched picks tile shape, CTAs per SM and
    warps per tile for it, and the size whose tuned graph call is fastest wins.
    Returns (opts, brick, jobs) with `jobs` rewritten onto the volumes of that
    brick size."""
    best = None
    s = _stream(stream)
    for b in brick_sizes:
        vj = []
        for j in jobs:
            v = j["vol"]
            if int(v.info["brick"]) != b:
                cache = v.__dict__.setdefault("_rebricked", {})
                if b not in cache:
                    cache[b] = v.rebrick(b, stream)
                v = cache[b]
            vj.append(dict(j, vol=v))
        opts = autotune_batched(vj, cache_path, stream)
        cj = render_batched(vj, opts=opts, stream=stream)              # plan + graph
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            L.vr_render_batched(cj, opts, s)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        if best is None or ms < best[0]:
            best = (ms, opts, b, vj)
    return best[1], best[2], best[3]


def render_batched(jobs, use_graph: bool = True, tile=(8, 4), ctas_per_sm: int = 0, stream=None,
                   opts: L.vr_batch_opts | None = None):
    """jobs: list of dicts with keys vol, cam, tf, vmin, vmax, step, ert, bg, out, nsamples (optional).
    Renders all of them in one persistent launch per brick layout their views read."""
    cj = []
    for j in jobs:
        p = _params(j["tf"], j["vmin"], j["vmax"], j["step"], j.get("ert", 2.0), j.get("bg", (0, 0, 0, 0)),
                    L.VR_FILTER_SOFTWARE)
        ns = j.get("nsamples")
        H, W = int(j["cam"]["height"]), int(j["cam"]["width"])
        _need(j["out"], "jobs[%d].out" % len(cj), (H, W, 4), torch.float32, j["vol"].device)
        if ns is not None:
            _need(ns, "jobs[%d].nsamples" % len(cj), (H, W), torch.int32, j["vol"].device)
        cj.append(L.vr_job(j["vol"].handle, L.make_camera(j["cam"]), p, j["out"].data_ptr(),
                           ns.data_ptr() if ns is not None else None))
    if opts is None:
        opts = L.vr_batch_opts(int(use_graph), int(tile[0]), int(tile[1]), int(ctas_per_sm))
    L.vr_render_batched(cj, opts, _stream(stream))
    return cj
