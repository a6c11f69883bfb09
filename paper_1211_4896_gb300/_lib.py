"""ctypes binding of libvr.so: one Python function per C entry point, same
names, argument marshalling only (every step of the rendering runs in the
library's CUDA kernels).  The structures mirror include/vr.h.

The library is loaded from the package's ``_build`` folder; if it is missing
an ImportError-like RuntimeError is raised -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
# VR_LIBRARY selects another build of the library (the bounds-check variant
# _build/libvr_checked.so); the default is the in-tree libvr.so.
LIB_PATH = os.environ.get("VR_LIBRARY") or os.path.join(_HERE, "_build", "libvr.so")

VR_OK, VR_ERR_INVALID_ARG, VR_ERR_UNSUPPORTED, VR_ERR_OOM, VR_ERR_CUDA, VR_ERR_TIMEOUT, VR_ERR_INTERNAL = \
    0, -1, -2, -3, -4, -5, -6
VR_F32, VR_F16, VR_BF16 = 0, 1, 2
VR_CAMERA_ORTHO, VR_CAMERA_PERSPECTIVE = 0, 1
VR_FILTER_SOFTWARE, VR_FILTER_TEXTURE, VR_FILTER_SOFTWARE_STAGED = 0, 1, 2
VR_GRAD_ACCUMULATE, VR_GRAD_DIRECT, VR_GRAD_SCRATCH = 1, 2, 4
VR_MODE_COMPOSITE, VR_MODE_MIP, VR_MODE_SIGMA = 0, 1, 2

STATUS_NAMES = {0: "VR_OK", -1: "VR_ERR_INVALID_ARG", -2: "VR_ERR_UNSUPPORTED", -3: "VR_ERR_OOM",
                -4: "VR_ERR_CUDA", -5: "VR_ERR_TIMEOUT", -6: "VR_ERR_INTERNAL"}


class vr_camera(C.Structure):
    _fields_ = [("kind", C.c_int), ("eye", C.c_double * 3), ("forward", C.c_double * 3),
                ("up", C.c_double * 3), ("fov_y_deg", C.c_double), ("ortho_height", C.c_double),
                ("width", C.c_int), ("height", C.c_int)]


class vr_params(C.Structure):
    _fields_ = [("tf_rgba", C.c_void_p), ("tf_size", C.c_int), ("vmin", C.c_float), ("vmax", C.c_float),
                ("step", C.c_float), ("ert_threshold", C.c_float), ("bg_rgba", C.c_float * 4),
                ("filter", C.c_int), ("mode", C.c_int), ("minimap", C.c_void_p), ("minimap_region", C.c_int * 3),
                ("skip_empty", C.c_int)]


class vr_volume_info_t(C.Structure):
    _fields_ = [("dims", C.c_int64 * 3), ("store_dtype", C.c_int), ("brick", C.c_int),
                ("bricks", C.c_int64 * 3), ("bytes", C.c_int64), ("dense_bytes", C.c_int64),
                ("copy_bytes", C.c_int64), ("copies", C.c_int), ("scratch_bytes", C.c_int64)]


class vr_job(C.Structure):
    _fields_ = [("vol", C.c_void_p), ("cam", vr_camera), ("params", vr_params),
                ("dev_rgba_out", C.c_void_p), ("dev_nsamples_out", C.c_void_p)]


class vr_grad_view(C.Structure):
    _fields_ = [("cam", vr_camera), ("rgba", C.c_void_p), ("nsamples", C.c_void_p), ("grad_rgba", C.c_void_p)]


class vr_batch_opts(C.Structure):
    _fields_ = [("use_graph", C.c_int), ("tile_w", C.c_int), ("tile_h", C.c_int), ("ctas_per_sm", C.c_int),
                ("warps_per_tile", C.c_int)]


# every symbol include/vr.h declares
EXPORTS = ("vr_volume_create", "vr_volume_rebrick", "vr_volume_update", "vr_volume_destroy", "vr_volume_info",
           "vr_view_layout",
           "vr_render",
           "vr_render_backward", "vr_render_backward_views", "vr_render_batched", "vr_autotune_batched", "vr_render_batched_noalloc",
           "vr_minimap", "vr_profile", "vr_render_subbox", "vr_render_subbox_of", "vr_composite", "vr_moments",
           "vr_histogram",
           "vr_median", "vr_check", "vr_selftest_timeout", "vr_selftest_bounds", "vr_bounds_checked",
           "vr_debug_fail_alloc", "vr_last_error", "vr_version")
VR_NOALLOC_MAX_JOBS = 256

_lock = threading.Lock()
_lib = None


class VRError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__("%s failed: %s: %s" % (fn, STATUS_NAMES.get(status, status), msg))
        self.status = status


def load() -> C.CDLL:
    """Loads libvr.so (building it first if the sources are newer and nvcc is
    available).  Raises RuntimeError when it cannot be had."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libvr.so is not built (%s); run __graft_entry__.build() or "
                               "python -m paper_1211_4896_gb300.build" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        P, vp = C.POINTER, C.c_void_p
        L.vr_volume_create.argtypes = [vp, C.c_int, C.c_int, P(C.c_int64 * 3), P(C.c_double * 3),
                                       P(C.c_double * 3), C.c_int, vp, P(vp)]
        L.vr_volume_rebrick.argtypes = [vp, C.c_int, vp, P(vp)]
        L.vr_volume_update.argtypes = [vp, vp, C.c_int, vp]
        L.vr_volume_destroy.argtypes = [vp]
        L.vr_volume_info.argtypes = [vp, P(vr_volume_info_t)]
        L.vr_view_layout.argtypes = [vp, P(vr_camera), P(C.c_int)]
        L.vr_render.argtypes = [vp, P(vr_camera), P(vr_params), vp, vp, vp]
        L.vr_render_backward.argtypes = [vp, P(vr_camera), P(vr_params), vp, vp, vp, vp, vp, C.c_uint, vp]
        L.vr_render_backward_views.argtypes = [vp, P(vr_grad_view), C.c_int, P(vr_params), vp, vp, C.c_uint, vp]
        L.vr_render_batched.argtypes = [P(vr_job), C.c_int, P(vr_batch_opts), vp]
        L.vr_autotune_batched.argtypes = [P(vr_job), C.c_int, P(vr_batch_opts), vp]
        L.vr_render_batched_noalloc.argtypes = [P(vr_job), C.c_int, C.c_int, C.c_int, vp]
        L.vr_check.argtypes = [vp, vp]
        L.vr_selftest_timeout.argtypes = [vp, vp]
        L.vr_selftest_bounds.argtypes = [vp, vp]
        L.vr_debug_fail_alloc.argtypes = [C.c_int]
        L.vr_debug_fail_alloc.restype = None
        L.vr_bounds_checked.argtypes = []
        L.vr_bounds_checked.restype = C.c_int
        L.vr_minimap.argtypes = [vp, P(C.c_int * 3), vp, vp]
        L.vr_profile.argtypes = [vp, P(vr_camera), C.c_float, C.c_int, C.c_int, vp, C.c_uint32, vp, vp]
        L.vr_render_subbox.argtypes = [vp, P(vr_camera), P(vr_params), P(C.c_int * 3), P(C.c_int * 3), vp, vp, vp,
                                       vp]
        L.vr_render_subbox_of.argtypes = [vp, P(C.c_int64 * 3), P(C.c_int64 * 3), P(vr_camera), P(vr_params),
                                          P(C.c_int * 3), P(C.c_int * 3), vp, vp, vp, vp]
        L.vr_composite.argtypes = [C.c_int, P(vp), P(vp), C.c_int, C.c_int, P(C.c_float * 4), vp, vp]
        L.vr_moments.argtypes = [vp, vp, vp]
        L.vr_histogram.argtypes = [vp, C.c_double, C.c_double, C.c_int, vp, vp]
        L.vr_median.argtypes = [vp, vp, vp]
        for name in ("vr_volume_create", "vr_volume_rebrick", "vr_volume_update", "vr_volume_destroy",
                     "vr_volume_info", "vr_view_layout",
                     "vr_render",
                     "vr_render_backward", "vr_render_backward_views", "vr_render_batched", "vr_autotune_batched",
                     "vr_render_batched_noalloc", "vr_minimap", "vr_profile", "vr_render_subbox", "vr_render_subbox_of",
                     "vr_composite",
                     "vr_moments", "vr_histogram", "vr_median", "vr_check", "vr_selftest_timeout",
                     "vr_selftest_bounds"):
            getattr(L, name).restype = C.c_int
        L.vr_last_error.argtypes = []
        L.vr_last_error.restype = C.c_char_p
        L.vr_version.argtypes = []
        L.vr_version.restype = C.c_char_p
        _lib = L
        return L


def last_error() -> str:
    return load().vr_last_error().decode()


def _check(fn: str, status: int):
    if status != VR_OK:
        raise VRError(fn, status, last_error())


# ---------------------------------------------------------------------------
# Struct builders
# ---------------------------------------------------------------------------

def make_camera(cam: dict) -> vr_camera:
    return vr_camera(int(cam["kind"]), (C.c_double * 3)(*cam["eye"]), (C.c_double * 3)(*cam["forward"]),
                     (C.c_double * 3)(*cam["up"]), float(cam.get("fov_y_deg", 0.0)),
                     float(cam.get("ortho_height", 0.0)), int(cam["width"]), int(cam["height"]))


def make_params(tf_ptr: int, K: int, vmin: float, vmax: float, step: float, ert: float = 2.0,
                bg=(0.0, 0.0, 0.0, 0.0), filter: int = VR_FILTER_SOFTWARE, mode: int = VR_MODE_COMPOSITE,
                minimap_ptr: int | None = None, region=(1, 1, 1), skip_empty: bool = False) -> vr_params:
    return vr_params(tf_ptr, int(K), float(vmin), float(vmax), float(step), float(ert), (C.c_float * 4)(*bg),
                     int(filter), int(mode), minimap_ptr, (C.c_int * 3)(*[int(r) for r in region]),
                     int(bool(skip_empty)))


# ---------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def vr_volume_create(dev_cube: int, src_dtype: int, store_dtype: int, dims, origin=None, spacing=None,
                     brick: int = 0, stream: int = 0) -> int:
    L = load()
    out = C.c_void_p()
    d = (C.c_int64 * 3)(*dims)
    o = (C.c_double * 3)(*origin) if origin is not None else None
    s = (C.c_double * 3)(*spacing) if spacing is not None else None
    _check("vr_volume_create", L.vr_volume_create(dev_cube, src_dtype, store_dtype, C.byref(d),
                                                  C.byref(o) if o else None, C.byref(s) if s else None,
                                                  int(brick), stream, C.byref(out)))
    return out.value


def vr_volume_rebrick(vol: int, brick: int, stream: int = 0) -> int:
    out = C.c_void_p()
    _check("vr_volume_rebrick", load().vr_volume_rebrick(vol, int(brick), stream, C.byref(out)))
    return out.value


def vr_volume_update(vol: int, dev_cube: int, src_dtype: int, stream: int = 0):
    _check("vr_volume_update", load().vr_volume_update(vol, dev_cube, src_dtype, stream))


def vr_volume_destroy(vol: int):
    _check("vr_volume_destroy", load().vr_volume_destroy(vol))


def vr_view_layout(vol: int, cam: vr_camera) -> int:
    """-1 for the x-fastest bricks, else the id of the copy this view reads."""
    out = C.c_int(0)
    _check("vr_view_layout", load().vr_view_layout(vol, C.byref(cam), C.byref(out)))
    return out.value


def vr_volume_info(vol: int) -> dict:
    info = vr_volume_info_t()
    _check("vr_volume_info", load().vr_volume_info(vol, C.byref(info)))
    return dict(dims=tuple(info.dims), store_dtype=info.store_dtype, brick=info.brick,
                bricks=tuple(info.bricks), bytes=info.bytes, dense_bytes=info.dense_bytes,
                copy_bytes=info.copy_bytes, copies=info.copies, scratch_bytes=info.scratch_bytes)


def vr_render(vol: int, cam: vr_camera, params: vr_params, dev_rgba_out: int, dev_nsamples_out: int | None,
              stream: int = 0):
    _check("vr_render", load().vr_render(vol, C.byref(cam), C.byref(params), dev_rgba_out, dev_nsamples_out,
                                         stream))


def vr_render_backward(vol: int, cam: vr_camera, params: vr_params, dev_rgba: int, dev_nsamples: int,
                       dev_grad_rgba: int, dev_grad_tf: int, dev_grad_vox: int | None, flags: int = 0,
                       stream: int = 0):
    _check("vr_render_backward", load().vr_render_backward(vol, C.byref(cam), C.byref(params), dev_rgba,
                                                           dev_nsamples, dev_grad_rgba, dev_grad_tf,
                                                           dev_grad_vox, int(flags), stream))


def vr_render_backward_views(vol: int, views, params: vr_params, dev_grad_tf: int, dev_grad_vox: int | None,
                             flags: int = 0, stream: int = 0):
    """views: a sequence of vr_grad_view (camera, image, sample counts and
    dL/d(image) pointers of each view)."""
    arr = (vr_grad_view * len(views))(*views)
    _check("vr_render_backward_views", load().vr_render_backward_views(vol, arr, len(views), C.byref(params),
                                                                       dev_grad_tf, dev_grad_vox, int(flags),
                                                                       stream))


def vr_render_batched(jobs, opts: vr_batch_opts | None = None, stream: int = 0):
    arr = (vr_job * len(jobs))(*jobs)
    _check("vr_render_batched", load().vr_render_batched(arr, len(jobs), C.byref(opts) if opts else None,
                                                         stream))


def vr_autotune_batched(jobs, opts: vr_batch_opts | None = None, stream: int = 0) -> vr_batch_opts:
    arr = (vr_job * len(jobs))(*jobs)
    best = opts if opts is not None else vr_batch_opts(0, 0, 0, 0)
    _check("vr_autotune_batched", load().vr_autotune_batched(arr, len(jobs), C.byref(best), stream))
    return best


def vr_render_batched_noalloc(jobs, tile_w: int = 0, tile_h: int = 0, stream: int = 0):
    """Same jobs as vr_render_batched, with no device allocation (static scratch)."""
    arr = (vr_job * len(jobs))(*jobs)
    _check("vr_render_batched_noalloc", load().vr_render_batched_noalloc(arr, len(jobs), int(tile_w), int(tile_h),
                                                                         stream))


def vr_minimap(vol: int, region, dev_minimap: int, stream: int = 0):
    _check("vr_minimap", load().vr_minimap(vol, C.byref((C.c_int * 3)(*[int(r) for r in region])), dev_minimap,
                                           stream))


def vr_profile(vol: int, cam: vr_camera, step: float, i: int, j: int, dev_values: int | None, max_values: int,
               dev_count: int, stream: int = 0):
    _check("vr_profile", load().vr_profile(vol, C.byref(cam), float(step), int(i), int(j), dev_values,
                                           int(max_values), dev_count, stream))


def vr_render_subbox(vol: int, cam: vr_camera, params: vr_params, cell_lo, cell_hi, dev_partial: int,
                     dev_depth: int, dev_count: int | None, stream: int = 0):
    _check("vr_render_subbox", load().vr_render_subbox(vol, C.byref(cam), C.byref(params),
                                                       C.byref((C.c_int * 3)(*[int(x) for x in cell_lo])),
                                                       C.byref((C.c_int * 3)(*[int(x) for x in cell_hi])),
                                                       dev_partial, dev_depth, dev_count, stream))


def vr_render_subbox_of(vol: int, global_dims, offset, cam: vr_camera, params: vr_params, cell_lo, cell_hi,
                        dev_partial: int, dev_depth: int, dev_count: int | None, stream: int = 0):
    _check("vr_render_subbox_of",
           load().vr_render_subbox_of(vol, C.byref((C.c_int64 * 3)(*[int(x) for x in global_dims])),
                                      C.byref((C.c_int64 * 3)(*[int(x) for x in offset])), C.byref(cam),
                                      C.byref(params), C.byref((C.c_int * 3)(*[int(x) for x in cell_lo])),
                                      C.byref((C.c_int * 3)(*[int(x) for x in cell_hi])), dev_partial, dev_depth,
                                      dev_count, stream))


def vr_composite(dev_partials, dev_depths, width: int, height: int, bg, dev_rgba_out: int, stream: int = 0):
    k = len(dev_partials)
    _check("vr_composite", load().vr_composite(k, (C.c_void_p * k)(*dev_partials), (C.c_void_p * k)(*dev_depths),
                                               int(width), int(height), C.byref((C.c_float * 4)(*bg)),
                                               dev_rgba_out, stream))


def vr_moments(vol: int, dev_out: int, stream: int = 0):
    _check("vr_moments", load().vr_moments(vol, dev_out, stream))


def vr_histogram(vol: int, lo: float, hi: float, nbins: int, dev_counts: int, stream: int = 0):
    _check("vr_histogram", load().vr_histogram(vol, float(lo), float(hi), int(nbins), dev_counts, stream))


def vr_median(vol: int, dev_median: int, stream: int = 0):
    _check("vr_median", load().vr_median(vol, dev_median, stream))


def vr_selftest_bounds(vol: int, stream: int = 0):
    _check("vr_selftest_bounds", load().vr_selftest_bounds(vol, stream))


def vr_debug_fail_alloc(after: int):
    """Makes the library's device allocation after `after` successful ones
    fail once (negative: cancel)."""
    load().vr_debug_fail_alloc(int(after))


def vr_bounds_checked() -> bool:
    """True for the bounds-check build of the library."""
    return bool(load().vr_bounds_checked())


def vr_selftest_timeout(vol: int, stream: int = 0):
    _check("vr_selftest_timeout", load().vr_selftest_timeout(vol, stream))


def vr_check(vol: int, stream: int = 0):
    """Raises VRError(VR_ERR_TIMEOUT) if a bounded device wait of an earlier call gave up."""
    _check("vr_check", load().vr_check(vol, stream))


def vr_version() -> str:
    return load().vr_version().decode()
