"""FP64 CPU ray caster (the oracle) -- ctypes front end.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never calls it, and it never calls the CUDA library.

The arithmetic lives in ``vr_oracle.c`` (plain C, double precision); this file
builds it with gcc and marshals numpy arrays.  Cameras are the plain dicts of
the ``synth`` module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vr_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

DT_F32, DT_F64, DT_F16, DT_BF16 = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile vr_oracle.c into a shared library (gcc, no FMA contraction so
    x86_64 and aarch64 round identically)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Camera(C.Structure):
    _fields_ = [("kind", C.c_int), ("eye", C.c_double * 3), ("forward", C.c_double * 3),
                ("up", C.c_double * 3), ("fov_y_deg", C.c_double), ("ortho_height", C.c_double),
                ("width", C.c_int), ("height", C.c_int)]


class Volume(C.Structure):
    _fields_ = [("data", C.c_void_p), ("dtype", C.c_int), ("n", C.c_int64 * 3),
                ("origin", C.c_double * 3), ("spacing", C.c_double * 3)]


class Params(C.Structure):
    _fields_ = [("tf", C.c_void_p), ("K", C.c_int), ("vmin", C.c_double), ("vmax", C.c_double),
                ("step", C.c_double), ("ert", C.c_double), ("bg", C.c_double * 4)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.POINTER
            L.orc_render.argtypes = [P(Volume), P(Camera), P(Params), C.c_int, C.c_int, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
            L.orc_render.restype = C.c_int
            L.orc_render_backward.argtypes = [P(Volume), P(Camera), P(Params), C.c_int, C.c_int, C.c_void_p,
                                              C.c_void_p, C.c_void_p, C.c_int]
            L.orc_render_backward.restype = C.c_int
            L.orc_render_backward_kinks.argtypes = [P(Volume), P(Camera), P(Params), C.c_int, C.c_int, C.c_void_p,
                                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                                    C.c_int]
            L.orc_render_backward_kinks.restype = C.c_int
            L.orc_trilinear.argtypes = [P(Volume), P(C.c_double * 3)]
            L.orc_trilinear.restype = C.c_double
            L.orc_tf_lookup.argtypes = [P(Params), C.c_double, P(C.c_double * 4)]
            L.orc_tf_lookup.restype = None
            L.orc_ray.argtypes = [P(Volume), P(Camera), P(Params), C.c_int, C.c_int,
                                  P(C.c_double * 3), P(C.c_double * 3), P(C.c_double)]
            L.orc_ray.restype = C.c_int64
            L.orc_profile.argtypes = [P(Volume), P(Camera), P(Params), C.c_int, C.c_int, C.c_void_p, C.c_int64]
            L.orc_profile.restype = C.c_int64
            L.orc_render_mip.argtypes = [P(Volume), P(Camera), P(Params), C.c_int, C.c_int, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_int]
            L.orc_render_mip.restype = C.c_int
            L.orc_minimap.argtypes = [P(Volume), P(C.c_int * 3), C.c_void_p, P(C.c_int64 * 3)]
            L.orc_minimap.restype = C.c_int
            L.orc_minimap_sample.argtypes = [C.c_void_p, P(C.c_int64 * 3), P(C.c_int * 3), P(C.c_double * 3),
                                             P(C.c_double * 2)]
            L.orc_minimap_sample.restype = None
            L.orc_render_sigma.argtypes = [P(Volume), P(Camera), P(Params), C.c_void_p, P(C.c_int64 * 3),
                                           P(C.c_int * 3), C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int]
            L.orc_render_sigma.restype = C.c_int
            L.orc_render_subbox.argtypes = [P(Volume), P(Camera), P(Params), P(C.c_int64 * 3), P(C.c_int64 * 3),
                                            C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_render_subbox.restype = C.c_int
            L.orc_composite.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_int64, P(C.c_double * 4), C.c_void_p]
            L.orc_composite.restype = None
            L.orc_moments.argtypes = [P(Volume), P(C.c_double * 5)]
            L.orc_moments.restype = C.c_int
            L.orc_histogram.argtypes = [P(Volume), C.c_double, C.c_double, C.c_int, C.c_void_p]
            L.orc_histogram.restype = C.c_int
            L.orc_median.argtypes = [P(Volume), P(C.c_double), P(C.c_int)]
            L.orc_median.restype = C.c_int
            _lib = L
    return _lib


def _dtype_code(a: np.ndarray, bits: str | None):
    if bits == "f16":
        return DT_F16
    if bits == "bf16":
        return DT_BF16
    if a.dtype == np.float32:
        return DT_F32
    if a.dtype == np.float64:
        return DT_F64
    raise TypeError("cube must be float32/float64, or uint16 bits with bits='f16'/'bf16'")


class _Call:
    """Keeps the numpy buffers alive for the duration of one C call."""

    def __init__(self, cube, cam, tf, vmin, vmax, step, ert, bg, origin, spacing, bits):
        cube = np.ascontiguousarray(cube)
        if cube.ndim != 3:
            raise ValueError("cube must be (nz, ny, nx)")
        self.cube = cube
        self.tf = np.ascontiguousarray(np.asarray(tf, dtype=np.float64).reshape(-1, 4))
        nz, ny, nx = cube.shape
        self.vol = Volume(cube.ctypes.data, _dtype_code(cube, bits), (C.c_int64 * 3)(nx, ny, nz),
                          (C.c_double * 3)(*origin), (C.c_double * 3)(*spacing))
        self.cam = Camera(int(cam["kind"]), (C.c_double * 3)(*cam["eye"]),
                          (C.c_double * 3)(*cam["forward"]), (C.c_double * 3)(*cam["up"]),
                          float(cam.get("fov_y_deg", 0.0)), float(cam.get("ortho_height", 0.0)),
                          int(cam["width"]), int(cam["height"]))
        self.par = Params(self.tf.ctypes.data, self.tf.shape[0], float(vmin), float(vmax), float(step),
                          float(ert), (C.c_double * 4)(*bg))


def render(cube, cam, tf, vmin, vmax, step, ert=2.0, bg=(0.0, 0.0, 0.0, 0.0), origin=(0.0, 0.0, 0.0),
           spacing=(1.0, 1.0, 1.0), rows=None, nthreads=None, bits=None):
    """FP64 render.  Returns dict(rgba (H,W,4) f64, n_used (H,W) i32,
    margin_n, margin_ert (H,W) f64).  ``rows=(r0, r1)`` renders only those
    rows (others stay zero)."""
    c = _Call(cube, cam, tf, vmin, vmax, step, ert, bg, origin, spacing, bits)
    H, W = c.cam.height, c.cam.width
    rgba = np.zeros((H, W, 4), dtype=np.float64)
    n_used = np.zeros((H, W), dtype=np.int32)
    m_n = np.full((H, W), np.inf)
    m_e = np.full((H, W), np.inf)
    r0, r1 = rows if rows is not None else (0, H)
    nt = nthreads or os.cpu_count() or 1
    rc = lib().orc_render(C.byref(c.vol), C.byref(c.cam), C.byref(c.par), int(r0), int(r1),
                          rgba.ctypes.data, n_used.ctypes.data, m_n.ctypes.data, m_e.ctypes.data, int(nt))
    if rc != 0:
        raise ValueError("orc_render failed (%d)" % rc)
    return dict(rgba=rgba, n_used=n_used, margin_n=m_n, margin_ert=m_e)


def render_backward(cube, cam, tf, vmin, vmax, step, grad_rgba, ert=2.0, bg=(0.0, 0.0, 0.0, 0.0),
                    origin=(0.0, 0.0, 0.0), spacing=(1.0, 1.0, 1.0), want_vox=True, nthreads=None,
                    bits=None, rows=None, kink_eps=None):
    """FP64 gradients (grad_tf (K,4), grad_vox (nz,ny,nx) or None) of
    L given dL/dI = grad_rgba (H,W,4).  With kink_eps (in table entries) two
    more arrays are returned: per voxel, the bound on how far its gradient
    moves when samples within kink_eps of a table-interval end (vmin and vmax
    included) take the slope of the other side, and the sum of the
    magnitudes that make up its gradient terms before cancellation
    (orc_render_backward_kinks)."""
    c = _Call(cube, cam, tf, vmin, vmax, step, ert, bg, origin, spacing, bits)
    g = np.ascontiguousarray(np.asarray(grad_rgba, dtype=np.float64))
    if g.shape != (c.cam.height, c.cam.width, 4):
        raise ValueError("grad_rgba must be (H, W, 4)")
    gtf = np.zeros(c.tf.shape, dtype=np.float64)
    gvox = np.zeros(c.cube.shape, dtype=np.float64) if want_vox else None
    nt = nthreads or os.cpu_count() or 1
    r0, r1 = rows if rows is not None else (0, c.cam.height)
    if kink_eps is None:
        rc = lib().orc_render_backward(C.byref(c.vol), C.byref(c.cam), C.byref(c.par), int(r0), int(r1),
                                       g.ctypes.data, gtf.ctypes.data, gvox.ctypes.data if gvox is not None else None,
                                       int(nt))
    else:
        kink = np.zeros(c.cube.shape, dtype=np.float64)
        mag = np.zeros(c.cube.shape, dtype=np.float64)
        rc = lib().orc_render_backward_kinks(C.byref(c.vol), C.byref(c.cam), C.byref(c.par), int(r0), int(r1),
                                             g.ctypes.data, gtf.ctypes.data,
                                             gvox.ctypes.data if gvox is not None else None, kink.ctypes.data,
                                             mag.ctypes.data, float(kink_eps), int(nt))
    if rc != 0:
        raise ValueError("orc_render_backward failed (%d)" % rc)
    return (gtf, gvox) if kink_eps is None else (gtf, gvox, kink, mag)


def trilinear(cube, p, origin=(0.0, 0.0, 0.0), spacing=(1.0, 1.0, 1.0), bits=None):
    """Trilinear value at voxel-space position p = (x, y, z)."""
    c = _Call(cube, dict(kind=0, eye=(0, 0, 0), forward=(0, 0, 1), up=(0, 1, 0), width=1, height=1),
              [[0, 0, 0, 0], [0, 0, 0, 0]], 0.0, 1.0, 1.0, 2.0, (0, 0, 0, 0), origin, spacing, bits)
    return lib().orc_trilinear(C.byref(c.vol), C.byref((C.c_double * 3)(*p)))


def tf_lookup(tf, vmin, vmax, value):
    c = _Call(np.zeros((2, 2, 2), np.float32), dict(kind=0, eye=(0, 0, 0), forward=(0, 0, 1),
              up=(0, 1, 0), width=1, height=1), tf, vmin, vmax, 1.0, 2.0, (0, 0, 0, 0),
              (0, 0, 0), (1, 1, 1), None)
    out = (C.c_double * 4)()
    lib().orc_tf_lookup(C.byref(c.par), float(value), C.byref(out))
    return np.array(list(out))


def ray(cube_shape, cam, step, i, j, origin=(0.0, 0.0, 0.0), spacing=(1.0, 1.0, 1.0)):
    """(n_samples, ov, dv, t_in) of pixel (i, j) -- voxel-space ray setup."""
    dummy = np.zeros(cube_shape, np.float32)
    c = _Call(dummy, cam, [[0, 0, 0, 0], [0, 0, 0, 0]], 0.0, 1.0, step, 2.0, (0, 0, 0, 0), origin,
              spacing, None)
    ov = (C.c_double * 3)()
    dv = (C.c_double * 3)()
    tin = C.c_double()
    n = lib().orc_ray(C.byref(c.vol), C.byref(c.cam), C.byref(c.par), int(i), int(j), C.byref(ov),
                      C.byref(dv), C.byref(tin))
    return int(n), np.array(list(ov)), np.array(list(dv)), tin.value


def profile(cube, cam, step, i, j, origin=(0.0, 0.0, 0.0), spacing=(1.0, 1.0, 1.0), bits=None):
    """3D spectrum tool (Section 4.4): trilinear values of the samples along
    pixel (i, j)'s clipped ray, at the renderer's sample positions."""
    c = _Call(cube, cam, [[0, 0, 0, 0], [0, 0, 0, 0]], 0.0, 1.0, step, 2.0, (0, 0, 0, 0), origin, spacing, bits)
    n = lib().orc_profile(C.byref(c.vol), C.byref(c.cam), C.byref(c.par), int(i), int(j), None, 0)
    if n < 0:
        raise ValueError("orc_profile failed")
    out = np.zeros(max(int(n), 1), dtype=np.float64)
    lib().orc_profile(C.byref(c.vol), C.byref(c.cam), C.byref(c.par), int(i), int(j), out.ctypes.data, int(n))
    return out[:int(n)]


def render_mip(cube, cam, tf, vmin, vmax, step, bg=(0.0, 0.0, 0.0, 0.0), origin=(0.0, 0.0, 0.0),
               spacing=(1.0, 1.0, 1.0), rows=None, nthreads=None, bits=None):
    """Maximum intensity projection (Section 3.3.1).  Returns dict(rgba, n_used,
    vmax (H,W) f64 -- each ray's largest value, NaN on a miss)."""
    c = _Call(cube, cam, tf, vmin, vmax, step, 2.0, bg, origin, spacing, bits)
    H, W = c.cam.height, c.cam.width
    rgba = np.zeros((H, W, 4), dtype=np.float64)
    n_used = np.zeros((H, W), dtype=np.int32)
    vm = np.full((H, W), np.nan)
    r0, r1 = rows if rows is not None else (0, H)
    rc = lib().orc_render_mip(C.byref(c.vol), C.byref(c.cam), C.byref(c.par), int(r0), int(r1), rgba.ctypes.data,
                              n_used.ctypes.data, vm.ctypes.data, int(nthreads or os.cpu_count() or 1))
    if rc != 0:
        raise ValueError("orc_render_mip failed (%d)" % rc)
    return dict(rgba=rgba, n_used=n_used, vmax=vm)


def minimap(cube, region, bits=None):
    """Statistical mini-map (Section 4.5): (mk, mj, mi, 2) array of the mean and
    population standard deviation of each region of region = (rx, ry, rz)
    voxels (the last region of an axis keeps the remainder)."""
    c = _Call(cube, dict(kind=0, eye=(0, 0, 0), forward=(0, 0, 1), up=(0, 1, 0), width=1, height=1),
              [[0, 0, 0, 0], [0, 0, 0, 0]], 0.0, 1.0, 1.0, 2.0, (0, 0, 0, 0), (0, 0, 0), (1, 1, 1), bits)
    nz, ny, nx = c.cube.shape
    m = [-(-n // r) for n, r in zip((nx, ny, nz), region)]
    out = np.zeros((m[2], m[1], m[0], 2), dtype=np.float64)
    mm = (C.c_int64 * 3)()
    rc = lib().orc_minimap(C.byref(c.vol), C.byref((C.c_int * 3)(*region)), out.ctypes.data, C.byref(mm))
    if rc != 0:
        raise ValueError("orc_minimap failed (%d)" % rc)
    return out


def minimap_sample(stats, region, p):
    """(mean, sd) of the mini-map at voxel position p = (x, y, z)."""
    stats = np.ascontiguousarray(stats, dtype=np.float64)
    mk, mj, mi = stats.shape[:3]
    out = (C.c_double * 2)()
    lib().orc_minimap_sample(stats.ctypes.data, C.byref((C.c_int64 * 3)(mi, mj, mk)),
                             C.byref((C.c_int * 3)(*region)), C.byref((C.c_double * 3)(*p)), C.byref(out))
    return out[0], out[1]


def render_sigma(cube, cam, tf, vmin, vmax, step, stats, region, ert=2.0, bg=(0.0, 0.0, 0.0, 0.0),
                 origin=(0.0, 0.0, 0.0), spacing=(1.0, 1.0, 1.0), rows=None, nthreads=None, bits=None):
    """Sigma-clipping render (Section 4.5): each sample value becomes
    (v - mean)/sd of the mini-map `stats` at its position before the table
    lookup; [vmin, vmax] are in units of sd.  Returns dict(rgba, n_used)."""
    c = _Call(cube, cam, tf, vmin, vmax, step, ert, bg, origin, spacing, bits)
    st = np.ascontiguousarray(stats, dtype=np.float64)
    mk, mj, mi = st.shape[:3]
    H, W = c.cam.height, c.cam.width
    rgba = np.zeros((H, W, 4), dtype=np.float64)
    n_used = np.zeros((H, W), dtype=np.int32)
    r0, r1 = rows if rows is not None else (0, H)
    rc = lib().orc_render_sigma(C.byref(c.vol), C.byref(c.cam), C.byref(c.par), st.ctypes.data,
                                C.byref((C.c_int64 * 3)(mi, mj, mk)), C.byref((C.c_int * 3)(*region)), int(r0),
                                int(r1), rgba.ctypes.data, n_used.ctypes.data, int(nthreads or os.cpu_count() or 1))
    if rc != 0:
        raise ValueError("orc_render_sigma failed (%d)" % rc)
    return dict(rgba=rgba, n_used=n_used)


def _vol_only(cube, bits=None):
    return _Call(cube, dict(kind=0, eye=(0, 0, 0), forward=(0, 0, 1), up=(0, 1, 0), width=1, height=1),
                 [[0, 0, 0, 0], [0, 0, 0, 0]], 0.0, 1.0, 1.0, 2.0, (0, 0, 0, 0), (0, 0, 0), (1, 1, 1), bits)


def moments(cube, bits=None):
    """Global statistics of the non-NaN voxels (Section 4.2): dict(count,
    mean, sd (population), min, max), FP64."""
    c = _vol_only(cube, bits)
    out = (C.c_double * 5)()
    if lib().orc_moments(C.byref(c.vol), C.byref(out)) != 0:
        raise ValueError("orc_moments failed")
    return dict(count=int(out[0]), mean=out[1], sd=out[2], min=out[3], max=out[4])


def histogram(cube, lo, hi, nbins, bits=None):
    """Histogram of the non-NaN voxels over [lo, hi] in nbins equal bins
    (Section 4.1; the value hi falls in the last bin)."""
    c = _vol_only(cube, bits)
    counts = np.zeros(int(nbins), dtype=np.uint64)
    if lib().orc_histogram(C.byref(c.vol), float(lo), float(hi), int(nbins), counts.ctypes.data) != 0:
        raise ValueError("orc_histogram failed")
    return counts


def median(cube, bits=None):
    """Torben's median of the non-NaN voxels (Section 4.3 and the paper's
    appendix): the value of rank (n + 1) // 2.  Returns (median, passes)."""
    c = _vol_only(cube, bits)
    m = C.c_double()
    it = C.c_int()
    if lib().orc_median(C.byref(c.vol), C.byref(m), C.byref(it)) != 0:
        raise ValueError("orc_median failed (no values)")
    return m.value, it.value


def render_subbox(cube, cam, tf, vmin, vmax, step, lo, hi, rows=None, origin=(0.0, 0.0, 0.0),
                  spacing=(1.0, 1.0, 1.0), bits=None):
    """Sort-last partial render (Sections 3.2, 3.4) of the samples whose cell
    lies in [lo, hi) (per axis x, y, z), at the whole volume's sample
    positions: dict(partial (H,W,4) = premultiplied C and T, depth (H,W) =
    ray parameter of the first sample or inf, count (H,W))."""
    c = _Call(cube, cam, tf, vmin, vmax, step, 2.0, (0, 0, 0, 0), origin, spacing, bits)
    H, W = c.cam.height, c.cam.width
    part = np.zeros((H, W, 4))
    part[..., 3] = 1.0
    depth = np.full((H, W), np.inf)
    count = np.zeros((H, W), np.int32)
    r0, r1 = rows if rows is not None else (0, H)
    rc = lib().orc_render_subbox(C.byref(c.vol), C.byref(c.cam), C.byref(c.par), C.byref((C.c_int64 * 3)(*lo)),
                                 C.byref((C.c_int64 * 3)(*hi)), int(r0), int(r1), part.ctypes.data,
                                 depth.ctypes.data, count.ctypes.data)
    if rc != 0:
        raise ValueError("orc_render_subbox failed")
    return dict(partial=part, depth=depth, count=count)


def composite(partials, depths, bg=(0.0, 0.0, 0.0, 0.0)):
    """Over-composite of partial images in per-pixel depth order."""
    ps = [np.ascontiguousarray(p, dtype=np.float64) for p in partials]
    ds = [np.ascontiguousarray(d, dtype=np.float64) for d in depths]
    k = len(ps)
    H, W = ds[0].shape
    out = np.zeros((H, W, 4))
    pp = (C.c_void_p * k)(*[p.ctypes.data for p in ps])
    dd = (C.c_void_p * k)(*[d.ctypes.data for d in ds])
    lib().orc_composite(k, pp, dd, H * W, C.byref((C.c_double * 4)(*bg)), out.ctypes.data)
    return out
