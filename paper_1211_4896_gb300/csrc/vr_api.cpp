// vr_api.cpp -- host side of the C ABI declared in include/vr.h: argument
// validation, volume handles, camera preparation and kernel dispatch.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "vr_internal.h"

namespace vr {

static thread_local std::string g_err;

#ifdef VR_BOUNDS_CHECK
static constexpr bool kBoundsChecked = true;
#else
static constexpr bool kBoundsChecked = false;
#endif

void set_error(const std::string &msg) { g_err = msg; }

vr_status cuda_fail(cudaError_t e, const char *what)
{
    set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return e == cudaErrorMemoryAllocation ? VR_ERR_OOM : VR_ERR_CUDA;
}

bool is_aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// VR_LOG=1 in the environment: one line on stderr per launch decision (brick
// layout of a view, grid of a launch, the backward's voxel-gradient form, the
// groups of a batch).
bool log_enabled()
{
    static const bool on = [] {
        const char *e = std::getenv("VR_LOG");
        return e && e[0] && e[0] != '0';
    }();
    return on;
}

void log_line(const char *fmt, ...)
{
    if (!log_enabled()) return;
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    std::fprintf(stderr, "vr: %s\n", buf);
}

// Every device allocation of the library goes through dev_alloc, so that a
// test can make one of them fail (vr_debug_fail_alloc) and check the error
// paths and fallbacks.
static std::mutex g_fail_mu;
static long long g_fail_after = -1;      // successful allocations before the injected failure; -1: none

cudaError_t dev_alloc(void **p, size_t bytes)
{
    {
        std::lock_guard<std::mutex> g(g_fail_mu);
        if (g_fail_after == 0) {
            g_fail_after = -1;
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
        if (g_fail_after > 0) --g_fail_after;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t dev_alloc_layers(cudaArray_t *a, int u, int v, int layers)
{
    {
        std::lock_guard<std::mutex> g(g_fail_mu);
        if (g_fail_after == 0) {
            g_fail_after = -1;
            *a = nullptr;
            return cudaErrorMemoryAllocation;
        }
        if (g_fail_after > 0) --g_fail_after;
    }
    const cudaChannelFormatDesc fd = cudaCreateChannelDesc<float>();
    return cudaMalloc3DArray(a, &fd, make_cudaExtent((size_t)u, (size_t)v, (size_t)layers),
                             cudaArrayLayered | cudaArraySurfaceLoadStore);
}

bool copy_built(const vr_volume *vol, int copy)
{
    if (copy_layers(copy)) return vol->layers[copy - 9].tex != 0;
    return copy >= 1 && copy < 9 && vol->copies[copy] != nullptr;
}

static vr_status invalid(const std::string &msg)
{
    set_error(msg);
    return VR_ERR_INVALID_ARG;
}

int sm_count()
{
    static std::mutex mu;
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(mu);
    if (dev < 0 || dev >= 64) return 1;
    if (!cached[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = n > 0 ? n : 1;
    }
    return cached[dev];
}

static bool finite3(const double v[3]) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// Checks of the camera that need no volume.
static vr_status check_camera(const vr_camera *cam)
{
    if (!cam) return invalid("camera is NULL");
    if (cam->kind != VR_CAMERA_ORTHO && cam->kind != VR_CAMERA_PERSPECTIVE)
        return invalid("camera.kind must be VR_CAMERA_ORTHO (0) or VR_CAMERA_PERSPECTIVE (1)");
    if (cam->width < 1 || cam->height < 1 || cam->width > 32768 || cam->height > 32768)
        return invalid("camera.width and camera.height must be in [1, 32768]");
    if (!finite3(cam->eye) || !finite3(cam->forward) || !finite3(cam->up))
        return invalid("camera eye/forward/up must be finite");
    const double fl = std::sqrt(dot3(cam->forward, cam->forward)), ul = std::sqrt(dot3(cam->up, cam->up));
    if (!(fl > 0.0) || !(ul > 0.0)) return invalid("camera forward and up must be non-zero");
    double x[3];
    cross3(cam->forward, cam->up, x);
    if (!(std::sqrt(dot3(x, x)) > 1e-9 * fl * ul)) return invalid("camera up must not be parallel to forward");
    if (cam->kind == VR_CAMERA_PERSPECTIVE) {
        if (!(cam->fov_y_deg > 0.0 && cam->fov_y_deg < 180.0))
            return invalid("camera.fov_y_deg must be in (0, 180) for a perspective camera");
    } else if (!(cam->ortho_height > 0.0) || !std::isfinite(cam->ortho_height)) {
        return invalid("camera.ortho_height must be finite and > 0 for an orthographic camera");
    }
    return VR_OK;
}

static vr_status check_params(const vr_params *p)
{
    if (!p) return invalid("params is NULL");
    if (!p->tf_rgba) return invalid("params.tf_rgba is NULL");
    if (!is_aligned16(p->tf_rgba)) return invalid("params.tf_rgba must be 16-byte aligned");
    if (p->tf_size < 2 || p->tf_size > 4096) return invalid("params.tf_size must be in [2, 4096]");
    if (!std::isfinite(p->vmin) || !std::isfinite(p->vmax) || !(p->vmax > p->vmin))
        return invalid("params.vmin/vmax must be finite with vmax > vmin");
    if (!std::isfinite(p->step) || !(p->step > 0.0f)) return invalid("params.step must be finite and > 0");
    if (!(p->ert_threshold > 0.0f)) return invalid("params.ert_threshold must be > 0 (values > 1 disable it)");
    for (int c = 0; c < 4; ++c)
        if (!std::isfinite(p->bg_rgba[c])) return invalid("params.bg_rgba must be finite");
    if (p->filter != VR_FILTER_SOFTWARE && p->filter != VR_FILTER_TEXTURE && p->filter != VR_FILTER_SOFTWARE_STAGED)
        return invalid("params.filter must be VR_FILTER_SOFTWARE (0), VR_FILTER_TEXTURE (1) or "
                       "VR_FILTER_SOFTWARE_STAGED (2)");
    if (p->mode != VR_MODE_COMPOSITE && p->mode != VR_MODE_MIP && p->mode != VR_MODE_SIGMA)
        return invalid("params.mode must be VR_MODE_COMPOSITE (0), VR_MODE_MIP (1) or VR_MODE_SIGMA (2)");
    if (p->mode == VR_MODE_SIGMA) {
        if (!p->minimap || (reinterpret_cast<uintptr_t>(p->minimap) & 7u) != 0)
            return invalid("params.minimap must be non-NULL and 8-byte aligned for VR_MODE_SIGMA");
        for (int a = 0; a < 3; ++a)
            if (p->minimap_region[a] < 1) return invalid("params.minimap_region must be >= 1 per axis");
    }
    return VR_OK;
}

// The paths that implement a mode other than the composite.
static vr_status check_mode_path(const vr_params *p, const char *who)
{
    if (p->mode != VR_MODE_COMPOSITE)
        return (set_error(std::string(who) + ": only VR_MODE_COMPOSITE is supported here"), VR_ERR_UNSUPPORTED);
    return VR_OK;
}

static vr_status check_volume(const vr_volume *vol)
{
    if (!vol) return invalid("volume handle is NULL");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != vol->device) return invalid("the volume lives on another device than the current one");
    return VR_OK;
}

// Longest chord of the box in world units divided by the step must stay within
// the range where the float sample index is exact.
static vr_status check_step(const vr_volume *vol, const vr_params *p)
{
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double e = (double)(vol->dims[a] - 1) * vol->spacing[a];
        d2 += e * e;
    }
    if (std::sqrt(d2) / (double)p->step > 16777216.0) return invalid("params.step too small: > 2^24 samples per ray");
    return VR_OK;
}

vr_status prepare_params(const vr_params *p, ParamDev *o)
{
    o->tf = reinterpret_cast<const float4 *>(p->tf_rgba);
    o->K = p->tf_size;
    o->vmin = p->vmin;
    o->scale01 = (float)(1.0 / ((double)p->vmax - (double)p->vmin));
    o->km1 = (float)(p->tf_size - 1);
    const double su = (double)(p->tf_size - 1) / ((double)p->vmax - (double)p->vmin);
    o->su = (float)su;
    o->ou = (float)(-(double)p->vmin * su);
    o->step = p->step;
    o->t_stop = (float)(1.0 - (double)p->ert_threshold);
    o->bg = make_float4(p->bg_rgba[0], p->bg_rgba[1], p->bg_rgba[2], p->bg_rgba[3]);
    return VR_OK;
}

vr_status prepare_camera(const vr_volume *vol, const vr_camera *cam, CamDev *o)
{
    return prepare_camera_grid(vol->origin, vol->spacing, vol->dims, cam, o);
}

// The camera in the voxel coordinates of a grid of dims voxels whose first
// voxel sits at origin (world units).
vr_status prepare_camera_grid(const double origin[3], const double spacing[3], const int64_t dims[3],
                              const vr_camera *cam, CamDev *o)
{
    double f[3] = {cam->forward[0], cam->forward[1], cam->forward[2]};
    const double fl = std::sqrt(dot3(f, f));
    for (double &x : f) x /= fl;
    double r[3], u[3];
    cross3(f, cam->up, r);
    const double rl = std::sqrt(dot3(r, r));
    for (double &x : r) x /= rl;
    cross3(r, f, u);
    const double W = cam->width, H = cam->height, aspect = W / H;
    // anchor plane through the volume centre, perpendicular to f
    double centre[3];
    for (int a = 0; a < 3; ++a) centre[a] = origin[a] + 0.5 * (double)(dims[a] - 1) * spacing[a];
    double ce[3] = {centre[0] - cam->eye[0], centre[1] - cam->eye[1], centre[2] - cam->eye[2]};
    const double D = dot3(ce, f);
    double Q0[3], A[3], B[3], wa[3], wb[3];
    // screen offsets: sx = hi * 2/W, sy = -hj * 2/H with hi = i - (W-1)/2, hj = j - (H-1)/2
    if (cam->kind == VR_CAMERA_ORTHO) {
        const double hh = 0.5 * cam->ortho_height;
        for (int a = 0; a < 3; ++a) {
            Q0[a] = cam->eye[a] + D * f[a];
            A[a] = hh * aspect * r[a] * (2.0 / W);
            B[a] = -hh * u[a] * (2.0 / H);
            wa[a] = wb[a] = 0.0;
        }
    } else {
        const double th = std::tan(cam->fov_y_deg * M_PI / 360.0);
        for (int a = 0; a < 3; ++a) {
            Q0[a] = cam->eye[a] + D * f[a];
            wa[a] = th * aspect * r[a] * (2.0 / W);
            wb[a] = -th * u[a] * (2.0 / H);
            A[a] = D * wa[a];
            B[a] = D * wb[a];
        }
    }
    o->W = cam->width;
    o->H = cam->height;
    o->persp = cam->kind == VR_CAMERA_PERSPECTIVE;
    o->q0 = make_float3((float)((Q0[0] - origin[0]) / spacing[0]),
                        (float)((Q0[1] - origin[1]) / spacing[1]),
                        (float)((Q0[2] - origin[2]) / spacing[2]));
    o->qa = make_float3((float)(A[0] / spacing[0]), (float)(A[1] / spacing[1]),
                        (float)(A[2] / spacing[2]));
    o->qb = make_float3((float)(B[0] / spacing[0]), (float)(B[1] / spacing[1]),
                        (float)(B[2] / spacing[2]));
    o->wf = make_float3((float)f[0], (float)f[1], (float)f[2]);
    o->wa = make_float3((float)wa[0], (float)wa[1], (float)wa[2]);
    o->wb = make_float3((float)wb[0], (float)wb[1], (float)wb[2]);
    o->inv_sp = make_float3((float)(1.0 / spacing[0]), (float)(1.0 / spacing[1]),
                            (float)(1.0 / spacing[2]));
    o->dist = (float)D;
    return VR_OK;
}

VolDev vol_dev(const vr_volume *vol)
{
    VolDev v;
    v.data = vol->bricks;
    v.nx = (int)vol->dims[0];
    v.ny = (int)vol->dims[1];
    v.nz = (int)vol->dims[2];
    v.nbx = (int)vol->nb[0];
    v.nby = (int)vol->nb[1];
    v.nbz = (int)vol->nb[2];
    v.log2b = vol->log2b;
    v.stride = vol->stride;
    v.order = 0;
    v.paired = 0;
    v.nelem = vol->nb[0] * vol->nb[1] * vol->nb[2] * vol->stride;
    v.status = vol->counters + vol->counter_slots - 1;
    return v;
}

VolDev vol_dev_copy(const vr_volume *vol, int copy)
{
    VolDev v = vol_dev(vol);
    if (copy_layers(copy) && vol->layers[copy - 9].tex) {
        v.data = reinterpret_cast<const void *>(static_cast<uintptr_t>(vol->layers[copy - 9].tex));
        v.order = copy - 9;
        v.paired = 3;
        v.nelem = 0;
    } else if (copy >= 1 && copy < 9 && vol->copies[copy]) {
        v.data = vol->copies[copy];
        v.order = copy_order(copy);
        v.paired = copy_blocked(copy) ? 2 : (copy_paired(copy) ? 1 : 0);
        if (copy_blocked(copy)) {
            v.stride = blocked_stride(vol->log2b, vol->store_dtype == VR_F32 ? 4 : 2);
            v.nelem = vol->nb[0] * vol->nb[1] * vol->nb[2] * v.stride;
        }
    }
    return v;
}

// Distance between neighbouring rays at the volume centre, in voxels along
// the image's horizontal direction r (world pitch of one pixel there,
// divided by the spacing along r).
static double ray_pitch_voxels(const vr_volume *vol, const vr_camera *cam, const double r[3])
{
    double pitch = 0.0;
    if (cam->kind == VR_CAMERA_ORTHO) {
        pitch = cam->ortho_height / cam->height;
    } else {
        double f[3] = {cam->forward[0], cam->forward[1], cam->forward[2]};
        const double fl = std::sqrt(dot3(f, f));
        double d = 0.0;
        for (int a = 0; a < 3; ++a)
            d += (vol->origin[a] + 0.5 * (double)(vol->dims[a] - 1) * vol->spacing[a] - cam->eye[a]) * f[a] / fl;
        pitch = 2.0 * std::fabs(d) * std::tan(cam->fov_y_deg * M_PI / 360.0) / cam->height;
    }
    double q = 0.0;
    for (int a = 0; a < 3; ++a) q += (r[a] / vol->spacing[a]) * (r[a] / vol->spacing[a]);
    return pitch * std::sqrt(q);
}

// Brick copy for a camera.  Its fastest axis is the one along which the
// image's horizontal direction (in voxel units) is longest, so that a warp's
// row of eight rays reads neighbouring elements; a view along x reads the
// bricks themselves.  16-bit volumes take paired copies (two corners per
// load) while neighbouring rays are closer than VR_PAIRED_MAX_PITCH voxels
// (default 3) at the volume centre, where a warp's gathers share cache lines
// and the number of loads bounds the march; sparser rays each touch their own
// sectors in DRAM, so the plain copy (half the bytes of a paired one) serves,
// or, for the forward kernels of a 16-bit volume, a blocked copy (a cell's
// 2 x 2 columns in 32-byte blocks deep along the view direction).
// A copy is built on first use when `may_build`, the stream is not being
// captured and the device keeps an eighth of its memory free besides it; it
// is complete before the call returns, so any stream may read it.  Otherwise
// (or with VR_BRICK_COPIES=0 in the environment) the bricks serve (-1).
int preferred_copy(vr_volume *vol, const vr_camera *cam, bool may_build, cudaStream_t s, unsigned kinds)
{
    const bool allow_blocked = (kinds & kReadsBlocked) != 0;
    static const bool enabled = [] {
        const char *e = std::getenv("VR_BRICK_COPIES");
        return !(e && e[0] == '0');
    }();
    static const double max_pitch = [] {
        const char *e = std::getenv("VR_PAIRED_MAX_PITCH");
        return e ? std::atof(e) : 3.0;
    }();
    static const double sparse_pitch = [] {
        const char *e = std::getenv("VR_SPARSE_MIN_PITCH");
        return e ? std::atof(e) : 3.0;
    }();
    // layout of sparse views (VR_SPARSE_LAYOUT): 'b' blocked copies (forward
    // kernels only), 'i' as dense views (rows along the image's horizontal
    // axis); default 'b' for 16-bit storage in bricks smaller than 64^3 and
    // 'i' otherwise, as measured on the four 1080p views of the 4096 x 4096 x
    // 1024 cube (16-bit in 16^3 bricks: blocked 83.6 against 80.2 Gsamples/s
    // for rows; in 64^3 bricks, this cube's default: rows 119 against 92.4;
    // float: the two blocked copies its views want do not fit beside the
    // cube, and the row copies serve every view)
    static const char sparse_env = [] {
        const char *e = std::getenv("VR_SPARSE_LAYOUT");
        return e && (e[0] == 'b' || e[0] == 'i') ? e[0] : 0;
    }();
    const char sparse_mode = sparse_env ? sparse_env : (vol->store_dtype == VR_F32 || vol->log2b >= 6 ? 'i' : 'b');
    if (!enabled) return -1;
    double f[3] = {cam->forward[0], cam->forward[1], cam->forward[2]}, r[3];
    cross3(f, cam->up, r);
    const double rl = std::sqrt(dot3(r, r));
    for (double &x : r) x /= rl;
    double best = -1.0;
    int axis = 0;
    for (int a = 0; a < 3; ++a) {
        const double c = std::fabs(r[a]) / vol->spacing[a];
        if (c > best * (1.0 + 1e-9)) {
            best = c;
            axis = a;
        }
    }
    const double pitch = ray_pitch_voxels(vol, cam, r);
    // Dense views of a float volume read a texture-layer copy across the axis
    // the view direction runs along most (in voxel units), so that the image's
    // rows and columns lie in the layers, where the texture's tiling keeps both
    // local (VR_TEX_LAYERS=0, read at each call, turns this off).  Measured on
    // the 1024^3 eight-view workload: 177 against 141 Gsamples/s for the brick
    // copies, bit-identical images.  16-bit storage keeps its paired copies
    // (the gathers there are bound by the texture unit's texel rate).
    const char *tl = std::getenv("VR_TEX_LAYERS");
    if ((kinds & kReadsLayers) && vol->store_dtype == VR_F32 && pitch < sparse_pitch && !(tl && tl[0] == '0')) {
        int w = 0;
        double m = -1.0;
        for (int a = 0; a < 3; ++a) {
            const double c = std::fabs(cam->forward[a]) / vol->spacing[a];
            if (c > m * (1.0 + 1e-9)) m = c, w = a;
        }
        const int lcopy = 9 + w;
        if (copy_built(vol, lcopy)) return lcopy;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        size_t free_b = 0, total_b = 0;
        if (may_build && cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone &&
            cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && free_b >= copy_bytes(vol, lcopy) + total_b / 8) {
            log_line("view %dx%d prefers texture layers across axis %d; building them", cam->width, cam->height, w);
            if (build_layers(vol, w, s) == cudaSuccess) return lcopy;
        }
        cudaGetLastError();        // no layers (limits, memory, capture): the brick copies serve
    }
    const bool paired = vol->store_dtype != VR_F32 && pitch < max_pitch;
    int copy = paired ? 3 + axis : axis;
    if (pitch >= sparse_pitch && sparse_mode == 'b' && allow_blocked) {
        // rays too far apart to share sectors: each ray reads its own, so the
        // blocks are deep along the axis w the rays advance along most
        int w = 0;
        double m = -1.0;
        for (int a = 0; a < 3; ++a) {
            const double c = std::fabs(cam->forward[a]) / vol->spacing[a];
            if (c > m * (1.0 + 1e-9)) m = c, w = a;
        }
        copy = 6 + w;
    }
    if (copy == 0) return -1;
    if (vol->copies[copy]) return copy;
    if (!may_build) return -1;
    log_line("view %dx%d prefers brick copy %d (%s); building it", cam->width, cam->height, copy,
             copy_paired(copy) ? "paired" : (copy_blocked(copy) ? "blocked" : "plain"));
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return -1;
    }
    const size_t bytes = copy_bytes(vol, copy);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess || free_b < bytes + total_b / 8) {
        cudaGetLastError();
        return -1;
    }
    void *p = nullptr;
    if (dev_alloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    vol->copies[copy] = p;
    if (launch_copy(vol, copy, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(p);
        vol->copies[copy] = nullptr;
        return -1;
    }
    return copy;
}

// Voxel-gradient scratch for a backward pass.  One 16-byte quad reduction per
// plane of four corners replaces two to four scalar or pair reductions into
// the dense gradient, at the cost of clearing and gathering 16 bytes per
// voxel once per call, and its DRAM traffic (it does not stay in L2) once
// per view; it pays where each voxel takes many samples: by default where
// the call's views put at least one sample per voxel on average, estimated
// from the ray pitch and the step at the volume centre
// (VR_GRAD_DIRECT / VR_GRAD_SCRATCH override it).  Created
// on first use when the stream is not being captured and the device keeps an
// eighth of its memory free besides it.
static float4 *grad_quad_for(vr_volume *vol, const vr_grad_view *views, int n, const vr_params *params,
                             unsigned flags, cudaStream_t s)
{
    if (flags & VR_GRAD_DIRECT) return nullptr;
    if (!(flags & VR_GRAD_SCRATCH)) {
        const double sp = (vol->spacing[0] + vol->spacing[1] + vol->spacing[2]) / 3.0;
        const double unit[3] = {1.0, 0.0, 0.0};
        const double step = params->step / sp;                                  // in voxels
        double density = 0.0;                                                   // samples per voxel, all views
        for (int q = 0; q < n; ++q) {
            const double pitch = ray_pitch_voxels(vol, &views[q].cam, unit) * vol->spacing[0] / sp;   // in voxels
            if (pitch > 0.0) density += 1.0 / (pitch * pitch * step);
        }
        // every view's kernel reads and writes the scratch once more (it does not
        // stay in L2), so the views must be dense on average, not only together
        if (!(density >= (double)n)) {
            log_line("backward of %d view(s): direct voxel-gradient reductions (%.2f samples per voxel per view)", n,
                     density / n);
            return nullptr;
        }
    }
    log_line("backward of %d view(s): voxel gradient through the quad scratch", n);
    if (vol->gquad) return vol->gquad;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return nullptr;
    }
    const size_t bytes = sizeof(float4) * (size_t)vol->dims[0] * (size_t)vol->dims[1] * (size_t)vol->dims[2];
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess || free_b < bytes + total_b / 8) {
        cudaGetLastError();
        return nullptr;
    }
    void *p = nullptr;
    if (dev_alloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    vol->gquad = static_cast<float4 *>(p);
    return vol->gquad;
}

// Carry axis of the backward's voxel-gradient sums: the axis along which the
// view direction (in voxel units) is longest, so that most of a ray's cell
// steps move along it.
static int carry_axis(const vr_volume *vol, const vr_camera *cam)
{
    int a = 0;
    double best = -1.0;
    for (int q = 0; q < 3; ++q) {
        const double m = std::fabs(cam->forward[q] / vol->spacing[q]);
        if (m > best) best = m, a = q;
    }
    return a;
}

// The last slot of the ring is the volume's device status word.
vr_status next_counter(vr_volume *vol, unsigned **ctr)
{
    *ctr = vol->counters + vol->next_counter;
    vol->next_counter = (vol->next_counter + 1) % (vol->counter_slots - 1);
    return VR_OK;
}

static unsigned *status_word(vr_volume *vol) { return vol->counters + vol->counter_slots - 1; }

// Backward scratch (per-warp gradient rows), grown on demand.  Growing waits
// for the stream so that no running kernel still uses the old buffer.
cudaError_t ensure_wtab(vr_volume *vol, size_t floats, cudaStream_t s)
{
    if (floats <= vol->wtab_cap) return cudaSuccess;
    if (vol->wtab) {
        cudaStreamSynchronize(s);
        cudaFree(vol->wtab);
        vol->wtab = nullptr;
        vol->wtab_cap = 0;
    }
    cudaError_t e = dev_alloc(reinterpret_cast<void **>(&vol->wtab), floats * sizeof(float));
    if (e != cudaSuccess) {
        vol->wtab = nullptr;
        return e;
    }
    vol->wtab_cap = floats;
    return cudaSuccess;
}

// The dense row-padded copy used by the staged kernels, built from the bricks
// on first use.
static vr_status ensure_dense(vr_volume *vol, cudaStream_t s)
{
    if (vol->dense) return VR_OK;
    const int px = (int)((vol->dims[0] + 7) / 8 * 8);
    const size_t bytes = (size_t)px * (size_t)vol->dims[1] * (size_t)vol->dims[2] * (vol->store_dtype == VR_F32 ? 4 : 2);
    void *p = nullptr;
    if (dev_alloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("staged filter: cannot allocate the dense copy (" + std::to_string(bytes) + " bytes)");
        return VR_ERR_OOM;
    }
    vol->dense = p;
    vol->dense_px = px;
    vol->dense_bytes = bytes;
    cudaError_t e = launch_dense_from_bricks(vol, s);
    if (e != cudaSuccess) return cuda_fail(e, "staged filter: dense copy");
    return VR_OK;
}

vr_status validate_job(const vr_job *J, int q)
{
    const std::string where = "jobs[" + std::to_string(q) + "]: ";
    vr_status st = check_camera(&J->cam);
    if (st == VR_OK) st = check_params(&J->params);
    if (st == VR_OK) st = check_volume(J->vol);
    if (st == VR_OK) st = check_step(J->vol, &J->params);
    if (st == VR_OK) st = check_mode_path(&J->params, "batched render");
    if (st != VR_OK) set_error(where + g_err);
    return st;
}

static size_t dtype_size(vr_dtype d) { return d == VR_F32 ? 4 : 2; }

static void free_volume(vr_volume *vol)
{
    if (vol->tex) cudaDestroyTextureObject(vol->tex);
    if (vol->tex_array) cudaFreeArray(vol->tex_array);
    if (vol->bricks) cudaFree(vol->bricks);
    if (vol->dense) cudaFree(vol->dense);
    if (vol->wtab) cudaFree(vol->wtab);
    if (vol->gquad) cudaFree(vol->gquad);
    if (vol->stats) cudaFree(vol->stats);
    if (vol->brick_range) cudaFree(vol->brick_range);
    for (void *o : vol->copies)
        if (o) cudaFree(o);
    free_layers(vol);
    if (vol->counters) cudaFree(vol->counters);
    for (cudaStream_t a : vol->aux)
        if (a) cudaStreamDestroy(a);
    for (cudaEvent_t ev : vol->aux_ev)
        if (ev) cudaEventDestroy(ev);
    delete vol;
}

}  // namespace vr

using namespace vr;

extern "C" {

const char *vr_last_error(void) { return g_err.c_str(); }

const char *vr_version(void) { return "vr-gb300 0.1 (sm_103a)"; }

// A volume handle with its bricks and counters allocated (not filled).
static vr_status make_volume(vr_dtype src_dtype, vr_dtype store_dtype, const int64_t dims[3], const double origin[3],
                             const double spacing[3], int brick, vr_volume **out)
{
    *out = nullptr;
    if (!dims) return invalid("dims is NULL");
    if ((unsigned)src_dtype > VR_BF16 || (unsigned)store_dtype > VR_BF16)
        return invalid("dtype must be VR_F32, VR_F16 or VR_BF16");
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 2 || dims[a] > (1 << 20)) return invalid("each of dims must be in [2, 2^20]");
    if (dims[0] * dims[1] > (int64_t)1 << 31) return invalid("nx * ny must be <= 2^31");
    if (origin && !finite3(origin)) return invalid("origin must be finite");
    if (spacing && !(spacing[0] > 0 && spacing[1] > 0 && spacing[2] > 0 && finite3(spacing)))
        return invalid("spacing must be finite and > 0");
    if (brick == 0) {
        // 16^3 bricks, or 64^3 once 16^3 bricks would pass 16 GiB: the rays of
        // such a volume's views are far apart and cross a brick every B steps,
        // and larger bricks (less apron, fewer brick changes) were faster on
        // the four 1080p views of the 4096 x 4096 x 1024 cube (float 59-63 ->
        // 72-84, 16-bit 80-86 -> 88-97 Gsamples/s per view)
        double bytes16 = store_dtype == VR_F32 ? 4.0 : 2.0;
        for (int a = 0; a < 3; ++a) bytes16 *= (double)((dims[a] - 1 + 15) / 16) * 17.0;
        brick = bytes16 > 16.0 * (1 << 30) ? 64 : 16;
    }
    int log2b = 0;
    switch (brick) {
    case 16: log2b = 4; break;
    case 32: log2b = 5; break;
    case 64: log2b = 6; break;
    default: return invalid("brick must be 0 (auto), 16, 32 or 64");
    }
    vr_volume *vol = new (std::nothrow) vr_volume();
    if (!vol) return invalid("host allocation failed");
    for (int a = 0; a < 3; ++a) {
        vol->dims[a] = dims[a];
        vol->origin[a] = origin ? origin[a] : 0.0;
        vol->spacing[a] = spacing ? spacing[a] : 1.0;
        vol->nb[a] = (dims[a] - 1 + brick - 1) / brick;       // bricks cover cells [0, n-2]
    }
    vol->src_dtype = src_dtype;
    vol->store_dtype = store_dtype;
    vol->brick = brick;
    vol->log2b = log2b;
    const long long b1 = brick + 1;
    vol->stride = (b1 * b1 * b1 + 63) / 64 * 64;                // 64-element (>=128 B) aligned bricks
    const long long nbricks = vol->nb[0] * vol->nb[1] * vol->nb[2];
    if (nbricks >= (1LL << 31)) {
        free_volume(vol);
        return invalid("the volume needs 2^31 or more bricks");
    }
    vol->bytes = (size_t)nbricks * (size_t)vol->stride * dtype_size(store_dtype);
    cudaError_t e = cudaGetDevice(&vol->device);
    if (e != cudaSuccess) { free_volume(vol); return cuda_fail(e, "cudaGetDevice"); }
    e = dev_alloc(&vol->bricks, vol->bytes);
    if (e != cudaSuccess) {
        vol->bricks = nullptr;
        free_volume(vol);
        cudaGetLastError();
        set_error("vr_volume_create: cannot allocate " + std::to_string(vol->bytes) + " bytes of bricks");
        return VR_ERR_OOM;
    }
    vol->counter_slots = 64;
    e = dev_alloc(reinterpret_cast<void **>(&vol->counters), sizeof(unsigned) * vol->counter_slots);
    if (e != cudaSuccess) { vol->counters = nullptr; free_volume(vol); return cuda_fail(e, "cudaMalloc(counters)"); }
    *out = vol;
    return VR_OK;
}

vr_status vr_volume_create(const void *dev_cube, vr_dtype src_dtype, vr_dtype store_dtype, const int64_t dims[3],
                           const double origin[3], const double spacing[3], int brick, void *cuda_stream,
                           vr_volume_t *out)
{
    g_err.clear();
    if (!out) return invalid("out is NULL");
    *out = nullptr;
    if (!dev_cube) return invalid("dev_cube is NULL");
    vr_volume *vol = nullptr;
    vr_status st = make_volume(src_dtype, store_dtype, dims, origin, spacing, brick, &vol);
    if (st != VR_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaMemsetAsync(vol->counters, 0, sizeof(unsigned) * vol->counter_slots, s);
    if (e == cudaSuccess) e = launch_brick(dev_cube, src_dtype, vol, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { free_volume(vol); return cuda_fail(e, "vr_volume_create: bricking"); }
    *out = vol;
    return VR_OK;
}

vr_status vr_volume_rebrick(vr_volume_t src, int brick, void *cuda_stream, vr_volume_t *out)
{
    g_err.clear();
    if (!out) return invalid("out is NULL");
    *out = nullptr;
    vr_status st = check_volume(src);
    if (st != VR_OK) return st;
    vr_volume *vol = nullptr;
    st = make_volume(src->src_dtype, src->store_dtype, src->dims, src->origin, src->spacing, brick, &vol);
    if (st != VR_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaMemsetAsync(vol->counters, 0, sizeof(unsigned) * vol->counter_slots, s);
    if (e == cudaSuccess) e = launch_rebrick(src, vol, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { free_volume(vol); return cuda_fail(e, "vr_volume_rebrick"); }
    *out = vol;
    return VR_OK;
}

vr_status vr_volume_update(vr_volume_t vol, const void *dev_cube, vr_dtype src_dtype, void *cuda_stream)
{
    g_err.clear();
    vr_status st = check_volume(vol);
    if (st != VR_OK) return st;
    if (!dev_cube) return invalid("dev_cube is NULL");
    if (src_dtype != vol->src_dtype) return invalid("src_dtype differs from the one given at creation");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (vol->tex) {            // the hardware-filter copy is now stale
        cudaStreamSynchronize(s);
        cudaDestroyTextureObject(vol->tex);
        cudaFreeArray(vol->tex_array);
        vol->tex = 0;
        vol->tex_array = nullptr;
    }
    cudaError_t e = launch_brick(dev_cube, src_dtype, vol, s);
    for (int c = 1; c < kCopyIds && e == cudaSuccess; ++c)
        if (copy_built(vol, c)) e = launch_copy(vol, c, s);
    if (e == cudaSuccess && vol->brick_range) e = launch_brick_range(vol_dev(vol), vol->store_dtype, vol->brick_range, s);
    if (e == cudaSuccess && vol->dense) e = launch_densify(dev_cube, src_dtype, vol, s);
    if (e != cudaSuccess) return cuda_fail(e, "vr_volume_update");
    return VR_OK;
}

vr_status vr_volume_destroy(vr_volume_t vol)
{
    g_err.clear();
    if (!vol) return VR_OK;
    cudaDeviceSynchronize();
    purge_plans(vol);
    free_volume(vol);
    return VR_OK;
}

vr_status vr_view_layout(vr_volume_t vol, const vr_camera *cam, int *layout)
{
    g_err.clear();
    vr_status st = check_camera(cam);
    if (st != VR_OK) return st;
    if (!vol) return invalid("volume handle is NULL");
    if (!layout) return invalid("layout is NULL");
    *layout = preferred_copy(vol, cam, false, nullptr, kReadsBlocked | kReadsLayers);
    return VR_OK;
}

vr_status vr_volume_info(vr_volume_t vol, vr_volume_info_t *out)
{
    g_err.clear();
    if (!vol) return invalid("volume handle is NULL");
    if (!out) return invalid("out is NULL");
    for (int a = 0; a < 3; ++a) {
        out->dims[a] = vol->dims[a];
        out->bricks[a] = vol->nb[a];
    }
    out->store_dtype = vol->store_dtype;
    out->brick = vol->brick;
    out->bytes = (int64_t)vol->bytes;
    out->dense_bytes = (int64_t)vol->dense_bytes;
    out->copy_bytes = 0;
    out->copies = 0;
    out->scratch_bytes = (int64_t)(vol->wtab_cap * sizeof(float)) +
                         (vol->gquad ? (int64_t)sizeof(float4) * vol->dims[0] * vol->dims[1] * vol->dims[2] : 0);
    for (int c = 1; c < kCopyIds; ++c)
        if (copy_built(vol, c)) {
            out->copy_bytes += (int64_t)copy_bytes(vol, c);
            out->copies |= 1 << c;
        }
    return VR_OK;
}

vr_status vr_render(vr_volume_t vol, const vr_camera *cam, const vr_params *params, float *dev_rgba_out,
                    uint32_t *dev_nsamples_out, void *cuda_stream)
{
    g_err.clear();
    vr_status st = check_camera(cam);
    if (st == VR_OK) st = check_params(params);
    if (st != VR_OK) return st;
    if (!dev_rgba_out) return invalid("dev_rgba_out is NULL");
    if (!is_aligned16(dev_rgba_out)) return invalid("dev_rgba_out must be 16-byte aligned");
    if ((reinterpret_cast<uintptr_t>(dev_nsamples_out) & 3u) != 0) return invalid("dev_nsamples_out must be 4-byte aligned");
    st = check_volume(vol);
    if (st == VR_OK) st = check_step(vol, params);
    if (st != VR_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    CamDev c;
    ParamDev p;
    prepare_camera(vol, cam, &c);
    prepare_params(params, &p);
    unsigned *ctr;
    next_counter(vol, &ctr);
    cudaError_t e;
    if (params->mode != VR_MODE_COMPOSITE && params->filter != VR_FILTER_SOFTWARE)
        return (set_error("vr_render: VR_MODE_MIP and VR_MODE_SIGMA need VR_FILTER_SOFTWARE"), VR_ERR_UNSUPPORTED);
    if (params->skip_empty && (params->mode != VR_MODE_COMPOSITE || params->filter != VR_FILTER_SOFTWARE))
        return (set_error("vr_render: skip_empty needs VR_MODE_COMPOSITE and VR_FILTER_SOFTWARE"),
                VR_ERR_UNSUPPORTED);
    if (params->skip_empty) {
        const size_t nbr = (size_t)(vol->nb[0] * vol->nb[1] * vol->nb[2]);
        if (!vol->brick_range) {
            // the ranges, then one transparency bit per brick (rewritten by every call)
            e = dev_alloc(reinterpret_cast<void **>(&vol->brick_range),
                          nbr * sizeof(float2) + (nbr + 31) / 32 * sizeof(uint32_t));
            if (e != cudaSuccess) {
                vol->brick_range = nullptr;
                return cuda_fail(e, "vr_render: brick ranges");
            }
            e = launch_brick_range(vol_dev(vol), vol->store_dtype, vol->brick_range, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                cudaFree(vol->brick_range);
                vol->brick_range = nullptr;
                return cuda_fail(e, "vr_render: brick ranges");
            }
        }
        e = launch_forward_skip(vol_dev_copy(vol, preferred_copy(vol, cam, true, s, kReadsLayers)), vol->store_dtype,
                                c, p,
                                vol->brick_range, reinterpret_cast<uint32_t *>(vol->brick_range + nbr),
                                reinterpret_cast<float4 *>(dev_rgba_out), dev_nsamples_out, ctr, s);
    } else if (params->mode == VR_MODE_MIP) {
        e = launch_mip(vol_dev_copy(vol, preferred_copy(vol, cam, true, s, kReadsLayers)), vol->store_dtype, c, p,
                       reinterpret_cast<float4 *>(dev_rgba_out), dev_nsamples_out, ctr, s);
    } else if (params->mode == VR_MODE_SIGMA) {
        e = launch_sigma(vol_dev_copy(vol, preferred_copy(vol, cam, true, s, kReadsLayers)), vol->store_dtype, c, p,
                         params->minimap, params->minimap_region, reinterpret_cast<float4 *>(dev_rgba_out),
                         dev_nsamples_out, ctr, s);
    } else if (params->filter == VR_FILTER_TEXTURE) {
        st = build_texture(vol, s);
        if (st != VR_OK) return st;
        e = launch_forward_texture(vol, c, p, reinterpret_cast<float4 *>(dev_rgba_out), dev_nsamples_out, ctr, s);
    } else if (params->filter == VR_FILTER_SOFTWARE_STAGED) {
        st = ensure_dense(vol, s);
        if (st != VR_OK) return st;
        e = launch_forward_staged(dense_dev(vol), vol->store_dtype, c, p, reinterpret_cast<float4 *>(dev_rgba_out),
                                  dev_nsamples_out, ctr, status_word(vol), s);
    } else {
        e = launch_forward(vol_dev_copy(vol, preferred_copy(vol, cam, true, s, kReadsBlocked | kReadsLayers)),
                           vol->store_dtype, c, p,
                           reinterpret_cast<float4 *>(dev_rgba_out), dev_nsamples_out, ctr, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "vr_render launch");
    return VR_OK;
}

static vr_status backward_views(vr_volume_t vol, const vr_grad_view *views, int n, const vr_params *params,
                                double *dev_grad_tf, float *dev_grad_vox, unsigned flags, void *cuda_stream,
                                const char *who)
{
    g_err.clear();
    if (n < 1 || !views) return invalid(std::string(who) + ": at least one view is required");
    if (n > 4096) return invalid(std::string(who) + ": at most 4096 views per call");
    vr_status st = check_params(params);
    if (st == VR_OK) st = check_mode_path(params, who);
    if (st != VR_OK) return st;
    for (int q = 0; q < n; ++q) {
        st = check_camera(&views[q].cam);
        if (st != VR_OK) return (n > 1 ? set_error("views[" + std::to_string(q) + "]: " + g_err) : void()), st;
    }
    if (params->filter == VR_FILTER_TEXTURE)
        return (set_error(std::string(who) + ": only the software filters are differentiable"), VR_ERR_UNSUPPORTED);
    if (!(params->bg_rgba[3] < 1.0f))
        return (set_error(std::string(who) + ": bg alpha must be < 1 (T_final is recovered from the output alpha)"),
                VR_ERR_UNSUPPORTED);
    for (int q = 0; q < n; ++q) {
        const vr_grad_view &w = views[q];
        if (!w.rgba || !w.nsamples || !w.grad_rgba)
            return invalid("dev_rgba, dev_nsamples and dev_grad_rgba must not be NULL");
        if (!is_aligned16(w.rgba) || !is_aligned16(w.grad_rgba))
            return invalid("dev_rgba and dev_grad_rgba must be 16-byte aligned");
        if ((reinterpret_cast<uintptr_t>(w.nsamples) & 3u) != 0) return invalid("dev_nsamples must be 4-byte aligned");
    }
    if (!dev_grad_tf) return invalid("dev_grad_tf must not be NULL");
    if ((reinterpret_cast<uintptr_t>(dev_grad_tf) & 7u) != 0) return invalid("dev_grad_tf must be 8-byte aligned");
    if (flags & ~(unsigned)(VR_GRAD_ACCUMULATE | VR_GRAD_DIRECT | VR_GRAD_SCRATCH))
        return invalid("flags: unknown bits");
    if ((flags & VR_GRAD_DIRECT) && (flags & VR_GRAD_SCRATCH))
        return invalid("flags: VR_GRAD_DIRECT and VR_GRAD_SCRATCH exclude each other");
    if (params->tf_size > backward_max_tf_size())
        return (set_error(std::string(who) + ": tf_size above " + std::to_string(backward_max_tf_size()) +
                          " (per-warp gradient bins must fit in shared memory)"), VR_ERR_UNSUPPORTED);
    if ((reinterpret_cast<uintptr_t>(dev_grad_vox) & 3u) != 0) return invalid("dev_grad_vox must be 4-byte aligned");
    st = check_volume(vol);
    if (st == VR_OK) st = check_step(vol, params);
    if (st != VR_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    ParamDev p;
    prepare_params(params, &p);
    const long long nvox = (long long)vol->dims[0] * vol->dims[1] * vol->dims[2];
    unsigned *ctr;
    next_counter(vol, &ctr);
    const bool acc = (flags & VR_GRAD_ACCUMULATE) != 0;
    cudaError_t e = cudaSuccess;
    if (params->filter == VR_FILTER_SOFTWARE_STAGED) {
        st = ensure_dense(vol, s);
        if (st != VR_OK) return st;
        for (int q = 0; q < n && e == cudaSuccess; ++q) {
            CamDev c;
            prepare_camera(vol, &views[q].cam, &c);
            e = launch_backward_staged(dense_dev(vol), vol->store_dtype, c, p,
                                       reinterpret_cast<const float4 *>(views[q].rgba), views[q].nsamples,
                                       reinterpret_cast<const float4 *>(views[q].grad_rgba), dev_grad_tf,
                                       dev_grad_vox, nvox, acc || q > 0, ctr, status_word(vol), s);
        }
    } else {
        std::vector<BwdView> bv((size_t)n);
        int votes[3] = {0, 0, 0};
        for (int q = 0; q < n; ++q) {
            prepare_camera(vol, &views[q].cam, &bv[q].c);
            bv[q].v = vol_dev_copy(vol, preferred_copy(vol, &views[q].cam, true, s, kReadsLayers));
            bv[q].rgba = reinterpret_cast<const float4 *>(views[q].rgba);
            bv[q].grad_rgba = reinterpret_cast<const float4 *>(views[q].grad_rgba);
            bv[q].nsamples = views[q].nsamples;
            bv[q].carry_axis = carry_axis(vol, &views[q].cam);
            ++votes[bv[q].carry_axis];
        }
        const int quad_axis = votes[2] >= votes[0] && votes[2] >= votes[1] ? 2 : (votes[0] >= votes[1] ? 0 : 1);
        float4 *quad = dev_grad_vox ? grad_quad_for(vol, views, n, params, flags, s) : nullptr;
        e = launch_backward(vol, bv.data(), n, p, dev_grad_tf, dev_grad_vox, quad, quad_axis, nvox, acc, ctr, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, who);
    return VR_OK;
}

vr_status vr_render_backward(vr_volume_t vol, const vr_camera *cam, const vr_params *params, const float *dev_rgba,
                             const uint32_t *dev_nsamples, const float *dev_grad_rgba, double *dev_grad_tf,
                             float *dev_grad_vox, unsigned flags, void *cuda_stream)
{
    if (!cam) {
        g_err.clear();
        return invalid("camera is NULL");
    }
    vr_grad_view w;
    w.cam = *cam;
    w.rgba = dev_rgba;
    w.nsamples = dev_nsamples;
    w.grad_rgba = dev_grad_rgba;
    return backward_views(vol, &w, 1, params, dev_grad_tf, dev_grad_vox, flags, cuda_stream, "vr_render_backward");
}

vr_status vr_render_backward_views(vr_volume_t vol, const vr_grad_view *views, int n, const vr_params *params,
                                   double *dev_grad_tf, float *dev_grad_vox, unsigned flags, void *cuda_stream)
{
    return backward_views(vol, views, n, params, dev_grad_tf, dev_grad_vox, flags, cuda_stream,
                          "vr_render_backward_views");
}

vr_status vr_minimap(vr_volume_t vol, const int region[3], float *dev_minimap, void *cuda_stream)
{
    g_err.clear();
    vr_status st = check_volume(vol);
    if (st != VR_OK) return st;
    if (!region) return invalid("region is NULL");
    for (int a = 0; a < 3; ++a)
        if (region[a] < 1) return invalid("region must be >= 1 per axis");
    if (!dev_minimap || (reinterpret_cast<uintptr_t>(dev_minimap) & 7u) != 0)
        return invalid("dev_minimap must be non-NULL and 8-byte aligned");
    cudaError_t e = launch_minimap(vol_dev(vol), vol->store_dtype, region, dev_minimap,
                                   static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail(e, "vr_minimap launch");
    return VR_OK;
}

vr_status vr_profile(vr_volume_t vol, const vr_camera *cam, float step, int i, int j, float *dev_values,
                     uint32_t max_values, uint32_t *dev_count, void *cuda_stream)
{
    g_err.clear();
    vr_status st = check_camera(cam);
    if (st == VR_OK) st = check_volume(vol);
    if (st != VR_OK) return st;
    if (!std::isfinite(step) || !(step > 0.0f)) return invalid("step must be finite and > 0");
    if (i < 0 || j < 0 || i >= cam->width || j >= cam->height) return invalid("pixel (i, j) outside the image");
    if (!dev_count || (reinterpret_cast<uintptr_t>(dev_count) & 3u) != 0)
        return invalid("dev_count must be non-NULL and 4-byte aligned");
    if (max_values > 0 && (!dev_values || (reinterpret_cast<uintptr_t>(dev_values) & 3u) != 0))
        return invalid("dev_values must be non-NULL and 4-byte aligned when max_values > 0");
    vr_params tmp{};
    tmp.step = step;
    st = check_step(vol, &tmp);
    if (st != VR_OK) return st;
    CamDev c;
    prepare_camera(vol, cam, &c);
    cudaError_t e = launch_profile(vol_dev(vol), vol->store_dtype, c, step, i, j, dev_values, max_values, dev_count,
                                   static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail(e, "vr_profile launch");
    return VR_OK;
}

static vr_status subbox_of(vr_volume_t vol, const int64_t gdims[3], const int64_t offset[3], const vr_camera *cam,
                           const vr_params *params, const int cell_lo[3], const int cell_hi[3], float *dev_partial,
                           float *dev_depth, uint32_t *dev_count, void *cuda_stream, const char *who)
{
    g_err.clear();
    vr_status st = check_camera(cam);
    if (st == VR_OK) st = check_params(params);
    if (st == VR_OK) st = check_mode_path(params, who);
    if (st != VR_OK) return st;
    if (params->filter != VR_FILTER_SOFTWARE)
        return (set_error(std::string(who) + ": software filter only"), VR_ERR_UNSUPPORTED);
    st = check_volume(vol);
    if (st == VR_OK) st = check_step(vol, params);
    if (st != VR_OK) return st;
    if (!gdims || !offset) return invalid("global_dims and offset must not be NULL");
    for (int a = 0; a < 3; ++a) {
        if (gdims[a] < 2 || gdims[a] > (int64_t)1 << 30) return invalid("global_dims must be in [2, 2^30] per axis");
        if (offset[a] < 0 || offset[a] + vol->dims[a] > gdims[a])
            return invalid("need 0 <= offset and offset + dims <= global_dims per axis");
    }
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double e = (double)(gdims[a] - 1) * vol->spacing[a];
        d2 += e * e;
    }
    if (std::sqrt(d2) / (double)params->step > 16777216.0) return invalid("params.step too small: > 2^24 samples per ray");
    if (!cell_lo || !cell_hi) return invalid("cell_lo and cell_hi must not be NULL");
    for (int a = 0; a < 3; ++a)
        if (cell_lo[a] < offset[a] || cell_hi[a] > offset[a] + vol->dims[a] - 1 || cell_lo[a] >= cell_hi[a])
            return invalid("need offset <= cell_lo < cell_hi <= offset + dims - 1 (cells) per axis");
    if (!dev_partial || !is_aligned16(dev_partial)) return invalid("dev_partial must be non-NULL and 16-byte aligned");
    if (!dev_depth || (reinterpret_cast<uintptr_t>(dev_depth) & 3u) != 0)
        return invalid("dev_depth must be non-NULL and 4-byte aligned");
    if ((reinterpret_cast<uintptr_t>(dev_count) & 3u) != 0) return invalid("dev_count must be 4-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the camera in the whole grid's voxel coordinates: its first voxel sits
    // offset voxels before this volume's
    double gorigin[3];
    for (int a = 0; a < 3; ++a) gorigin[a] = vol->origin[a] - (double)offset[a] * vol->spacing[a];
    CamDev c;
    ParamDev p;
    prepare_camera_grid(gorigin, vol->spacing, gdims, cam, &c);
    prepare_params(params, &p);
    unsigned *ctr;
    next_counter(vol, &ctr);
    const int gd[3] = {(int)gdims[0], (int)gdims[1], (int)gdims[2]};
    const int off[3] = {(int)offset[0], (int)offset[1], (int)offset[2]};
    cudaError_t e = launch_subbox(vol_dev_copy(vol, preferred_copy(vol, cam, true, s, kReadsLayers)), vol->store_dtype,
                                  c, p,
                                  cell_lo, cell_hi, gd, off, reinterpret_cast<float4 *>(dev_partial), dev_depth,
                                  dev_count, ctr, s);
    if (e != cudaSuccess) return cuda_fail(e, who);
    return VR_OK;
}

vr_status vr_render_subbox(vr_volume_t vol, const vr_camera *cam, const vr_params *params, const int cell_lo[3],
                           const int cell_hi[3], float *dev_partial, float *dev_depth, uint32_t *dev_count,
                           void *cuda_stream)
{
    if (!vol) {
        g_err.clear();
        return invalid("volume handle is NULL");
    }
    const int64_t zero[3] = {0, 0, 0};
    return subbox_of(vol, vol->dims, zero, cam, params, cell_lo, cell_hi, dev_partial, dev_depth, dev_count,
                     cuda_stream, "vr_render_subbox");
}

vr_status vr_render_subbox_of(vr_volume_t vol, const int64_t global_dims[3], const int64_t offset[3],
                              const vr_camera *cam, const vr_params *params, const int cell_lo[3],
                              const int cell_hi[3], float *dev_partial, float *dev_depth, uint32_t *dev_count,
                              void *cuda_stream)
{
    return subbox_of(vol, global_dims, offset, cam, params, cell_lo, cell_hi, dev_partial, dev_depth, dev_count,
                     cuda_stream, "vr_render_subbox_of");
}

vr_status vr_composite(int k, const float *const *dev_partials, const float *const *dev_depths, int width,
                       int height, const float bg_rgba[4], float *dev_rgba_out, void *cuda_stream)
{
    g_err.clear();
    if (k < 1 || k > kMaxPartials) return invalid("k must be in [1, " + std::to_string(kMaxPartials) + "]");
    if (!dev_partials || !dev_depths) return invalid("dev_partials and dev_depths must not be NULL");
    if (width < 1 || height < 1 || width > 32768 || height > 32768)
        return invalid("width and height must be in [1, 32768]");
    if (!bg_rgba) return invalid("bg_rgba is NULL");
    for (int q = 0; q < k; ++q) {
        if (!dev_partials[q] || !is_aligned16(dev_partials[q]))
            return invalid("dev_partials[" + std::to_string(q) + "] must be non-NULL and 16-byte aligned");
        if (!dev_depths[q] || (reinterpret_cast<uintptr_t>(dev_depths[q]) & 3u) != 0)
            return invalid("dev_depths[" + std::to_string(q) + "] must be non-NULL and 4-byte aligned");
    }
    if (!dev_rgba_out || !is_aligned16(dev_rgba_out)) return invalid("dev_rgba_out must be non-NULL and 16-byte aligned");
    cudaError_t e = launch_composite(k, dev_partials, dev_depths, (long long)width * height, bg_rgba, dev_rgba_out,
                                     static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail(e, "vr_composite launch");
    return VR_OK;
}

static vr_status ensure_stats(vr_volume *vol)
{
    if (vol->stats) return VR_OK;
    cudaError_t e = dev_alloc(&vol->stats, stats_scratch_bytes());
    if (e != cudaSuccess) {
        vol->stats = nullptr;
        return cuda_fail(e, "statistics scratch");
    }
    return VR_OK;
}

vr_status vr_moments(vr_volume_t vol, double *dev_out, void *cuda_stream)
{
    g_err.clear();
    vr_status st = check_volume(vol);
    if (st != VR_OK) return st;
    if (!dev_out || (reinterpret_cast<uintptr_t>(dev_out) & 7u) != 0)
        return invalid("dev_out must be non-NULL and 8-byte aligned");
    st = ensure_stats(vol);
    if (st != VR_OK) return st;
    cudaError_t e = launch_moments(vol_dev(vol), vol->store_dtype, vol->stats, dev_out,
                                   static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail(e, "vr_moments launch");
    return VR_OK;
}

vr_status vr_histogram(vr_volume_t vol, double lo, double hi, int nbins, uint64_t *dev_counts, void *cuda_stream)
{
    g_err.clear();
    vr_status st = check_volume(vol);
    if (st != VR_OK) return st;
    if (!std::isfinite(lo) || !std::isfinite(hi) || !(hi > lo)) return invalid("lo/hi must be finite with hi > lo");
    if (nbins < 1 || nbins > 16384) return invalid("nbins must be in [1, 16384]");
    if (!dev_counts || (reinterpret_cast<uintptr_t>(dev_counts) & 7u) != 0)
        return invalid("dev_counts must be non-NULL and 8-byte aligned");
    cudaError_t e = launch_histogram(vol_dev(vol), vol->store_dtype, lo, hi, nbins,
                                     reinterpret_cast<unsigned long long *>(dev_counts),
                                     static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail(e, "vr_histogram launch");
    return VR_OK;
}

vr_status vr_median(vr_volume_t vol, double *dev_median, void *cuda_stream)
{
    g_err.clear();
    vr_status st = check_volume(vol);
    if (st != VR_OK) return st;
    if (!dev_median || (reinterpret_cast<uintptr_t>(dev_median) & 7u) != 0)
        return invalid("dev_median must be non-NULL and 8-byte aligned");
    st = ensure_stats(vol);
    if (st != VR_OK) return st;
    cudaError_t e = launch_median(vol_dev(vol), vol->store_dtype, vol->stats, dev_median,
                                  static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail(e, "vr_median launch");
    return VR_OK;
}

vr_status vr_selftest_timeout(vr_volume_t vol, void *cuda_stream)
{
    g_err.clear();
    vr_status st = check_volume(vol);
    if (st != VR_OK) return st;
    cudaError_t e = launch_wait_selftest(status_word(vol), static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail(e, "vr_selftest_timeout launch");
    return VR_OK;
}

void vr_debug_fail_alloc(int after)
{
    std::lock_guard<std::mutex> g(g_fail_mu);
    g_fail_after = after < 0 ? -1 : after;
}

vr_status vr_selftest_bounds(vr_volume_t vol, void *cuda_stream)
{
    g_err.clear();
    vr_status st = check_volume(vol);
    if (st != VR_OK) return st;
    cudaError_t e = launch_bounds_selftest(status_word(vol), static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail(e, "vr_selftest_bounds launch");
    return VR_OK;
}

int vr_bounds_checked(void) { return kBoundsChecked ? 1 : 0; }

vr_status vr_check(vr_volume_t vol, void *cuda_stream)
{
    g_err.clear();
    vr_status st = check_volume(vol);
    if (st != VR_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    unsigned flag = 0;
    cudaError_t e = cudaMemcpyAsync(&flag, status_word(vol), sizeof flag, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "vr_check");
    if (flag) {
        cudaMemsetAsync(status_word(vol), 0, sizeof(unsigned), s);
        cudaStreamSynchronize(s);
        if (flag & kStatusTimeout) {
            set_error("a bounded device-side wait gave up in an earlier call on this volume (its results are invalid)");
            return VR_ERR_TIMEOUT;
        }
        set_error("an index outside its buffer was caught in an earlier call on this volume and the access "
                  "skipped (its results are invalid)");
        return VR_ERR_INTERNAL;
    }
    return VR_OK;
}

}  // extern "C"
