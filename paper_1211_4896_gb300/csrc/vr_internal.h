// vr_internal.h -- host/device structures shared by the library's translation
// units (not part of the public ABI; see include/vr.h for that).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>

#include "../../include/vr.h"

namespace vr {

// Camera prepared on the host in double precision and rounded once to float.
// A ray of pixel (i, j) is anchored at the point where it crosses the plane
// through the volume centre perpendicular to the view direction:
//   q(i, j) = q0 + hi * qa + hj * qb        (voxel space; hi = i - (W-1)/2,
//                                            hj = j - (H-1)/2, both exact)
//   unit direction: orthographic wf; perspective normalize(wf + hi*wa + hj*wb)
//   (world space), multiplied by inv_sp for voxel space.
// Positions are q + s d with s in world units; the eye sits at s = -dist |w|.
// Anchoring near the volume keeps every float magnitude ~ the volume size, so
// rounding does not grow with the eye distance.
struct CamDev {
    int W, H, persp;
    float3 q0, qa, qb;     // voxel space
    float3 wf, wa, wb;     // world space (unnormalised direction basis)
    float3 inv_sp;         // 1 / spacing
    float dist;            // signed distance eye -> anchor plane along f
};

// Transfer function and compositing parameters (device view of vr_params).
struct ParamDev {
    const float4 *tf;
    int K;
    float vmin, scale01;   // s = (v - vmin) * scale01, scale01 = 1/(vmax - vmin)
    float km1;             // K - 1
    float su, ou;          // table coordinate u = v * su + ou = (v - vmin) (K-1)/(vmax - vmin)
    float step;
    float t_stop;          // stop once T <= t_stop  (t_stop = 1 - ert_threshold, < 0 disables)
    float4 bg;
};

// Bricked volume view.  Brick (bx, by, bz) holds voxels [bx*B, bx*B + B] per
// axis (B+1 per axis, the +1 apron duplicates the first layer of the next
// brick), x fastest, then y, then z; bricks are stored in x-fastest brick
// order, `stride` elements apart.
struct VolDev {
    const void *data;
    int nx, ny, nz;
    int nbx, nby, nbz;
    int log2b;             // B = 1 << log2b
    long long stride;      // elements per brick (>= (B+1)^3, padded)
    int order;             // element order inside a brick (0: x, 1: y, 2: z fastest)
    int paired;            // 1: each element holds (own value, next value along the fastest axis);
                           // 2: blocked, 2 x 2 x BW blocks of one 32-byte sector deep along axis `order`;
                           // 3: texture layers across axis `order`, `data` holds the cudaTextureObject_t
    long long nelem;       // elements in the buffer (bricks x stride), for the bounds-check build
    unsigned *status;      // the volume's status word (timeouts, caught out-of-range indices)
};

// Dense copy of the volume, x fastest, rows padded to a multiple of 8
// elements so that 16-byte asynchronous copies of any x-aligned run are legal.
struct DenseDev {
    const void *data;
    int nx, ny, nz;
    int px;                // row pitch in elements
};

}  // namespace vr

struct vr_volume {
    int64_t dims[3];
    double origin[3], spacing[3];
    vr_dtype src_dtype, store_dtype;
    int brick, log2b;
    int64_t nb[3];
    long long stride;
    void *bricks = nullptr;
    size_t bytes = 0;
    int device = 0;
    // work-queue counters (a small ring so consecutive calls do not reuse a
    // counter that an earlier, still running launch may read)
    unsigned *counters = nullptr;      // last slot: device status word (timeouts)
    int counter_slots = 0;
    int next_counter = 0;
    // copies of the bricks, built on the first software-filter call that
    // prefers them, indexed by copy id: 1, 2 plain copies with y / z fastest
    // (bytes each); 3, 4, 5 paired 16-bit copies with x / y / z fastest
    // (2 * bytes each); 6, 7, 8 blocked copies deep along x / y / z (sparse
    // views, forward only); [0] unused (the bricks themselves are copy -1).
    // Copy ids 9, 10, 11 are the texture-layer copies below.
    void *copies[9] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    // texture-layer copies of a float volume (copy ids 9, 10, 11: layers
    // across x / y / z), built on the first dense view that prefers them: the
    // layered array, the surface that fills it and the texture that reads it
    struct Layers {
        cudaArray_t array = nullptr;
        cudaSurfaceObject_t surf = 0;
        cudaTextureObject_t tex = 0;
    } layers[3];
    // backward scratch: one FP32 row of K RGBA gradient bins per warp
    float *wtab = nullptr;
    size_t wtab_cap = 0;         // floats
    // backward scratch: the voxel-gradient quads (one float4 per voxel),
    // created on the first backward whose rays are dense enough to use it
    float4 *gquad = nullptr;
    // dense padded copy used by the shared-memory staged kernels
    void *dense = nullptr;
    int dense_px = 0;
    size_t dense_bytes = 0;
    // scratch of the statistics passes (created on first use)
    void *stats = nullptr;
    // per-brick value range (min, max) for empty-space skipping (first use)
    float2 *brick_range = nullptr;
    // hardware-filter copy (created on first texture-filter render)
    cudaArray_t tex_array = nullptr;
    cudaTextureObject_t tex = 0;
    // backward of several views: two streams that overlap one view's last
    // tiles with the next view's first, and the events that fork them from and
    // join them to the caller's stream (created on first use)
    cudaStream_t aux[2] = {nullptr, nullptr};
    cudaEvent_t aux_ev[3] = {nullptr, nullptr, nullptr};
};

namespace vr {

void set_error(const std::string &msg);
vr_status cuda_fail(cudaError_t e, const char *what);
bool is_aligned16(const void *p);
cudaError_t dev_alloc(void **p, size_t bytes);     // every device allocation of the library
bool log_enabled();                                  // VR_LOG set
void log_line(const char *fmt, ...);                 // one "vr: ..." line on stderr when VR_LOG is set

// Host-side preparation (vr_api.cpp).
vr_status prepare_camera(const vr_volume *vol, const vr_camera *cam, CamDev *out);
vr_status prepare_camera_grid(const double origin[3], const double spacing[3], const int64_t dims[3],
                              const vr_camera *cam, CamDev *out);
vr_status prepare_params(const vr_params *p, ParamDev *out);
VolDev vol_dev(const vr_volume *vol);
vr_status next_counter(vr_volume *vol, unsigned **ctr);
int sm_count();

// Launchers (each .cu file).
cudaError_t launch_brick(const void *src, vr_dtype src_dtype, vr_volume *vol, cudaStream_t s);
cudaError_t launch_rebrick(const vr_volume *src, vr_volume *dst, cudaStream_t s);   // same dims and storage
vr_status build_texture(vr_volume *vol, cudaStream_t s);
cudaError_t launch_forward(const VolDev &v, vr_dtype dt, const CamDev &c, const ParamDev &p, float4 *out,
                           uint32_t *nsamples, unsigned *counter, cudaStream_t s);
cudaError_t launch_forward_texture(const vr_volume *vol, const CamDev &c, const ParamDev &p, float4 *out,
                                   uint32_t *nsamples, unsigned *counter, cudaStream_t s);
// Brick copy a software-filter view reads: -1 the bricks themselves, else a
// copy id of vr_volume.copies (element order copy_order, paired if >= 3).
// Bits of a volume's device status word (read and cleared by vr_check).
constexpr unsigned kStatusTimeout = 1u;        // a bounded wait gave up
constexpr unsigned kStatusOutOfBounds = 2u;    // an index outside its buffer was caught and skipped

constexpr int kCopyIds = 12;
inline bool copy_paired(int copy) { return copy >= 3 && copy < 6; }
inline bool copy_blocked(int copy) { return copy >= 6 && copy < 9; }
inline bool copy_layers(int copy) { return copy >= 9 && copy < 12; }
inline int copy_order(int copy) { return copy >= 9 ? copy - 9 : (copy >= 6 ? copy - 6 : (copy >= 3 ? copy - 3 : copy)); }
// Whether copy id `copy` exists on vol.
bool copy_built(const vr_volume *vol, int copy);
// Elements per brick of a blocked copy (B = 1 << log2b; elem_bytes 4 or 2).
long long blocked_stride(int log2b, int elem_bytes);
VolDev vol_dev_copy(const vr_volume *vol, int copy);
// kinds: the copy kinds the caller's kernels read besides plain and paired
// copies (kReadsBlocked: the forward and the batched forward; kReadsLayers:
// those, the backward, maximum intensity projection, sigma clipping, the
// skipping march and the sort-last sub-box renders).
constexpr unsigned kReadsBlocked = 1u, kReadsLayers = 2u;
int preferred_copy(vr_volume *vol, const vr_camera *cam, bool may_build, cudaStream_t s, unsigned kinds = 0u);
size_t copy_bytes(const vr_volume *vol, int copy);
cudaError_t launch_copy(vr_volume *vol, int copy, cudaStream_t s);
// Texture-layer copy across `axis` (float storage): allocates the layered
// array (through the library's allocation hook), its surface and texture,
// and fills it from the bricks; frees what it made on failure.
cudaError_t build_layers(vr_volume *vol, int axis, cudaStream_t s);
void free_layers(vr_volume *vol);
cudaError_t dev_alloc_layers(cudaArray_t *a, int u, int v, int layers);   // hook of dev_alloc for arrays
// One view of a backward call: the layout it reads (a brick copy or the
// bricks), its camera, the forward's image and sample counts, dL/d(image),
// and the axis along which its direct voxel-gradient sums are carried.
struct BwdView {
    VolDev v;
    CamDev c;
    const float4 *rgba, *grad_rgba;
    const uint32_t *nsamples;
    int carry_axis;
};
cudaError_t launch_backward(vr_volume *vol, const BwdView *views, int n, const ParamDev &p, double *grad_tf,
                            float *grad_vox, float4 *grad_quad, int quad_axis, long long nvox, bool accumulate,
                            unsigned *counter, cudaStream_t s);
cudaError_t ensure_wtab(vr_volume *vol, size_t floats, cudaStream_t s);
int backward_max_tf_size();
DenseDev dense_dev(const vr_volume *vol);
cudaError_t launch_densify(const void *src, vr_dtype src_dtype, vr_volume *vol, cudaStream_t s);
cudaError_t launch_dense_from_bricks(vr_volume *vol, cudaStream_t s);
cudaError_t launch_forward_staged(const DenseDev &d, vr_dtype dt, const CamDev &c, const ParamDev &p, float4 *out,
                                  uint32_t *nsamples, unsigned *counter, unsigned *status, cudaStream_t s);
cudaError_t launch_backward_staged(const DenseDev &d, vr_dtype dt, const CamDev &c, const ParamDev &p,
                                   const float4 *rgba, const uint32_t *nsamples, const float4 *grad_rgba,
                                   double *grad_tf, float *grad_vox, long long nvox, bool accumulate,
                                   unsigned *counter, unsigned *status, cudaStream_t s);
int occupancy_blocks(const void *fn, int threads, size_t smem);
cudaError_t launch_wait_selftest(unsigned *status, cudaStream_t s);
cudaError_t launch_bounds_selftest(unsigned *status, cudaStream_t s);
// Other uses of the march (vr_modes.cu).
cudaError_t launch_mip(const VolDev &v, vr_dtype dt, const CamDev &c, const ParamDev &p, float4 *out,
                       uint32_t *nsamples, unsigned *counter, cudaStream_t s);
cudaError_t launch_sigma(const VolDev &v, vr_dtype dt, const CamDev &c, const ParamDev &p, const float *minimap,
                         const int region[3], float4 *out, uint32_t *nsamples, unsigned *counter, cudaStream_t s);
cudaError_t launch_minimap(const VolDev &v, vr_dtype dt, const int region[3], float *dev_out, cudaStream_t s);
cudaError_t launch_profile(const VolDev &v, vr_dtype dt, const CamDev &c, float step, int i, int j, float *values,
                           unsigned max_values, unsigned *count, cudaStream_t s);
// Sort-last sub-box render and depth-ordered composite (vr_modes.cu).
constexpr int kMaxPartials = 64;
cudaError_t launch_subbox(const VolDev &v, vr_dtype dt, const CamDev &c, const ParamDev &p, const int lo[3],
                          const int hi[3], const int gdim[3], const int off[3], float4 *partial, float *depth,
                          uint32_t *count, unsigned *counter, cudaStream_t s);
cudaError_t launch_composite(int k, const float *const *partials, const float *const *depths, long long npx,
                             const float bg[4], float *out, cudaStream_t s);
// Empty-space skipping (vr_skip.cu).
cudaError_t launch_brick_range(const VolDev &v, vr_dtype dt, float2 *range, cudaStream_t s);
cudaError_t launch_forward_skip(const VolDev &v, vr_dtype dt, const CamDev &c, const ParamDev &p,
                                const float2 *range, uint32_t *mask, float4 *out, uint32_t *nsamples,
                                unsigned *counter, cudaStream_t s);
// Global statistics (vr_stats.cu).
size_t stats_scratch_bytes();
cudaError_t launch_moments(const VolDev &v, vr_dtype dt, void *scratch, double *out, cudaStream_t s);
cudaError_t launch_histogram(const VolDev &v, vr_dtype dt, double lo, double hi, int nbins,
                             unsigned long long *counts, cudaStream_t s);
cudaError_t launch_median(const VolDev &v, vr_dtype dt, void *scratch, double *median, cudaStream_t s);
vr_status validate_job(const vr_job *job, int index);
void purge_plans(const vr_volume *vol);

}  // namespace vr
