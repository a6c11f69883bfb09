/*
 * vr.h -- C ABI of the GB300 direct-volume-rendering library (libvr.so).
 *
 * Direct volume rendering of a 3D float image (a radio spectral cube, axes
 * RA x Dec x frequency) by ray casting: each pixel's ray is clipped to the
 * volume box, sampled at a constant step with trilinear interpolation, every
 * sample is mapped through a 1D RGBA transfer function, and the samples are
 * composited front to back with optional early ray termination.
 *
 * Method: Hassan, Fluke, Barnes & Kilborn (2012), "Tera-scale astronomical
 * data analysis and visualization": Section 3.3 (transfer functions: the
 * data range is partitioned into levels, each with a colour and an opacity in
 * [0,1]), Section 3.4 (front-to-back composition of colour and opacity), and
 * Section 4.4 (constant-step samples with trilinear interpolation).  Early ray
 * termination, the adjoint pass and the batched launch are extensions that
 * the paper does not describe.
 *
 * Conventions shared by every entry point
 *   - Pointers named dev_* are CUDA device pointers owned by the caller.  The
 *     library owns only what it allocates inside a vr_volume_t.
 *   - Every call that takes `cuda_stream` (a cudaStream_t, NULL = legacy
 *     default stream) enqueues work on that stream and returns.  It
 *     synchronises only in vr_volume_create / vr_volume_destroy, vr_check,
 *     and on the first use of something a volume builds or grows lazily (a
 *     brick copy, the per-brick value ranges of empty-space skipping, a
 *     larger backward scratch, a batch plan), as the entry points say; device
 *     allocations happen only then too.
 *   - Arguments are validated on the host before anything is enqueued; an
 *     invalid call returns a negative vr_status, enqueues nothing, and sets a
 *     thread-local message readable with vr_last_error().
 *   - A volume handle must not be used by two calls that run concurrently on
 *     different streams (its work counters and scratch are per handle), and
 *     must not be destroyed while work that uses it is in flight.
 *   - Geometry: voxel (x, y, z) is at world position origin + (x, y, z) *
 *     spacing; the box is the closed [0, n-1] per axis (voxel centres at
 *     integer indices).  Dense cubes are x-fastest (x = RA, then y = Dec,
 *     then z = frequency, the FITS axis order).
 *   - Images are row-major float32 RGBA, H rows of W pixels, row 0 at the
 *     top (+up), straight (not premultiplied) colour.
 */
#ifndef VR_H
#define VR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VR_OK = 0,
    VR_ERR_INVALID_ARG = -1,   /* bad pointer, size, dtype or parameter */
    VR_ERR_UNSUPPORTED = -2,   /* valid but not implemented for this combination */
    VR_ERR_OOM = -3,           /* a device allocation failed */
    VR_ERR_CUDA = -4,          /* a CUDA runtime call failed (message has the CUDA error) */
    VR_ERR_TIMEOUT = -5,       /* a bounded device-side wait gave up */
    VR_ERR_INTERNAL = -6
} vr_status;

typedef enum { VR_F32 = 0, VR_F16 = 1, VR_BF16 = 2 } vr_dtype;

enum { VR_CAMERA_ORTHO = 0, VR_CAMERA_PERSPECTIVE = 1 };
enum { VR_FILTER_SOFTWARE = 0, VR_FILTER_TEXTURE = 1, VR_FILTER_SOFTWARE_STAGED = 2 };

/* What the ray computes (vr_params.mode). */
enum {
    VR_MODE_COMPOSITE = 0,    /* generic transfer function, front-to-back composite (Sections 3.3.2, 3.4) */
    VR_MODE_MIP = 1,          /* maximum intensity projection (Section 3.3.1) */
    VR_MODE_SIGMA = 2         /* sigma-clipping transfer function (Section 4.5) */
};

typedef struct vr_volume *vr_volume_t;   /* opaque, library-owned */

/* Camera.  Basis: f = normalize(forward), r = normalize(f x up), u = r x f.
 * Pixel (i, j) has screen coordinates sx = 2 (i + 1/2)/W - 1 and
 * sy = 1 - 2 (j + 1/2)/H, aspect = W/H.
 *   orthographic: origin eye + sx (ortho_height/2) aspect r + sy (ortho_height/2) u,
 *                 direction f, no near clip;
 *   perspective:  origin eye, direction normalize(f + sx tan(fov/2) aspect r
 *                 + sy tan(fov/2) u), samples only at t >= 0.
 * The user controls the viewport this way (Section 3.1 of the paper). */
typedef struct {
    int kind;                 /* VR_CAMERA_ORTHO or VR_CAMERA_PERSPECTIVE */
    double eye[3];            /* world coordinates */
    double forward[3];        /* need not be unit length; must not be parallel to up */
    double up[3];
    double fov_y_deg;         /* perspective: full vertical field of view, (0, 180) */
    double ortho_height;      /* orthographic: world height of the image, > 0 */
    int width, height;        /* image size in pixels, each in [1, 32768] */
} vr_camera;

/* Rendering parameters (Section 3.3: the transfer function maps each data
 * level to a colour and an opacity in [0, 1]).  Sample value v maps to
 * u = clamp((v - vmin)/(vmax - vmin), 0, 1) (K - 1); entries floor(u) and
 * floor(u)+1 are blended linearly (the last interval is closed).  Samples are
 * at t_in + (k + 1/2) step for k = 0, 1, ... while <= t_out; compositing is
 * C += T a rgb, T *= 1 - a, stopping after the sample at which 1 - T >=
 * ert_threshold (a value > 1 disables early termination).  The pixel is
 * (C + T bg.rgb, 1 - T + T bg.a). */
typedef struct {
    const float *tf_rgba;     /* device, K x 4 float32 RGBA, 16-byte aligned */
    int tf_size;              /* K, in [2, 4096] */
    float vmin, vmax;         /* value range mapped onto the table, vmax > vmin */
    float step;               /* world units along the unit ray, > 0 */
    float ert_threshold;      /* early-termination opacity in (0, 1]; > 1 disables */
    float bg_rgba[4];         /* background, straight RGBA */
    int filter;               /* VR_FILTER_SOFTWARE: FP32 trilinear gathered from the bricks through
                                   L1 (the default, fastest measured path);
                                 VR_FILTER_SOFTWARE_STAGED: FP32 trilinear with the volume staged
                                   slab by slab in shared memory by bulk copies (bit-identical
                                   results; allocates a dense copy on first use);
                                 VR_FILTER_TEXTURE: hardware filter, 8-bit fractional weights,
                                   float32/float16 storage only, forward only */
    int mode;                 /* VR_MODE_*; 0 for the composite.  VR_MODE_MIP: the pixel is the table
                                   entry of the ray's largest sample value composited once over the
                                   background, (a rgb + (1 - a) bg.rgb, a + (1 - a) bg.a); a miss shows
                                   the background; no early termination; nsamples = all samples.
                                 VR_MODE_SIGMA: the composite, with every sample value v replaced
                                   by (v - mean) / sd of the mini-map (vr_minimap) trilinearly
                                   interpolated at the sample; [vmin, vmax] are then in units of sd.
                                 Both: software filter (VR_FILTER_SOFTWARE) and vr_render only. */
    const float *minimap;     /* VR_MODE_SIGMA: device mini-map of vr_minimap for this volume and
                                   minimap_region, 8-byte aligned; otherwise ignored */
    int minimap_region[3];    /* VR_MODE_SIGMA: region size in voxels per axis, each >= 1 */
    int skip_empty;           /* 1: skip the samples of bricks whose whole value range maps to
                                   table entries of zero opacity (exact: such samples add nothing
                                   and do not change T; images and sample counts are bit-identical
                                   to skip_empty = 0).  Composite mode, VR_FILTER_SOFTWARE, vr_render
                                   only; the first such call builds a per-brick value range
                                   (8 bytes per brick, plus one transparency bit per brick that
                                   each call recomputes for its table) and synchronises
                                   cuda_stream. */
} vr_params;

typedef struct {
    int64_t dims[3];
    vr_dtype store_dtype;
    int brick;                /* B: bricks of B^3 cells stored with a +1 apron, (B+1)^3 voxels */
    int64_t bricks[3];        /* bricks per axis */
    int64_t bytes;            /* device bytes held by the bricked copy */
    int64_t dense_bytes;      /* device bytes of the dense row-padded copy (0 until the first
                                 staged call) */
    int64_t copy_bytes;       /* device bytes of the brick copies (see vr_volume_create) */
    int copies;               /* which copies exist: bit 1 / 2 plain y- / z-fastest; bit 3 / 4 / 5
                                 paired x- / y- / z-fastest (16-bit storage); bit 6 / 7 / 8
                                 blocked, deep along x / y / z (sparse views); bit 9 / 10 / 11
                                 texture layers across x / y / z (float storage, dense views) */
    int64_t scratch_bytes;    /* device bytes of the backward scratch: the per-warp table-gradient
                                 rows and, once a dense view has used it, the voxel-gradient quad
                                 scratch (16 bytes per voxel) */
} vr_volume_info_t;

/* ------------------------------------------------------------------------
 * Volume residency (Section 2: the whole data set is loaded into GPU memory
 * once and stays there; the paper keeps it in texture memory, this library in
 * a bricked HBM layout).
 *
 * Copies the dense cube dev_cube (src_dtype, dims = {nx, ny, nz}, each >= 2,
 * x fastest) into a bricked copy in store_dtype: bricks of B^3 cells, each
 * stored as (B+1)^3 voxels so that all 8 trilinear corners of any cell lie in
 * one brick, x fastest inside a brick.  F32 -> F16/BF16 rounds to nearest
 * even.  brick = 0 picks 16, or 64 for a volume whose 16^3 bricks would take
 * more than 16 GiB; otherwise 16, 32 or 64.  origin/spacing may be NULL (0
 * and 1).
 *
 * Copies made later, on first use: the first VR_FILTER_SOFTWARE_STAGED call
 * adds a dense copy with rows padded to 8 elements, streamed slab by slab
 * into shared memory.  The first software-filter call (render, backward or
 * batched) with a view whose image rows run closest to an axis adds a copy of
 * the bricks with that axis fastest inside each brick, so that the rays of
 * one warp read neighbouring elements: a plain copy for the y or z axis (the
 * bricks serve the x axis), as many bytes as the bricks.  For 16-bit storage
 * and rays closer than VR_PAIRED_MAX_PITCH voxels (environment, default 3)
 * at the volume centre, a paired copy for any axis instead, each element
 * holding its own value and the next one along that axis so that four loads
 * fetch a cell's eight corners (twice the bricks' bytes).  For rays at least
 * VR_SPARSE_MIN_PITCH voxels apart (default 3), which share no sectors, the
 * forward (vr_render, vr_render_batched) of a 16-bit volume in bricks smaller
 * than 64^3 reads a blocked copy instead (in 64^3 bricks the plain copies
 * measured faster and serve): blocks of 2 x 2 x 4 voxels, one 32-byte sector each, deep
 * along the axis the view direction is closest to (about 1.2x the bricks'
 * bytes); VR_SPARSE_LAYOUT=b asks for blocked copies (2 x 2 x 2 blocks) for
 * float volumes too, =i never.  For float storage and rays closer than
 * VR_SPARSE_MIN_PITCH, the forward, batched and backward calls read a
 * texture-layer copy instead (the paper's texture memory, Section 4.3): a 2D
 * layered texture (layers across the axis the view direction runs along
 * most, 4 bytes per voxel), whose four-texel gather at a cell's exact
 * integer corner fetches the cell's corners two per instruction (the values
 * stored, interpolated in software: bit-identical results); a volume beyond
 * the device's layered-texture limits (usually 32768 texels across a layer,
 * 2048 layers) keeps the brick copies; VR_TEX_LAYERS=0 (read at each call)
 * turns the layers off.  A copy is built
 * only outside stream capture, while the device keeps an eighth of its memory
 * free besides it (else the bricks themselves serve), synchronising
 * cuda_stream once; environment variable VR_BRICK_COPIES=0 turns copies off.
 * Results do not depend on which copy a view reads.  vr_volume_update
 * refreshes every copy; vr_volume_info reports them.  The
 * caller keeps dev_cube; the call synchronises `cuda_stream` before returning
 * the handle in *out.  Errors: INVALID_ARG, OOM, CUDA.
 * ---------------------------------------------------------------------- */
vr_status vr_volume_create(const void *dev_cube, vr_dtype src_dtype, vr_dtype store_dtype,
                           const int64_t dims[3], const double origin[3], const double spacing[3],
                           int brick, void *cuda_stream, vr_volume_t *out);

/* Re-bricks new voxel values (same dims and src_dtype as at creation) into an
 * existing handle, asynchronously on cuda_stream (e.g. after a gradient step
 * on the voxels). */
vr_status vr_volume_update(vr_volume_t vol, const void *dev_cube, vr_dtype src_dtype, void *cuda_stream);

/* A new handle holding the same voxels as `src` in bricks of another size
 * (16, 32 or 64; 0 = 16), built on the device from src's bricks (no dense
 * copy needed), for the batched autotuner's choice of brick size (not in the
 * paper).  Copies of src are not carried over; the new handle builds its own
 * on first use.  Synchronises cuda_stream.  Errors: INVALID_ARG, OOM, CUDA. */
vr_status vr_volume_rebrick(vr_volume_t src, int brick, void *cuda_stream, vr_volume_t *out);

/* Frees the handle and its device memory (synchronises the device). NULL is a no-op. */
vr_status vr_volume_destroy(vr_volume_t vol);

vr_status vr_volume_info(vr_volume_t vol, vr_volume_info_t *out);

/* The brick layout a software-filter render of this view reads as things
 * stand: *layout = -1 for the x-fastest bricks, else the copy id (1, 2: plain
 * copies with y / z fastest; 3, 4, 5: paired 16-bit copies with x / y / z
 * fastest; 6, 7, 8: blocked copies deep along x / y / z; 9, 10, 11:
 * texture layers across x / y / z; bit `id` of vr_volume_info's copies).  Builds nothing: a preferred
 * copy that does not exist yet reports -1 until a render builds it.  A batched
 * call launches one kernel per distinct layout of its views.  Errors:
 * INVALID_ARG. */
vr_status vr_view_layout(vr_volume_t vol, const vr_camera *cam, int *layout);

/* ------------------------------------------------------------------------
 * Forward render (Sections 3.3-3.4 and 4.4).
 *
 * Writes W*H float32 RGBA pixels to dev_rgba_out (16-byte aligned) and, when
 * dev_nsamples_out is not NULL, the number of samples composited per pixel
 * (after early termination; 0 when the ray misses the box).  The backward
 * pass needs both.  Errors: INVALID_ARG, UNSUPPORTED (texture filter on
 * bfloat16 storage), OOM (first texture-filter or staged call), CUDA.
 * ---------------------------------------------------------------------- */
vr_status vr_render(vr_volume_t vol, const vr_camera *cam, const vr_params *params, float *dev_rgba_out,
                    uint32_t *dev_nsamples_out, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Adjoint of vr_render (not in the paper): gradients of a scalar loss L with
 * respect to the transfer-function table and the voxel values, given
 * dev_grad_rgba = dL/d(image) (W*H*4 float32).
 *
 * Each ray is re-marched front to back from the forward's stored image and
 * sample count (recomputing per-sample state instead of storing it): the
 * transmittance behind sample k is recovered from the final colour and
 * transmittance, T_final = (1 - alpha_out)/(1 - bg.a), so bg.a must be < 1.
 * Early-termination decisions of the forward are kept (dev_nsamples).
 *   dev_grad_tf  (K*4 float64): each warp accumulates its rays' terms in a
 *                private FP32 row of K RGBA bins (16-byte vector reductions,
 *                L2-resident); one final kernel sums the rows in FP64 (the
 *                only FP64 step; the order of its atomics is not
 *                deterministic).
 *   dev_grad_vox (nx*ny*nz float32 dense, x fastest) or NULL: float
 *                reductions (summation order is not deterministic).  A
 *                ray's sums for its cell's eight corners are kept as two
 *                planes of four across the view's dominant axis and the
 *                shared plane is carried when the ray steps along it, so a
 *                straight run writes one plane per cell: into dev_grad_vox
 *                directly (x-neighbour pairs as 8-byte reductions where
 *                aligned) or, where the view puts at least one sample per
 *                voxel (ray pitch and step at the volume centre), as one
 *                16-byte reduction per plane into a library-owned scratch of
 *                one float4 per voxel, which a gather pass then adds into
 *                dev_grad_vox.  The scratch (16 bytes per voxel) is allocated
 *                on first use when the stream is not being captured and an
 *                eighth of the device memory stays free besides it;
 *                otherwise the direct form runs.  VR_GRAD_DIRECT forces the
 *                direct form, VR_GRAD_SCRATCH the scratch form (memory
 *                permitting); the staged filter's backward always scatters
 *                directly.
 * Both are overwritten, or added to when flags has VR_GRAD_ACCUMULATE (a
 * loss summed over several views: call once per view).
 * Only software filtering is differentiable.  Errors: INVALID_ARG (also
 * VR_GRAD_DIRECT with VR_GRAD_SCRATCH), UNSUPPORTED (texture filter,
 * bg.a >= 1, tf_size > 1600), CUDA.
 * ---------------------------------------------------------------------- */
enum { VR_GRAD_ACCUMULATE = 1, VR_GRAD_DIRECT = 2, VR_GRAD_SCRATCH = 4 };

vr_status vr_render_backward(vr_volume_t vol, const vr_camera *cam, const vr_params *params,
                             const float *dev_rgba, const uint32_t *dev_nsamples,
                             const float *dev_grad_rgba, double *dev_grad_tf, float *dev_grad_vox,
                             unsigned flags, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Adjoint over several views at once: the gradients of L = sum over the n
 * views of their losses (a table or volume fitted to several target
 * renderings), equal to n vr_render_backward calls with VR_GRAD_ACCUMULATE
 * after the first.  One call clears the outputs (unless VR_GRAD_ACCUMULATE),
 * launches one backward kernel per view into the same per-warp table rows
 * and voxel gradient, alternating between two streams of the volume's own
 * (forked from and joined back to cuda_stream, created on first use) so that
 * a view's kernel starts on the CTA slots the previous view's last tiles
 * leave free; then it runs the FP64 row sum and, with the quad scratch, its
 * gather once for all views; the scratch is chosen where the views
 * put at least one sample per voxel on average, with one quad orientation
 * (the carry axis most views share).  views is a host array of n (1..4096) entries; each view's
 * image, sample counts and dL/d(image) follow the rules of
 * vr_render_backward.  Errors as vr_render_backward.
 * ---------------------------------------------------------------------- */
typedef struct {
    vr_camera cam;
    const float *rgba;            /* this view's forward image (W*H*4 float32, 16-byte aligned) */
    const uint32_t *nsamples;     /* its sample counts (W*H, 4-byte aligned) */
    const float *grad_rgba;       /* dL/d(image) for this view (W*H*4 float32, 16-byte aligned) */
} vr_grad_view;

vr_status vr_render_backward_views(vr_volume_t vol, const vr_grad_view *views, int n, const vr_params *params,
                                   double *dev_grad_tf, float *dev_grad_vox, unsigned flags, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Batched render (not in the paper; its "many smaller cubes" future-work
 * item motivates it): n jobs, each with its own volume, camera, parameters
 * and output, rendered by one persistent kernel launch per brick layout the
 * views read (vr_view_layout: at most three for float storage, six for
 * 16-bit), whose CTAs pull the ray tiles of all its jobs from a shared work
 * queue; with use_graph the launches are replayed as one CUDA graph.
 * Results equal n vr_render calls.
 * Software filter only.
 * ---------------------------------------------------------------------- */
typedef struct {
    vr_volume_t vol;
    vr_camera cam;
    vr_params params;
    float *dev_rgba_out;
    uint32_t *dev_nsamples_out;   /* may be NULL */
} vr_job;

typedef struct {
    int use_graph;            /* 1: build a CUDA graph of the call on first use (counter reset, then
                                 one kernel node per brick layout, the layouts running concurrently)
                                 and replay it while the job list is unchanged (same pointers and
                                 parameters); 0: launch the layouts one after another */
    int tile_w, tile_h;       /* ray tile of one warp: tile_w * tile_h == 32; 0 = 8 x 4 */
    int ctas_per_sm;          /* persistent CTAs per SM; 0 = occupancy limit */
    int warps_per_tile;       /* 1, 2 or 4 warps of a CTA take one tile of tile_w x (tile_h x
                                 warps_per_tile) rays together, one part each, so that neighbouring
                                 parts share an SM's L1; 0 = 1 */
} vr_batch_opts;

/* All volumes of one batch must share store dtype and brick size
 * (UNSUPPORTED otherwise).  A job list is cached under its stream, options and
 * the named fields of its jobs (never the structs' padding): the first call
 * with a new list on a stream uploads its descriptors (synchronising
 * cuda_stream); with use_graph the first call also builds the graph.  A list
 * owns one work counter, so the same list on two streams gets two plans.
 * Past 64 cached lists the cache is emptied after a device synchronisation.  Within a layout the jobs
 * with the most work (pixels x samples along the box diagonal) are handed out
 * first.  Later calls with the same list only launch.  Errors: INVALID_ARG,
 * UNSUPPORTED, OOM, CUDA. */
vr_status vr_render_batched(const vr_job *jobs, int n, const vr_batch_opts *opts, void *cuda_stream);

/* Times candidate tile shapes, CTA counts and warps per tile for this job
 * list (it renders the jobs several times on cuda_stream and synchronises
 * it) and writes the fastest into *best.  best->use_graph is left
 * unchanged.  The brick size is the volumes' (see vr_volume_rebrick). */
vr_status vr_autotune_batched(const vr_job *jobs, int n, vr_batch_opts *best, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Batched render that allocates nothing (the paper has no counterpart).
 *
 * For callers that cannot call cudaMalloc while rendering: services that
 * run inside a fixed device-memory budget, processes whose device memory is
 * handed out by another allocator's pool (an allocation outside the pool
 * would break its accounting), and frame loops that cannot take the
 * device-wide synchronisation a cudaMalloc or cudaFree may cause.
 * vr_render_batched allocates a descriptor table
 * and a work counter for every new job list; this variant keeps both in one
 * static device array sized for VR_NOALLOC_MAX_JOBS jobs (about 64 KB, held by
 * every GPU that loads the library until the process exits), uploads the
 * descriptors with cudaMemcpyAsync and zeroes the work counters with
 * cudaMemsetAsync on cuda_stream.  The caller still passes the volumes and the
 * outputs.  Jobs are rendered exactly as by vr_render_batched (same kernels);
 * tile_w x tile_h is the warp's ray tile (0, 0 = 8 x 4).  It never builds a
 * brick copy (see vr_volume_create): a view reads such a copy only when an
 * earlier call built it.
 *   - n > VR_NOALLOC_MAX_JOBS returns VR_ERR_INVALID_ARG and launches nothing.
 *   - The first call on a device looks up the device address of the static
 *     array (cudaGetSymbolAddress) and the kernels' occupancy (both cached
 *     afterwards); make that first call before any stream capture.
 *   - Every call reuses the same array: calls that overlap on the GPU (two
 *     streams, or two host threads) race and must be serialised by the caller.
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA.
 * ---------------------------------------------------------------------- */
#define VR_NOALLOC_MAX_JOBS 256

vr_status vr_render_batched_noalloc(const vr_job *jobs, int n, int tile_w, int tile_h, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Statistical mini-map for the sigma-clipping transfer function (Section 4.5:
 * a scaled-down copy of the cube whose points summarise regions of it).
 *
 * The cube is split into regions of region[a] voxels per axis (the last
 * region of an axis keeps the remainder), m[a] = ceil(dims[a] / region[a])
 * regions per axis.  Writes m0 * m1 * m2 float pairs to dev_minimap (x
 * fastest; 8-byte aligned, caller-owned): the mean and the population
 * standard deviation of the region's stored voxel values, summed in FP64
 * (two passes) and rounded to float32.  Point (i, j, k) sits at voxel
 * ((i + 1/2) region - 1/2, ...) for the interpolation of VR_MODE_SIGMA.
 * Asynchronous on cuda_stream.  Errors: INVALID_ARG, CUDA.
 * ---------------------------------------------------------------------- */
vr_status vr_minimap(vr_volume_t vol, const int region[3], float *dev_minimap, void *cuda_stream);

/* ------------------------------------------------------------------------
 * 3D spectrum tool (Section 4.4: the data profile along the line of sight
 * of a picked screen position).
 *
 * Writes the trilinear values of the samples of pixel (i, j)'s clipped ray
 * (the renderer's sample positions t_in + (k + 1/2) step) to dev_values[k]
 * for k < min(n, max_values) and n to *dev_count (0 when the ray misses the
 * box).  dev_values holds max_values floats; both are caller-owned device
 * memory.  Asynchronous on cuda_stream.  Errors: INVALID_ARG, CUDA.
 * ---------------------------------------------------------------------- */
vr_status vr_profile(vr_volume_t vol, const vr_camera *cam, float step, int i, int j, float *dev_values,
                     uint32_t max_values, uint32_t *dev_count, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Sort-last rendering (Sections 3.2 and 3.4: each GPU renders its sub-cube,
 * the sub-images are merged in visibility order with the over operator).
 *
 * vr_render_subbox renders only the samples whose cell (the cell origin of
 * the trilinear interpolation, clamp(floor(p), 0, n-2) per axis) lies in
 * [cell_lo, cell_hi) -- cells, 0 <= cell_lo < cell_hi <= dims - 1 per axis --
 * at the sample positions of the whole volume's ray, so that the sub-images
 * of a partition of the cells composite to the whole render.  Per pixel it
 * writes the partial composite to dev_partial (float4: premultiplied colour
 * C.rgb and the transmittance T of these samples; (0, 0, 0, 1) when there are
 * none), the distance of the first such sample from the eye (perspective) or
 * the image plane (orthographic) to dev_depth (+inf when none) and, if
 * dev_count is not NULL, their number.  No early termination,
 * no background; composite mode, software filter.  Reads the brick copy the
 * view prefers, like vr_render.
 *
 * vr_composite merges k (1 .. 64) such partial images of one view (host array
 * of device pointers; width x height pixels each): per pixel in order of
 * depth, front first, C = C1 + T1 C2 + T1 T2 C3 + ..., T = T1 T2 ...; writes
 * (C + T bg.rgb, 1 - T + T bg.a) to dev_rgba_out.  All buffers caller-owned,
 * float4 arrays 16-byte aligned.  Errors: INVALID_ARG, UNSUPPORTED, CUDA.
 * ---------------------------------------------------------------------- */
vr_status vr_render_subbox(vr_volume_t vol, const vr_camera *cam, const vr_params *params, const int cell_lo[3],
                           const int cell_hi[3], float *dev_partial, float *dev_depth, uint32_t *dev_count,
                           void *cuda_stream);

/* vr_render_subbox_of: the same for a volume that holds only the voxels
 * [offset, offset + dims) of a larger grid of global_dims voxels -- one
 * GPU's sub-cube in the paper's object-space split, with the one-voxel
 * overlap its far cells need.  The volume's origin is that of its own first
 * voxel, so the whole grid's first voxel lies offset * spacing before it.
 * Rays are clipped to the whole grid's box and sampled at the whole render's
 * positions (the camera is set up in the whole grid's coordinates, so every
 * sub-cube computes bit-identical sample positions and each sample falls in
 * exactly one sub-box); cell_lo / cell_hi are cell indices of the whole grid
 * with offset <= cell_lo < cell_hi <= offset + dims - 1 per axis.  With
 * offset 0 and global_dims = dims it is vr_render_subbox.  Errors as
 * vr_render_subbox. */
vr_status vr_render_subbox_of(vr_volume_t vol, const int64_t global_dims[3], const int64_t offset[3],
                              const vr_camera *cam, const vr_params *params, const int cell_lo[3],
                              const int cell_hi[3], float *dev_partial, float *dev_depth, uint32_t *dev_count,
                              void *cuda_stream);
vr_status vr_composite(int k, const float *const *dev_partials, const float *const *dev_depths, int width,
                       int height, const float bg_rgba[4], float *dev_rgba_out, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Global statistics of the resident cube (Sections 4.1-4.3 of the paper).
 * Each is one or a few streaming passes over the bricks, asynchronous on
 * cuda_stream; every voxel counts once; NULL (NaN) voxels are left out.
 * Outputs are caller-owned device memory, 8-byte aligned.
 *
 * vr_moments writes 5 doubles: the count of non-NaN voxels, their mean,
 * population standard deviation, minimum and maximum (NaN without values).
 * Sums as in Section 4.2: runs of 16 values in FP32, the runs in FP64, about
 * a shift (the first voxel).
 *
 * vr_histogram writes nbins (1 .. 16384) uint64 counts of the values in
 * [lo, hi] (finite, hi > lo) in equal bins, the value hi in the last bin;
 * values outside are not counted (Section 4.1).
 *
 * vr_median writes 1 double: the value of rank (n + 1) / 2 (integer division,
 * 1-based) among the n non-NaN voxels -- the median for odd n, the lower
 * median for even n, the rank the paper's Torben method returns (Section
 * 4.3) -- by a three-pass radix select (NaN without values).
 * Errors: INVALID_ARG, OOM (first moments/median call), CUDA.
 * ---------------------------------------------------------------------- */
vr_status vr_moments(vr_volume_t vol, double *dev_out, void *cuda_stream);
vr_status vr_histogram(vr_volume_t vol, double lo, double hi, int nbins, uint64_t *dev_counts, void *cuda_stream);
vr_status vr_median(vr_volume_t vol, double *dev_median, void *cuda_stream);

/* Synchronises cuda_stream and reports whether a bounded device-side wait of an
 * earlier call on this volume gave up (the staged kernels wait on the copy
 * engine with an iteration limit; a timeout leaves that call's results
 * invalid): VR_ERR_TIMEOUT; or whether the bounds-check build caught an index
 * outside its buffer (and skipped that access): VR_ERR_INTERNAL.  Returns
 * VR_OK otherwise; each report is given once (the flags are cleared).  The
 * paper has no such mechanism; it is part of this library's failure
 * detection. */
vr_status vr_check(vr_volume_t vol, void *cuda_stream);

/* 1 when this library is the bounds-check build (compiled with
 * -DVR_BOUNDS_CHECK: every voxel gather, gradient scatter, table-bin,
 * per-brick and mini-map index is tested against its buffer in the kernels
 * before the access, a stand-in for a memory checker), else 0. */
int vr_bounds_checked(void);

/* Failure injection for tests (no counterpart in the paper): the library's
 * device allocation that follows `after` successful ones fails once, as if
 * the device were out of memory; a negative value cancels.  Every entry point
 * then reports VR_ERR_OOM or falls back as documented (a brick copy or the
 * backward's quad scratch that cannot be allocated is simply not used), and
 * leaves its handle usable.  Process-wide. */
void vr_debug_fail_alloc(int after);

/* Self-test of the bounds-check report (no counterpart in the paper): a
 * one-thread kernel tests an index one past the end of a range -- nothing is
 * read or written -- so the next vr_check returns VR_ERR_INTERNAL once.
 * Works in either build.  Errors: INVALID_ARG, CUDA. */
vr_status vr_selftest_bounds(vr_volume_t vol, void *cuda_stream);

/* Failure-detection self-test (no counterpart in the paper): enqueues on
 * cuda_stream one wait, with the staged kernels' bounded mbarrier wait, on a
 * barrier that nothing completes.  The wait gives up after 256 polls and
 * records the timeout in the volume's status word, so the next vr_check
 * returns VR_ERR_TIMEOUT (and clears it).  Nothing faults or hangs; the
 * device stays usable.  Errors: INVALID_ARG, CUDA. */
vr_status vr_selftest_timeout(vr_volume_t vol, void *cuda_stream);

/* Human-readable message of the last failed call on this thread ("" if none). */
const char *vr_last_error(void);

/* Library version string. */
const char *vr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* VR_H */
