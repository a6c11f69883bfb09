// vr_skip.cu -- exact empty-space skipping for the composite forward render.
//
// Each brick's value range [min, max] over its (B+1)^3 voxels bounds every
// sample interpolated inside its cells (trilinear interpolation is a convex
// combination of the corners).  When every table entry that range can reach
// has zero opacity, the brick's samples add nothing to the colour and leave
// the transmittance unchanged (C += T * 0 * c, T *= 1 - 0), so the march jumps
// over them: the image and the sample counts are bit-identical to the plain
// march.  The emptiness test is per brick and per table: a prefix count of
// the table's non-zero opacities, and the brick's range mapped to entries with
// one entry of margin on each side (the rounding of an interpolated value near
// the range's ends); a first kernel turns it into one bit per brick, which
// the march reads from shared memory.  A brick holding a NaN voxel is never
// skipped.
#include "vr_device.cuh"

#include <cmath>

namespace vr {

constexpr int kSkipThreads = 256;

// ---------------------------------------------------------------------------
// Per-brick value range: one CTA per brick, (NaN, NaN) when a voxel is NaN.
// ---------------------------------------------------------------------------
template <typename T, int LOG2B>
__global__ void __launch_bounds__(256) brick_range_kernel(const T *__restrict__ bricks, long long stride,
                                                           float2 *range)
{
    constexpr int B1 = (1 << LOG2B) + 1, N = B1 * B1 * B1;
    const T *b = bricks + (long long)blockIdx.x * stride;
    float mn = INFINITY, mx = -INFINITY;
    bool nan = false;
    for (int e = threadIdx.x; e < N; e += blockDim.x) {
        const float a = to_f(b[e]);
        if (a != a) nan = true;
        mn = fminf(mn, a);
        mx = fmaxf(mx, a);
    }
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(kFull, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
    }
    nan = __any_sync(kFull, nan);
    __shared__ float smn[8], smx[8];
    __shared__ int snan[8];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        smn[w] = mn;
        smx[w] = mx;
        snan[w] = nan;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bool any_nan = false;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            mn = fminf(mn, smn[q]);
            mx = fmaxf(mx, smx[q]);
            any_nan = any_nan || snan[q];
        }
        range[blockIdx.x] = any_nan ? make_float2(NAN, NAN) : make_float2(mn, mx);
    }
}

cudaError_t launch_brick_range(const VolDev &v, vr_dtype dt, float2 *range, cudaStream_t s)
{
    const unsigned nbricks = (unsigned)((long long)v.nbx * v.nby * v.nbz);
#define VR_RANGE(TT, LB) \
    brick_range_kernel<TT, LB><<<nbricks, 256, 0, s>>>(static_cast<const TT *>(v.data), v.stride, range)
#define VR_RANGE_DT(TT)                 \
    switch (v.log2b) {                  \
    case 4: VR_RANGE(TT, 4); break;     \
    case 5: VR_RANGE(TT, 5); break;     \
    default: VR_RANGE(TT, 6); break;    \
    }
    switch (dt) {
    case VR_F32: VR_RANGE_DT(float); break;
    case VR_F16: VR_RANGE_DT(__half); break;
    case VR_BF16: VR_RANGE_DT(__nv_bfloat16); break;
    }
#undef VR_RANGE_DT
#undef VR_RANGE
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The skipping march
// ---------------------------------------------------------------------------

// True when every table entry reachable from values in r has zero opacity.
__device__ __forceinline__ bool brick_transparent(float2 r, const ParamDev &p, const int *nz_prefix)
{
    if (!(r.x == r.x) || !(r.y == r.y)) return false;
    const float ulo = fminf(fmaxf(fmaf(r.x, p.su, p.ou), 0.0f), p.km1);
    const float uhi = fminf(fmaxf(fmaf(r.y, p.su, p.ou), 0.0f), p.km1);
    const int ilo = max(min(__float2int_rd(ulo), p.K - 2) - 1, 0);
    const int ihi = min(min(__float2int_rd(uhi), p.K - 2) + 2, p.K - 1);
    return nz_prefix[ihi + 1] - nz_prefix[ilo] == 0;
}

// One bit per brick for the table of this call: set when the brick is
// transparent.  One thread per brick; the table's prefix count of non-zero
// opacities is built in shared memory first.
__global__ void __launch_bounds__(256) brick_mask_kernel(const float2 *__restrict__ range, ParamDev p,
                                                          uint32_t *mask, long long nbricks)
{
    extern __shared__ int nz_prefix[];          // K + 1 counts of non-zero opacities below each entry
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int q = 0; q < p.K; ++q) {
            nz_prefix[q] = acc;
            acc += __ldg(&p.tf[q].w) != 0.0f;
        }
        nz_prefix[p.K] = acc;
    }
    __syncthreads();
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool empty = b < nbricks && brick_transparent(__ldg(range + b), p, nz_prefix);
    const unsigned word = __ballot_sync(kFull, empty);
    if ((threadIdx.x & 31) == 0 && b < nbricks) mask[b >> 5] = word;
}

// Ray parameter where the ray leaves [a, b] along one axis (its larger slab
// end), folded into s1; inv = 1 / direction (infinite for a zero component).
__device__ __forceinline__ void slab_exit(float q, float inv, float a, float b, float &s1)
{
    if (isinf(inv)) return;
    const float t0 = (a - q) * inv, t1 = (b - q) * inv;
    s1 = fminf(s1, fmaxf(t0, t1));
}

// The transparency bits, copied into shared memory when they fit (a bit test
// there instead of a dependent global load per brick a ray enters).
constexpr int kMaskSmemWords = 12288;          // 48 KB: 393216 bricks (a 1024^3 cube has 262144)

template <typename T, int LOG2B, int L>
__global__ void __launch_bounds__(kSkipThreads) skip_kernel(VolDev v, CamDev c, ParamDev p,
                                                             const uint32_t *__restrict__ gmask, int mask_words,
                                                             bool mask_in_smem, float4 *out, uint32_t *nsamples,
                                                             unsigned *counter, int tiles_x, unsigned ntiles)
{
    extern __shared__ uint32_t smask[];
    if (mask_in_smem) {
        for (int q = threadIdx.x; q < mask_words; q += blockDim.x) smask[q] = __ldg(gmask + q);
        __syncthreads();
    }
    const uint32_t *mask = mask_in_smem ? smask : gmask;
    const long long nbricks = (long long)v.nbx * v.nby * v.nbz;
    constexpr int B = 1 << LOG2B;
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned tile = 0;
        if (lane == 0) tile = atomicAdd(counter, 1u);
        tile = __shfl_sync(kFull, tile, 0);
        if (tile >= ntiles) break;
        const int i = (int)(tile % tiles_x) * 8 + (lane & 7);
        const int j = (int)(tile / tiles_x) * 4 + (lane >> 3);
        const bool inside = i < c.W && j < c.H;
        Ray ray;
        const bool hit = inside && setup_ray(c, v.nx, v.ny, v.nz, p.step, i, j, ray);
        bool active = hit;
        const float ix = 1.0f / ray.d.x, iy = 1.0f / ray.d.y, iz = 1.0f / ray.d.z, istep = 1.0f / p.step;
        // the brick of the last sample tested, and whether it is transparent:
        // consecutive samples mostly share a brick, so the range is read once
        long long last = -1;
        bool last_empty = false;
        // the first sample at or after k that is not in a transparent brick
        // (ray.n if none), with its cell
        auto next = [&](int k, Cell &cell) {
            while (k < ray.n) {
                cell = locate_t<T, LOG2B, L, false>(v, sample_pos(ray, k, p.step));
                const int bx = cell.x0 >> LOG2B, by = cell.y0 >> LOG2B, bz = cell.z0 >> LOG2B;
                const long long brick = ((long long)bz * v.nby + by) * v.nbx + bx;
                if (brick != last) {
                    last = brick;
                    bool ok = true;
                    if constexpr (kBoundsCheck) ok = index_ok(v.status, brick, nbricks);
                    last_empty = ok && ((mask[brick >> 5] >> (brick & 31)) & 1u);
                    if (last_empty) {
                        // every sample more than one step before the ray leaves the brick's
                        // box is inside it: jump there; the last ones are stepped one by one
                        float s1 = INFINITY;
                        slab_exit(ray.q.x, ix, (float)(bx * B), (float)(bx * B + B), s1);
                        slab_exit(ray.q.y, iy, (float)(by * B), (float)(by * B + B), s1);
                        slab_exit(ray.q.z, iz, (float)(bz * B), (float)(bz * B + B), s1);
                        const float ks = floorf(fmaf(s1 - ray.s_in, istep, -0.5f)) - 1.0f;
                        k = max(k + 1, ks < (float)ray.n ? (int)fmaxf(ks, 0.0f) + 1 : ray.n);
                        continue;
                    }
                }
                if (!last_empty) return k;
                ++k;
            }
            return ray.n;
        };
        Composite acc{0.0f, 0.0f, 0.0f, 1.0f};
        int k = 0, used = 0;
        Cell c0, c1;
        Gathered<T, L> f0, f1;
        if (active) {
            k = next(0, c0);
            if (k < ray.n) fetch_corners<T, LOG2B, L>(v, c0, f0);
            else active = false, used = ray.n;
        }
        auto step = [&](const Cell &cur, const Gathered<T, L> &fc, Cell &nxt, Gathered<T, L> &fn) {
            const int kn = next(k + 1, nxt);
            if (kn < ray.n) fetch_corners<T, LOG2B, L>(v, nxt, fn);
            TfPos tp;
            const float4 e = tf_lookup_l1(p, interp_corners(cur, fc), tp);
            const float aT = e.w * acc.T;
            acc.r = fmaf(aT, e.x, acc.r);
            acc.g = fmaf(aT, e.y, acc.g);
            acc.b = fmaf(aT, e.z, acc.b);
            acc.T = fmaf(-e.w, acc.T, acc.T);
            if (acc.T <= p.t_stop) {
                used = k + 1;
                active = false;
            } else if (kn >= ray.n) {
                used = ray.n;
                active = false;
            }
            k = kn;
        };
        for (;;) {
            if (!__any_sync(kFull, active)) break;
            if (active) step(c0, f0, c1, f1);
            if (!__any_sync(kFull, active)) break;
            if (active) step(c1, f1, c0, f0);
        }
        if (inside) write_pixel(p, acc, hit ? used : 0, out, nsamples, (long long)j * c.W + i);
    }
}

// The skipping march's layouts: those of visit_layout, and the texture
// layers instantiated with the volume's own brick size (LOG2B sizes the
// bricks whose transparency bits the march tests; the layers ignore it).
template <int LOG2B, typename F, typename R>
static R visit_skip_layers_b(const VolDev &v, F &&f, R none)
{
    if (v.order == 0) return f(Layout<TexLayers<float>, LOG2B, 0>{});
    if (v.order == 1) return f(Layout<TexLayers<float>, LOG2B, 1>{});
    if (v.order == 2) return f(Layout<TexLayers<float>, LOG2B, 2>{});
    return none;
}

template <typename F, typename R>
static R visit_skip_layout(const VolDev &v, vr_dtype dt, F &&f, R none)
{
    if (v.paired != 3) return visit_layout(v, dt, f, none);
    if (dt != VR_F32) return none;
    switch (v.log2b) {
    case 4: return visit_skip_layers_b<4>(v, f, none);
    case 5: return visit_skip_layers_b<5>(v, f, none);
    case 6: return visit_skip_layers_b<6>(v, f, none);
    }
    return none;
}

cudaError_t launch_forward_skip(const VolDev &v, vr_dtype dt, const CamDev &c, const ParamDev &p,
                                const float2 *range, uint32_t *mask, float4 *out, uint32_t *nsamples,
                                unsigned *counter, cudaStream_t s)
{
    const long long nbricks = (long long)v.nbx * v.nby * v.nbz;
    const int mask_words = (int)((nbricks + 31) / 32);
    brick_mask_kernel<<<(unsigned)((nbricks + 255) / 256), 256, sizeof(int) * (size_t)(p.K + 1), s>>>(range, p, mask,
                                                                                                   nbricks);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int tiles_x = (c.W + 7) / 8, tiles_y = (c.H + 3) / 4;
    const unsigned ntiles = (unsigned)tiles_x * (unsigned)tiles_y;
    e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const bool in_smem = mask_words <= kMaskSmemWords;
    const size_t smem = in_smem ? sizeof(uint32_t) * (size_t)mask_words : 0;
    return visit_skip_layout(
        v, dt,
        [&](auto lay) {
            using Y = decltype(lay);
            auto fn = skip_kernel<typename Y::type, Y::log2b, Y::order>;   // smem <= 48 KB: no opt-in
            const int per_sm = occupancy_blocks((const void *)fn, kSkipThreads, smem);
            unsigned grid = (unsigned)(per_sm * sm_count());
            const unsigned useful = (ntiles + kSkipThreads / 32 - 1) / (kSkipThreads / 32);
            if (grid > useful) grid = useful;
            if (grid < 1) grid = 1;
            log_line("skip %dx%d: %lld bricks, transparency bits in %s memory, grid %u", c.W, c.H, nbricks,
                     in_smem ? "shared" : "global", grid);
            fn<<<grid, kSkipThreads, smem, s>>>(v, c, p, mask, mask_words, in_smem, out, nsamples, counter, tiles_x,
                                                ntiles);
            return cudaGetLastError();
        },
        cudaErrorInvalidValue);
}

}  // namespace vr
