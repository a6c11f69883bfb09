// vr_forward.cu -- forward ray-casting kernels (Sections 3.3-3.4 and 4.4 of
// Hassan et al. 2012): per pixel, clip the ray to the box, sample at a
// constant step with trilinear interpolation, map each sample through the
// RGBA transfer function and composite front to back, stopping early once the
// accumulated opacity reaches the threshold.
//
// GB300 mapping: persistent warps, one 8x4 pixel tile per warp at a time,
// pulled from a global atomic queue (load balance across uneven ray lengths
// and early termination); voxel gathers go through the read-only L1 path from
// bricks (+apron) so all eight corners of a cell are at constant offsets in
// one brick, with the next sample's gathers in flight while the current one
// is composited; a warp vote retires the tile once every lane's ray has
// finished; float4 image stores.
#include "vr_device.cuh"

#include <cstdlib>
#include <map>
#include <mutex>

namespace vr {

constexpr int kFwdThreads = 256;

// Resident CTAs the register budget is sized for, and samples whose gathers
// are in flight ahead of the one composited: for the texture layers four
// CTAs (64 registers) with two samples ahead (the eight 1080p views of the
// 1024^3 cube 198.6 -> 209.3 Gsamples/s, against five CTAs at 48 registers
// with one; the batched kernel keeps the latter, 1% faster there); the
// compiler's choice and the march's own depth for the brick layouts.
template <typename T> struct FwdMinBlocks { static constexpr int value = 0; };   // 0: no minimum
template <> struct FwdMinBlocks<TexLayers<float>> { static constexpr int value = 4; };
template <typename T> struct FwdDepth { static constexpr int value = Pipeline<T>::depth; };
template <> struct FwdDepth<TexLayers<float>> { static constexpr int value = 2; };

template <typename T, int LOG2B, int L>
__global__ void __launch_bounds__(kFwdThreads, FwdMinBlocks<T>::value) fwd_kernel(VolDev v, CamDev c, ParamDev p, float4 *out,
                                                           uint32_t *nsamples, unsigned *counter, int tiles_x,
                                                           unsigned ntiles)
{
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
        Composite acc{0.0f, 0.0f, 0.0f, 1.0f};
        const int used = march_ray<T, LOG2B, L, IdentityMap, FwdDepth<T>::value>(v, p, ray, hit, acc);
        if (inside) write_pixel(p, acc, hit ? used : 0, out, nsamples, (long long)j * c.W + i);
    }
}

// Hardware-filter alternative: tex3D with cudaFilterModeLinear (texel
// centres at +0.5 in unnormalised coordinates).  Same camera, lookup and
// compositing; only the interpolation differs (8-bit fractional weights).
__global__ void __launch_bounds__(kFwdThreads) fwd_tex_kernel(cudaTextureObject_t tex, int nx, int ny, int nz,
                                                               CamDev c, ParamDev p, float4 *out,
                                                               uint32_t *nsamples, unsigned *counter,
                                                               int tiles_x, unsigned ntiles)
{
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
        const bool hit = inside && setup_ray(c, nx, ny, nz, p.step, i, j, ray);
        Composite acc{0.0f, 0.0f, 0.0f, 1.0f};
        int k = 0;
        bool active = hit;
        while (__any_sync(kFull, active)) {
            if (active) {
                const float3 pos = sample_pos(ray, k, p.step);
                const float val = tex3D<float>(tex, pos.x + 0.5f, pos.y + 0.5f, pos.z + 0.5f);
                TfPos tp;
                const float4 e = tf_lookup_l1(p, val, tp);
                const float aT = e.w * acc.T;
                acc.r = fmaf(aT, e.x, acc.r);
                acc.g = fmaf(aT, e.y, acc.g);
                acc.b = fmaf(aT, e.z, acc.b);
                acc.T = fmaf(-e.w, acc.T, acc.T);
                ++k;
                if (k >= ray.n || acc.T <= p.t_stop) active = false;
            }
        }
        if (inside) write_pixel(p, acc, hit ? k : 0, out, nsamples, (long long)j * c.W + i);
    }
}

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------

int occupancy_blocks(const void *fn, int threads, size_t smem)
{
    static std::mutex mu;
    static std::map<std::pair<const void *, size_t>, int> cache;
    std::lock_guard<std::mutex> g(mu);
    auto key = std::make_pair(fn, smem);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess || nb < 1) nb = 1;
    cache[key] = nb;
    return nb;
}

// Resident CTAs per SM for the persistent forward grid: the occupancy limit,
// at most `cap` (0: none), or VR_FWD_CTAS_PER_SM when set (a tuning knob:
// fewer resident warps thrash the L1 and L2 less).
static int fwd_ctas_per_sm(const void *fn, int cap)
{
    const int occ = occupancy_blocks(fn, kFwdThreads, 0);
    static const int env = [] {
        const char *s = std::getenv("VR_FWD_CTAS_PER_SM");
        return s ? std::atoi(s) : 0;
    }();
    const int want = env > 0 ? env : cap;
    return (want > 0 && want < occ) ? want : occ;
}

// CTAs per SM for the float brick layouts, which serve the views whose rays
// are too far apart for texture layers: three, where each resident ray keeps
// its own cache lines live and more of them thrash L1 and L2 (four 1080p
// views of the 4096 x 4096 x 1024 cube: along z 6.20 -> 5.45 ms, along x
// 7.19 -> 7.01 ms; two were slower again).  The other layouts: the occupancy
// limit (16-bit blocked copies measured the same at two, three and four).
template <typename T> struct FwdCtaCap { static constexpr int value = 0; };
template <> struct FwdCtaCap<float> { static constexpr int value = 3; };

template <typename T, int LOG2B, int L>
static cudaError_t launch_fwd_t(const VolDev &v, const CamDev &c, const ParamDev &p, float4 *out,
                                uint32_t *nsamples, unsigned *counter, cudaStream_t s)
{
    const int tiles_x = (c.W + 7) / 8, tiles_y = (c.H + 3) / 4;
    const unsigned ntiles = (unsigned)tiles_x * (unsigned)tiles_y;
    auto fn = fwd_kernel<T, LOG2B, L>;
    const int per_sm = fwd_ctas_per_sm((const void *)fn, FwdCtaCap<T>::value);
    unsigned grid = (unsigned)(per_sm * sm_count());
    const unsigned max_useful = (ntiles + kFwdThreads / 32 - 1) / (kFwdThreads / 32);
    if (grid > max_useful) grid = max_useful;
    if (grid < 1) grid = 1;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    log_line("forward %dx%d: layout order %d%s, %u tiles of 8x4 rays, grid %u x %d threads (%d per SM)", c.W, c.H,
             v.order, v.paired == 1 ? " paired" : (v.paired == 2 ? " blocked" : (v.paired == 3 ? " texture layers" : "")),
             ntiles, grid, kFwdThreads,
             per_sm);
    fn<<<grid, kFwdThreads, 0, s>>>(v, c, p, out, nsamples, counter, tiles_x, ntiles);
    return cudaGetLastError();
}

cudaError_t launch_forward(const VolDev &v, vr_dtype dt, const CamDev &c, const ParamDev &p, float4 *out,
                           uint32_t *nsamples, unsigned *counter, cudaStream_t s)
{
    return visit_layout_all(
        v, dt,
        [&](auto lay) {
            using Y = decltype(lay);
            return launch_fwd_t<typename Y::type, Y::log2b, Y::order>(v, c, p, out, nsamples, counter, s);
        },
        cudaErrorInvalidValue);
}

cudaError_t launch_forward_texture(const vr_volume *vol, const CamDev &c, const ParamDev &p, float4 *out,
                                   uint32_t *nsamples, unsigned *counter, cudaStream_t s)
{
    const int tiles_x = (c.W + 7) / 8, tiles_y = (c.H + 3) / 4;
    const unsigned ntiles = (unsigned)tiles_x * (unsigned)tiles_y;
    const int per_sm = occupancy_blocks((const void *)fwd_tex_kernel, kFwdThreads, 0);
    unsigned grid = (unsigned)(per_sm * sm_count());
    const unsigned max_useful = (ntiles + kFwdThreads / 32 - 1) / (kFwdThreads / 32);
    if (grid > max_useful) grid = max_useful;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    fwd_tex_kernel<<<grid, kFwdThreads, 0, s>>>(vol->tex, (int)vol->dims[0], (int)vol->dims[1], (int)vol->dims[2],
                                                c, p, out, nsamples, counter, tiles_x, ntiles);
    return cudaGetLastError();
}

}  // namespace vr
