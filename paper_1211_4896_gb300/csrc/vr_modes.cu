// vr_modes.cu -- the paper's other uses of the same ray march:
//   - maximum intensity projection (Section 3.3.1): the largest sample value
//     on each ray, shown through the colour map;
//   - the sigma-clipping transfer function (Section 4.5): a statistical
//     mini-map holds the mean and standard deviation of regions of the cube,
//     and each sample value is scaled by the statistics interpolated at its
//     position before the table lookup;
//   - the 3D spectrum tool (Section 4.4): the data profile along one pixel's
//     line of sight, at the renderer's sample positions.
// Same camera, clipping, sampling, brick layouts and work queue as
// vr_forward.cu.
#include "vr_device.cuh"

#include <cmath>

namespace vr {

constexpr int kModeThreads = 256;

// ---------------------------------------------------------------------------
// Maximum intensity projection
// ---------------------------------------------------------------------------

// Largest interpolated value of the ray's samples (all of them: no early
// termination); the next sample's gathers are issued before the current one
// is compared (two register sets in turn).
template <typename T, int LOG2B, int L>
__device__ __forceinline__ float march_max(const VolDev &v, const ParamDev &p, const Ray &ray, bool active)
{
    float m = -INFINITY;
    int k = 0;
    Cell c0, c1;
    Gathered<T, L> f0, f1;
    if (active) {
        c0 = locate<LOG2B, L>(v, sample_pos(ray, 0, p.step));
        fetch_corners<T, LOG2B, L>(v, c0, f0);
    }
    auto step = [&](const Cell &cur, const Gathered<T, L> &fc, Cell &nxt, Gathered<T, L> &fn) {
        const bool more = k + 1 < ray.n;
        if (more) {
            nxt = locate<LOG2B, L>(v, sample_pos(ray, k + 1, p.step));
            fetch_corners<T, LOG2B, L>(v, nxt, fn);
        }
        m = fmaxf(m, interp_corners(cur, fc));
        ++k;
        if (!more) active = false;
    };
    for (;;) {
        if (!__any_sync(kFull, active)) break;
        if (active) step(c0, f0, c1, f1);
        if (!__any_sync(kFull, active)) break;
        if (active) step(c1, f1, c0, f0);
    }
    return m;
}

// The pixel is the table entry of the largest value composited once over
// the background; a ray that misses the box shows the background.
template <typename T, int LOG2B, int L>
__global__ void __launch_bounds__(kModeThreads) mip_kernel(VolDev v, CamDev c, ParamDev p, float4 *out,
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
        const float m = march_max<T, LOG2B, L>(v, p, ray, hit);
        if (!inside) continue;
        const long long px = (long long)j * c.W + i;
        float4 o = p.bg;
        if (hit) {
            TfPos tp;
            const float4 e = tf_lookup_l1(p, m, tp);
            const float a = e.w, t = 1.0f - e.w;
            o = make_float4(fmaf(a, e.x, t * p.bg.x), fmaf(a, e.y, t * p.bg.y), fmaf(a, e.z, t * p.bg.z),
                            fmaf(t, p.bg.w, a));
        }
        out[px] = o;
        if (nsamples) nsamples[px] = hit ? (uint32_t)ray.n : 0u;
    }
}

// ---------------------------------------------------------------------------
// Sigma clipping
// ---------------------------------------------------------------------------

// Device view of a mini-map: (mean, sd) per point, x fastest; point i of an
// axis sits at voxel (i + 1/2) region - 1/2.
struct MiniDev {
    const float2 *mm;
    int mx, my, mz;
    float rx, ry, rz;          // 1 / region size
};

__device__ __forceinline__ void mini_axis(float p, float rinv, int m, int &i0, int &i1, float &w)
{
    if (m < 2) {
        i0 = i1 = 0;
        w = 0.0f;
        return;
    }
    const float g = fmaf(p + 0.5f, rinv, -0.5f);
    i0 = min(max(__float2int_rd(g), 0), m - 2);
    i1 = i0 + 1;
    w = fminf(fmaxf(g - (float)i0, 0.0f), 1.0f);
}

// The sample value in units of the local standard deviation above the local
// mean (trilinear on the mini-map at the sample's position; a standard
// deviation below 1e-30 counts as 1e-30).
struct SigmaMap {
    MiniDev m;
    __device__ __forceinline__ float operator()(float v, const Cell &c) const
    {
        int x0, x1, y0, y1, z0, z1;
        float wx, wy, wz;
        mini_axis((float)c.x0 + c.fx, m.rx, m.mx, x0, x1, wx);
        mini_axis((float)c.y0 + c.fy, m.ry, m.my, y0, y1, wy);
        mini_axis((float)c.z0 + c.fz, m.rz, m.mz, z0, z1, wz);
        const long long sy = m.mx, sz = (long long)m.mx * m.my;
        const float2 *b0 = m.mm + z0 * sz, *b1 = m.mm + z1 * sz;
        const float2 a000 = __ldg(b0 + y0 * sy + x0), a100 = __ldg(b0 + y0 * sy + x1);
        const float2 a010 = __ldg(b0 + y1 * sy + x0), a110 = __ldg(b0 + y1 * sy + x1);
        const float2 a001 = __ldg(b1 + y0 * sy + x0), a101 = __ldg(b1 + y0 * sy + x1);
        const float2 a011 = __ldg(b1 + y1 * sy + x0), a111 = __ldg(b1 + y1 * sy + x1);
        auto lerp = [](float a, float b, float w) { return fmaf(w, b - a, a); };
        const float mean = lerp(lerp(lerp(a000.x, a100.x, wx), lerp(a010.x, a110.x, wx), wy),
                                lerp(lerp(a001.x, a101.x, wx), lerp(a011.x, a111.x, wx), wy), wz);
        const float sd = lerp(lerp(lerp(a000.y, a100.y, wx), lerp(a010.y, a110.y, wx), wy),
                              lerp(lerp(a001.y, a101.y, wx), lerp(a011.y, a111.y, wx), wy), wz);
        return (v - mean) / fmaxf(sd, 1e-30f);
    }
};

template <typename T, int LOG2B, int L>
__global__ void __launch_bounds__(kModeThreads) sigma_kernel(VolDev v, CamDev c, ParamDev p, MiniDev m, float4 *out,
                                                              uint32_t *nsamples, unsigned *counter, int tiles_x,
                                                              unsigned ntiles)
{
    const int lane = threadIdx.x & 31;
    const SigmaMap map{m};
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
        const int used = march_ray<T, LOG2B, L, SigmaMap>(v, p, ray, hit, acc, map);
        if (inside) write_pixel(p, acc, hit ? used : 0, out, nsamples, (long long)j * c.W + i);
    }
}

template <typename K>
static unsigned persistent_grid(K fn, unsigned ntiles)
{
    const int per_sm = occupancy_blocks((const void *)fn, kModeThreads, 0);
    unsigned grid = (unsigned)(per_sm * sm_count());
    const unsigned useful = (ntiles + kModeThreads / 32 - 1) / (kModeThreads / 32);
    if (grid > useful) grid = useful;
    return grid < 1 ? 1 : grid;
}

cudaError_t launch_mip(const VolDev &v, vr_dtype dt, const CamDev &c, const ParamDev &p, float4 *out,
                       uint32_t *nsamples, unsigned *counter, cudaStream_t s)
{
    const int tiles_x = (c.W + 7) / 8, tiles_y = (c.H + 3) / 4;
    const unsigned ntiles = (unsigned)tiles_x * (unsigned)tiles_y;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    return visit_layout(
        v, dt,
        [&](auto lay) {
            using Y = decltype(lay);
            auto fn = mip_kernel<typename Y::type, Y::log2b, Y::order>;
            fn<<<persistent_grid(fn, ntiles), kModeThreads, 0, s>>>(v, c, p, out, nsamples, counter, tiles_x,
                                                                    ntiles);
            return cudaGetLastError();
        },
        cudaErrorInvalidValue);
}

cudaError_t launch_sigma(const VolDev &v, vr_dtype dt, const CamDev &c, const ParamDev &p, const float *minimap,
                         const int region[3], float4 *out, uint32_t *nsamples, unsigned *counter, cudaStream_t s)
{
    MiniDev m;
    m.mm = reinterpret_cast<const float2 *>(minimap);
    m.mx = (v.nx + region[0] - 1) / region[0];
    m.my = (v.ny + region[1] - 1) / region[1];
    m.mz = (v.nz + region[2] - 1) / region[2];
    m.rx = (float)(1.0 / region[0]);
    m.ry = (float)(1.0 / region[1]);
    m.rz = (float)(1.0 / region[2]);
    const int tiles_x = (c.W + 7) / 8, tiles_y = (c.H + 3) / 4;
    const unsigned ntiles = (unsigned)tiles_x * (unsigned)tiles_y;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    return visit_layout(
        v, dt,
        [&](auto lay) {
            using Y = decltype(lay);
            auto fn = sigma_kernel<typename Y::type, Y::log2b, Y::order>;
            fn<<<persistent_grid(fn, ntiles), kModeThreads, 0, s>>>(v, c, p, m, out, nsamples, counter, tiles_x,
                                                                    ntiles);
            return cudaGetLastError();
        },
        cudaErrorInvalidValue);
}

// ---------------------------------------------------------------------------
// Statistical mini-map: one CTA per region, two passes (mean, then the mean
// squared deviation) over the region's voxels with FP64 sums.
// ---------------------------------------------------------------------------

__device__ __forceinline__ double block_sum(double x, double *red)
{
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();                  // red[] may still be read by the previous call
    if (lane == 0) red[w] = x;
    __syncthreads();
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    return t;
}

// Voxel (x, y, z) of the x-fastest bricks: the brick that owns it (the last
// voxel of an axis may sit in the apron of the last brick).
template <typename T>
__device__ __forceinline__ float brick_voxel(const VolDev &v, int x, int y, int z)
{
    const int B = 1 << v.log2b, B1 = B + 1;
    const int bx = min(x >> v.log2b, v.nbx - 1), by = min(y >> v.log2b, v.nby - 1), bz = min(z >> v.log2b, v.nbz - 1);
    const long long brick = ((long long)bz * v.nby + by) * v.nbx + bx;
    const long long e = ((long long)(z - bz * B) * B1 + (y - by * B)) * B1 + (x - bx * B);
    return to_f(static_cast<const T *>(v.data)[brick * v.stride + e]);
}

template <typename T>
__global__ void __launch_bounds__(256) minimap_kernel(VolDev v, int rx, int ry, int rz, int mx, int my,
                                                       float2 *out)
{
    __shared__ double red[32];
    const long long q = blockIdx.x;
    const int i = (int)(q % mx), j = (int)((q / mx) % my), k = (int)(q / ((long long)mx * my));
    const int x0 = i * rx, y0 = j * ry, z0 = k * rz;
    const int lx = min(x0 + rx, v.nx) - x0, ly = min(y0 + ry, v.ny) - y0, lz = min(z0 + rz, v.nz) - z0;
    const long long cnt = (long long)lx * ly * lz;
    double s = 0.0;
    for (long long e = threadIdx.x; e < cnt; e += blockDim.x) {
        const int x = (int)(e % lx), y = (int)((e / lx) % ly), z = (int)(e / ((long long)lx * ly));
        s += (double)brick_voxel<T>(v, x0 + x, y0 + y, z0 + z);
    }
    const double mean = block_sum(s, red) / (double)cnt;
    double ss = 0.0;
    for (long long e = threadIdx.x; e < cnt; e += blockDim.x) {
        const int x = (int)(e % lx), y = (int)((e / lx) % ly), z = (int)(e / ((long long)lx * ly));
        const double d = (double)brick_voxel<T>(v, x0 + x, y0 + y, z0 + z) - mean;
        ss += d * d;
    }
    const double var = block_sum(ss, red) / (double)cnt;
    if (threadIdx.x == 0) out[q] = make_float2((float)mean, (float)sqrt(var));
}

cudaError_t launch_minimap(const VolDev &v, vr_dtype dt, const int region[3], float *dev_out, cudaStream_t s)
{
    const int mx = (v.nx + region[0] - 1) / region[0], my = (v.ny + region[1] - 1) / region[1],
              mz = (v.nz + region[2] - 1) / region[2];
    const long long n = (long long)mx * my * mz;
    if (n > 0x7fffffffLL) return cudaErrorInvalidValue;
    float2 *o = reinterpret_cast<float2 *>(dev_out);
    switch (dt) {
    case VR_F32: minimap_kernel<float><<<(unsigned)n, 256, 0, s>>>(v, region[0], region[1], region[2], mx, my, o); break;
    case VR_F16: minimap_kernel<__half><<<(unsigned)n, 256, 0, s>>>(v, region[0], region[1], region[2], mx, my, o); break;
    case VR_BF16:
        minimap_kernel<__nv_bfloat16><<<(unsigned)n, 256, 0, s>>>(v, region[0], region[1], region[2], mx, my, o);
        break;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// 3D spectrum tool: one thread per sample of pixel (i, j)'s ray.
// ---------------------------------------------------------------------------

template <typename T, int LOG2B>
__global__ void __launch_bounds__(256) profile_kernel(VolDev v, CamDev c, float step, int i, int j, float *values,
                                                       unsigned max_values, unsigned *count)
{
    Ray ray;
    const bool hit = setup_ray(c, v.nx, v.ny, v.nz, step, i, j, ray);
    const int n = hit ? ray.n : 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = (unsigned)n;
    const long long lim = min((long long)n, (long long)max_values);
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < lim; k += (long long)gridDim.x * blockDim.x) {
        const Cell cell = locate<LOG2B, 0>(v, sample_pos(ray, (int)k, step));
        Gathered<T, 0> f;
        fetch_corners<T, LOG2B, 0>(v, cell, f);
        values[k] = interp_corners(cell, f);
    }
}

cudaError_t launch_profile(const VolDev &v, vr_dtype dt, const CamDev &c, float step, int i, int j, float *values,
                           unsigned max_values, unsigned *count, cudaStream_t s)
{
    const unsigned blocks = max(1u, min((max_values + 255u) / 256u, 4096u));
    const VolDev vb = v;       // the x-fastest bricks (order 0, plain)
#define VR_PROFILE(TT, LB) profile_kernel<TT, LB><<<blocks, 256, 0, s>>>(vb, c, step, i, j, values, max_values, count)
#define VR_PROFILE_DT(TT)                  \
    switch (v.log2b) {                     \
    case 4: VR_PROFILE(TT, 4); break;      \
    case 5: VR_PROFILE(TT, 5); break;      \
    default: VR_PROFILE(TT, 6); break;     \
    }
    switch (dt) {
    case VR_F32: VR_PROFILE_DT(float); break;
    case VR_F16: VR_PROFILE_DT(__half); break;
    case VR_BF16: VR_PROFILE_DT(__nv_bfloat16); break;
    }
#undef VR_PROFILE_DT
#undef VR_PROFILE
    return cudaGetLastError();
}

}  // namespace vr
