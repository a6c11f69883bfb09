// vr_modes.cu -- the paper's other uses of the same ray march:
//   - maximum intensity projection (Section 3.3.1): the largest sample value
//     on each ray, shown through the colour map;
//   - the sigma-clipping transfer function (Section 4.5): a statistical
//     mini-map holds the mean and standard deviation of regions of the cube,
//     and each sample value is scaled by the statistics interpolated at its
//     position before the table lookup;
//   - the 3D spectrum tool (Section 4.4): the data profile along one pixel's
//     line of sight, at the renderer's sample positions;
//   - sort-last rendering (Sections 3.2, 3.4): partial images of sub-boxes of
//     cells, composited over one another in depth order.
// Same camera, clipping, sampling, brick layouts and work queue as
// vr_forward.cu.
#include "vr_device.cuh"

#include <algorithm>
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
        c0 = locate_t<T, LOG2B, L, false>(v, sample_pos(ray, 0, p.step));
        fetch_corners<T, LOG2B, L>(v, c0, f0);
    }
    auto step = [&](const Cell &cur, const Gathered<T, L> &fc, Cell &nxt, Gathered<T, L> &fn) {
        const bool more = k + 1 < ray.n;
        if (more) {
            nxt = locate_t<T, LOG2B, L, false>(v, sample_pos(ray, k + 1, p.step));
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
// Resident CTAs the maximum intensity projection's register budget is sized
// for: five for the texture layers (as the forward), the compiler's choice
// for the brick layouts.
template <typename T> struct ModeMinBlocks { static constexpr int value = 0; };   // 0: no minimum
template <> struct ModeMinBlocks<TexLayers<float>> { static constexpr int value = 5; };

template <typename T, int LOG2B, int L>
__global__ void __launch_bounds__(kModeThreads, ModeMinBlocks<T>::value) mip_kernel(VolDev v, CamDev c, ParamDev p, float4 *out,
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
    unsigned *status;          // the bounds-check build's report
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
        if constexpr (kBoundsCheck) {
            if (!index_ok(m.status, z0 * sz + y0 * sy + x0, sz * m.mz) ||
                !index_ok(m.status, z1 * sz + y1 * sy + x1, sz * m.mz))
                return 0.0f;
        }
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
    return visit_layout_tex(
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
    m.status = v.status;
    const int tiles_x = (c.W + 7) / 8, tiles_y = (c.H + 3) / 4;
    const unsigned ntiles = (unsigned)tiles_x * (unsigned)tiles_y;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    return visit_layout_tex(
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
// Sort-last rendering (Sections 3.2 and 3.4): the samples of the whole
// volume's ray whose cell lies in a sub-box [lo, hi) of cells, composited
// into a partial image (premultiplied C, transmittance T, depth of the first
// sample); partial images composite over one another in depth order.
// ---------------------------------------------------------------------------

// Ray parameters where the ray is inside [a, b] along one axis (intersected
// into [s0, s1]); false when it misses.
__device__ __forceinline__ bool slab_range(float q, float d, float a, float b, float &s0, float &s1)
{
    if (d == 0.0f) return q >= a && q <= b;
    const float inv = 1.0f / d;
    float t0 = (a - q) * inv, t1 = (b - q) * inv;
    if (t0 > t1) {
        const float t = t0;
        t0 = t1;
        t1 = t;
    }
    s0 = fmaxf(s0, t0);
    s1 = fminf(s1, t1);
    return s0 <= s1;
}

// Ray parameter of the eye (perspective) or of the image plane (orthographic)
// in the units of Ray: depths are reported from there, like the oracle's t.
__device__ __forceinline__ float eye_param(const CamDev &c, int i, int j)
{
    if (!c.persp) return -c.dist;
    const float hi = (float)i - 0.5f * (float)(c.W - 1);
    const float hj = (float)j - 0.5f * (float)(c.H - 1);
    const float wx = fmaf(hi, c.wa.x, fmaf(hj, c.wb.x, c.wf.x));
    const float wy = fmaf(hi, c.wa.y, fmaf(hj, c.wb.y, c.wf.y));
    const float wz = fmaf(hi, c.wa.z, fmaf(hj, c.wb.z, c.wf.z));
    return -c.dist * sqrtf(wx * wx + wy * wy + wz * wz);
}

template <typename T, int LOG2B, int L>
__global__ void __launch_bounds__(kModeThreads) subbox_kernel(VolDev v, CamDev c, ParamDev p, int3 lo, int3 hi,
                                                               int3 gdim, float3 off, float4 *partial, float *depth,
                                                               uint32_t *count, unsigned *counter, int tiles_x,
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
        const bool inside_img = i < c.W && j < c.H;
        Ray ray;
        // rays and samples of the whole grid (gdim voxels; the camera is in its
        // coordinates); the volume holds its voxels from off on
        bool active = inside_img && setup_ray(c, gdim.x, gdim.y, gdim.z, p.step, i, j, ray);
        // samples whose position lies in the sub-box widened by one voxel: the
        // exact cell test below decides each of them
        int k = 0, k_end = 0;
        if (active) {
            float s0 = -INFINITY, s1 = INFINITY;
            active = slab_range(ray.q.x, ray.d.x, (float)lo.x - 1.0f, (float)hi.x + 1.0f, s0, s1) &&
                     slab_range(ray.q.y, ray.d.y, (float)lo.y - 1.0f, (float)hi.y + 1.0f, s0, s1) &&
                     slab_range(ray.q.z, ray.d.z, (float)lo.z - 1.0f, (float)hi.z + 1.0f, s0, s1);
            if (active) {
                const float k0 = floorf((s0 - ray.s_in) / p.step - 0.5f) - 1.0f;
                const float k1 = ceilf((s1 - ray.s_in) / p.step - 0.5f) + 2.0f;
                k = (int)fmaxf(k0, 0.0f);
                k_end = (int)fminf(k1, (float)ray.n);
                active = k < k_end;
            }
        }
        float Cr = 0.0f, Cg = 0.0f, Cb = 0.0f, Tt = 1.0f;
        int first = -1, used = 0;
        Cell c0, c1;
        Gathered<T, L> f0, f1;
        auto local = [&](int q) {
            const float3 g = sample_pos(ray, q, p.step);
            return make_float3(g.x - off.x, g.y - off.y, g.z - off.z);     // exact for 0 <= off <= g
        };
        if (active) {
            c0 = locate_t<T, LOG2B, L, false>(v, local(k));
            fetch_corners<T, LOG2B, L>(v, c0, f0);
        }
        auto step = [&](const Cell &cur, const Gathered<T, L> &fc, Cell &nxt, Gathered<T, L> &fn) {
            const bool more = k + 1 < k_end;
            if (more) {
                nxt = locate_t<T, LOG2B, L, false>(v, local(k + 1));
                fetch_corners<T, LOG2B, L>(v, nxt, fn);
            }
            // the sample's cell in the whole grid, clamped as the whole render clamps it
            // (x0 + fx is the local position exactly)
            const int gx = min(max(__float2int_rd((float)cur.x0 + cur.fx) + (int)off.x, 0), gdim.x - 2);
            const int gy = min(max(__float2int_rd((float)cur.y0 + cur.fy) + (int)off.y, 0), gdim.y - 2);
            const int gz = min(max(__float2int_rd((float)cur.z0 + cur.fz) + (int)off.z, 0), gdim.z - 2);
            if (gx >= lo.x && gx < hi.x && gy >= lo.y && gy < hi.y && gz >= lo.z && gz < hi.z) {
                TfPos tp;
                const float4 e = tf_lookup_l1(p, interp_corners(cur, fc), tp);
                const float aT = e.w * Tt;
                Cr = fmaf(aT, e.x, Cr);
                Cg = fmaf(aT, e.y, Cg);
                Cb = fmaf(aT, e.z, Cb);
                Tt = fmaf(-e.w, Tt, Tt);
                if (first < 0) first = k;
                ++used;
            }
            ++k;
            if (!more) active = false;
        };
        for (;;) {
            if (!__any_sync(kFull, active)) break;
            if (active) step(c0, f0, c1, f1);
            if (!__any_sync(kFull, active)) break;
            if (active) step(c1, f1, c0, f0);
        }
        if (!inside_img) continue;
        const long long px = (long long)j * c.W + i;
        partial[px] = make_float4(Cr, Cg, Cb, Tt);
        depth[px] = first >= 0 ? fmaf((float)first + 0.5f, p.step, ray.s_in) - eye_param(c, i, j) : INFINITY;
        if (count) count[px] = (uint32_t)used;
    }
}

cudaError_t launch_subbox(const VolDev &v, vr_dtype dt, const CamDev &c, const ParamDev &p, const int lo[3],
                          const int hi[3], const int gdim[3], const int off[3], float4 *partial, float *depth,
                          uint32_t *count, unsigned *counter, cudaStream_t s)
{
    const int tiles_x = (c.W + 7) / 8, tiles_y = (c.H + 3) / 4;
    const unsigned ntiles = (unsigned)tiles_x * (unsigned)tiles_y;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const int3 l3 = make_int3(lo[0], lo[1], lo[2]), h3 = make_int3(hi[0], hi[1], hi[2]);
    const int3 g3 = make_int3(gdim[0], gdim[1], gdim[2]);
    const float3 o3 = make_float3((float)off[0], (float)off[1], (float)off[2]);
    return visit_layout_tex(
        v, dt,
        [&](auto lay) {
            using Y = decltype(lay);
            auto fn = subbox_kernel<typename Y::type, Y::log2b, Y::order>;
            fn<<<persistent_grid(fn, ntiles), kModeThreads, 0, s>>>(v, c, p, l3, h3, g3, o3, partial, depth, count,
                                                                    counter, tiles_x, ntiles);
            return cudaGetLastError();
        },
        cudaErrorInvalidValue);
}

// Over-composite of k partial images per pixel, ordered by depth (front
// first); the pixel is (C + T bg.rgb, 1 - T + T bg.a).
struct PartialList {
    const float4 *img[kMaxPartials];
    const float *depth[kMaxPartials];
};

__global__ void __launch_bounds__(256) composite_kernel(PartialList pl, int k, long long npx, float4 bg,
                                                         float4 *out)
{
    for (long long px = (long long)blockIdx.x * blockDim.x + threadIdx.x; px < npx;
         px += (long long)gridDim.x * blockDim.x) {
        float d[kMaxPartials];
        unsigned char ord[kMaxPartials];
        for (int q = 0; q < k; ++q) {
            d[q] = pl.depth[q][px];
            ord[q] = (unsigned char)q;
        }
        for (int q = 1; q < k; ++q)               // insertion sort by depth (stable)
            for (int r = q; r > 0 && d[ord[r]] < d[ord[r - 1]]; --r) {
                const unsigned char t = ord[r];
                ord[r] = ord[r - 1];
                ord[r - 1] = t;
            }
        float Cr = 0.0f, Cg = 0.0f, Cb = 0.0f, T = 1.0f;
        for (int q = 0; q < k; ++q) {
            const float4 s = pl.img[ord[q]][px];
            Cr = fmaf(T, s.x, Cr);
            Cg = fmaf(T, s.y, Cg);
            Cb = fmaf(T, s.z, Cb);
            T *= s.w;
        }
        out[px] = make_float4(fmaf(T, bg.x, Cr), fmaf(T, bg.y, Cg), fmaf(T, bg.z, Cb), fmaf(T, bg.w, 1.0f - T));
    }
}

cudaError_t launch_composite(int k, const float *const *partials, const float *const *depths, long long npx,
                             const float bg[4], float *out, cudaStream_t s)
{
    PartialList pl;
    for (int q = 0; q < k; ++q) {
        pl.img[q] = reinterpret_cast<const float4 *>(partials[q]);
        pl.depth[q] = depths[q];
    }
    const long long blocks = std::min<long long>((npx + 255) / 256, (long long)sm_count() * 16);
    composite_kernel<<<(unsigned)std::max<long long>(blocks, 1), 256, 0, s>>>(
        pl, k, npx, make_float4(bg[0], bg[1], bg[2], bg[3]), reinterpret_cast<float4 *>(out));
    return cudaGetLastError();
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
