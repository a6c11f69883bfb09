// vr_backward.cu -- adjoint of the forward ray caster (an extension; the paper
// renders only): gradients of a scalar loss with respect to the transfer-
// function table and the voxel values, given dL/d(image).
//
// Each ray is re-marched front to back from the forward's stored pixel and
// sample count; per-sample state is recomputed, not stored.  With C the
// composited colour, T_k the transmittance in front of sample k and
// I = (C + T_n bg.rgb, 1 - T_n (1 - bg.a)), g = dL/dI.rgb, gA = dL/dI.a,
// gT = g.bg.rgb - gA (1 - bg.a):
//   dL/dc_k = T_k a_k g
//   dL/da_k = T_k (c_k.g) - [ (C - C_<=k).g + gT T_n ] / (1 - a_k)
// where (C - C_<=k).g is the final colour minus the running colour, both
// dotted with g, so one scalar R_k is carried along the march.
//
// Persistent warps pull 8x4 ray tiles from the same atomic queue as the
// forward.  Every warp owns a private FP32 row of K RGBA gradient bins in
// global memory (L2-resident); a sample adds its two weighted contributions
// with two fire-and-forget 16-byte vector reductions.  One final kernel sums
// the warps' rows in FP64 (the only FP64 arithmetic: the cross-block sum).
// The voxel gradient is scattered into the dense layout with reductions, the
// two x-neighbours of a corner pair as one 8-byte reduction when aligned.
#include "vr_device.cuh"

namespace vr {

constexpr int kBwdThreads = 256;
constexpr int kBwdWarps = kBwdThreads / 32;

__device__ __forceinline__ void red_add_v4(float4 *a, float4 v)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"l"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

__device__ __forceinline__ void red_add_v2(float *a, float x, float y)
{
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};\n" ::"l"(a), "f"(x), "f"(y) : "memory");
}

__device__ __forceinline__ void red_add_f32(float *a, float x)
{
    asm volatile("red.global.add.f32 [%0], %1;\n" ::"l"(a), "f"(x) : "memory");
}

// dv distributed to the 8 corners of the cell whose (x0, y0, z0) corner is at gv.
__device__ __forceinline__ void scatter_corners(float *gv, long long nx, long long nyx, float fx, float fy, float fz,
                                                float dv)
{
    const float wx0 = 1.0f - fx, wy0 = 1.0f - fy, wz0 = 1.0f - fz;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float a = ((q & 1) ? fy : wy0) * ((q & 2) ? fz : wz0) * dv;
        float *b = gv + ((q & 1) ? nx : 0) + ((q & 2) ? nyx : 0);
        if ((reinterpret_cast<uintptr_t>(b) & 7u) == 0) {
            red_add_v2(b, wx0 * a, fx * a);
        } else {
            red_add_f32(b, wx0 * a);
            red_add_f32(b + 1, fx * a);
        }
    }
}

__device__ __forceinline__ float4 f4_axpy(float a, float4 x, float4 y)
{
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}

// A ray's pending table-gradient contributions: bins b and b+1 of this
// thread's row.  Consecutive samples whose bin pair coincides or overlaps are
// added here and reach memory once.
struct BinRun {
    int b = -1;
    float4 lo = {0.f, 0.f, 0.f, 0.f}, hi = {0.f, 0.f, 0.f, 0.f};
    __device__ __forceinline__ void add(float4 *row, int i0, float w0, float w1, float4 dr)
    {
        if (i0 == b) {
            lo = f4_axpy(w0, dr, lo);
            hi = f4_axpy(w1, dr, hi);
            return;
        }
        if (i0 == b + 1) {                 // new lower bin == pending upper bin
            red_add_v4(row + b, lo);
            lo = f4_axpy(w0, dr, hi);
        } else if (i0 + 1 == b) {          // new upper bin == pending lower bin
            red_add_v4(row + b + 1, hi);
            hi = f4_axpy(w1, dr, lo);
            lo = make_float4(w0 * dr.x, w0 * dr.y, w0 * dr.z, w0 * dr.w);
            b = i0;
            return;
        } else {
            flush(row);
            lo = make_float4(w0 * dr.x, w0 * dr.y, w0 * dr.z, w0 * dr.w);
        }
        hi = make_float4(w1 * dr.x, w1 * dr.y, w1 * dr.z, w1 * dr.w);
        b = i0;
    }
    __device__ __forceinline__ void flush(float4 *row)
    {
        if (b >= 0) {
            red_add_v4(row + b, lo);
            red_add_v4(row + b + 1, hi);
        }
        b = -1;
    }
};

// A ray's pending voxel-gradient contributions to the 8 corners of one cell.
struct CellRun {
    float *base = nullptr;             // corner (x0, y0, z0) in the dense gradient
    float acc[8];
    __device__ __forceinline__ void add(float *gv, float fx, float fy, float fz, float dv, long long nx,
                                        long long nyx)
    {
        if (gv != base) {
            flush(nx, nyx);
            base = gv;
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] = 0.0f;
        }
        const float wx0 = 1.0f - fx, wy0 = 1.0f - fy, wz0 = 1.0f - fz;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float a = ((q & 1) ? fy : wy0) * ((q & 2) ? fz : wz0) * dv;
            acc[2 * q] = fmaf(wx0, a, acc[2 * q]);
            acc[2 * q + 1] = fmaf(fx, a, acc[2 * q + 1]);
        }
    }
    __device__ __forceinline__ void flush(long long nx, long long nyx)
    {
        if (!base) return;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float *b = base + ((q & 1) ? nx : 0) + ((q & 2) ? nyx : 0);
            if ((reinterpret_cast<uintptr_t>(b) & 7u) == 0) {
                red_add_v2(b, acc[2 * q], acc[2 * q + 1]);
            } else {
                red_add_f32(b, acc[2 * q]);
                red_add_f32(b + 1, acc[2 * q + 1]);
            }
        }
        base = nullptr;
    }
};

template <typename VT, int LOG2B, int L>
__global__ void __launch_bounds__(kBwdThreads) bwd_kernel(VolDev v, CamDev c, ParamDev p,
                                                           const float4 *__restrict__ rgba,
                                                           const uint32_t *__restrict__ nsamples,
                                                           const float4 *__restrict__ grad_rgba, float4 *wtab,
                                                           float *grad_vox, unsigned *counter, int tiles_x,
                                                           unsigned ntiles)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4 *row = wtab + ((size_t)blockIdx.x * kBwdWarps + warp) * (size_t)p.K;     // this warp's bins
    const float vscale = p.km1 * p.scale01;    // du/dv inside the range
    const long long nyx = (long long)v.ny * v.nx;

    for (;;) {
        unsigned tile = 0;
        if (lane == 0) tile = atomicAdd(counter, 1u);
        tile = __shfl_sync(kFull, tile, 0);
        if (tile >= ntiles) break;
        const int i = (int)(tile % tiles_x) * 8 + (lane & 7);
        const int j = (int)(tile / tiles_x) * 4 + (lane >> 3);
        Ray ray;
        int n = 0;
        float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
        float R = 0.0f;
        if (i < c.W && j < c.H) {
            const long long px = (long long)j * c.W + i;
            n = (int)nsamples[px];
            if (n > 0 && setup_ray(c, v.nx, v.ny, v.nz, p.step, i, j, ray)) {
                n = min(n, ray.n);
                const float4 out = rgba[px];
                g = grad_rgba[px];
                const float Tn = (1.0f - out.w) / (1.0f - p.bg.w);
                const float Cg = (out.x - Tn * p.bg.x) * g.x + (out.y - Tn * p.bg.y) * g.y +
                                 (out.z - Tn * p.bg.z) * g.z;
                const float gT = g.x * p.bg.x + g.y * p.bg.y + g.z * p.bg.z - g.w * (1.0f - p.bg.w);
                R = Cg + gT * Tn;            // R_{-1}: (C - C_<=-1).g + gT T_n
            } else {
                n = 0;
            }
        }
        float T = 1.0f;
        int k = 0;
        bool active = n > 0;
        BinRun bins;
        CellRun cells;
        // one sample: gradient of (cell, f); the next sample's gathers go to (ncell, nf)
        auto step = [&](const Cell &cell, const Gathered<VT, L> &f, Cell &ncell, Gathered<VT, L> &nf) {
            const bool more = k + 1 < n;
            if (more) {
                ncell = locate<LOG2B, L>(v, sample_pos(ray, k + 1, p.step));
                fetch_corners<VT, LOG2B, L>(v, ncell, nf);
            }
            const float val = interp_corners(cell, f);
            TfPos tp;
            float4 de;
            const float4 e = tf_lookup_l1(p, val, tp, de);
            const float a = e.w;
            const float cg = e.x * g.x + e.y * g.y + e.z * g.z;
            const float aT = a * T;
            R = fmaf(-aT, cg, R);                       // R_k = R_{k-1} - T_k a_k (c_k.g)
            const float om = 1.0f - a;
            // om is in (0, 1] where it divides: the fast reciprocal-based division is
            // within 2 ulp there
            const float da = T * cg - (om > 0.0f ? __fdividef(R, om) : 0.0f);
            if (aT != 0.0f || da != 0.0f) {
                const float4 dr = make_float4(aT * g.x, aT * g.y, aT * g.z, da);
                bins.add(row, tp.i0, 1.0f - tp.w, tp.w, dr);
                if (grad_vox && tp.interior) {
                    const float dv = (dr.x * de.x + dr.y * de.y + dr.z * de.z + dr.w * de.w) * vscale;
                    if (dv != 0.0f)
                        cells.add(grad_vox + ((long long)cell.z0 * nyx + (long long)cell.y0 * v.nx + cell.x0),
                                  cell.fx, cell.fy, cell.fz, dv, v.nx, nyx);
                }
            }
            T = fmaf(-a, T, T);
            ++k;
            if (!more) active = false;
        };
        Cell c0, c1;
        Gathered<VT, L> f0, f1;
        if (active) {
            c0 = locate<LOG2B, L>(v, sample_pos(ray, 0, p.step));
            fetch_corners<VT, LOG2B, L>(v, c0, f0);
        }
        for (;;) {      // two register sets in turn (no copy of the prefetched sample)
            if (!__any_sync(kFull, active)) break;
            if (active) step(c0, f0, c1, f1);
            if (!__any_sync(kFull, active)) break;
            if (active) step(c1, f1, c0, f0);
        }
        bins.flush(row);
        cells.flush(v.nx, nyx);
    }
}

// Final cross-block sum of the warps' FP32 rows, in FP64.
__global__ void __launch_bounds__(256) reduce_rows(const float *__restrict__ rows, int nrows, int n, double *out,
                                                    int chunk)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int r0 = blockIdx.y * chunk, r1 = min(r0 + chunk, nrows);
    double acc = 0.0;
    for (int r = r0; r < r1; ++r) acc += (double)rows[(size_t)r * n + q];
    atomicAdd(out + q, acc);
}

template <typename T, int LOG2B, int L>
static cudaError_t launch_bwd_t(const VolDev &v, vr_volume *vol, const CamDev &c, const ParamDev &p, const float4 *rgba,
                                const uint32_t *nsamples, const float4 *grad_rgba, double *grad_tf, float *grad_vox,
                                long long nvox, bool accumulate, unsigned *counter, cudaStream_t s)
{
    auto fn = bwd_kernel<T, LOG2B, L>;
    const int tiles_x = (c.W + 7) / 8, tiles_y = (c.H + 3) / 4;
    const unsigned ntiles = (unsigned)tiles_x * (unsigned)tiles_y;
    const int per_sm = occupancy_blocks((const void *)fn, kBwdThreads, 0);
    unsigned grid = (unsigned)(per_sm * sm_count());
    const unsigned max_useful = (ntiles + kBwdWarps - 1) / kBwdWarps;
    if (grid > max_useful) grid = max_useful;
    if (grid < 1) grid = 1;
    const int nrows = (int)grid * kBwdWarps;
    const size_t need = (size_t)nrows * 4 * (size_t)p.K;          // floats
    cudaError_t e = ensure_wtab(vol, need, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(vol->wtab, 0, need * sizeof(float), s);
    if (e != cudaSuccess) return e;
    if (!accumulate) {
        e = cudaMemsetAsync(grad_tf, 0, sizeof(double) * 4 * (size_t)p.K, s);
        if (e == cudaSuccess && grad_vox) e = cudaMemsetAsync(grad_vox, 0, sizeof(float) * (size_t)nvox, s);
        if (e != cudaSuccess) return e;
    }
    e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    fn<<<grid, kBwdThreads, 0, s>>>(v, c, p, rgba, nsamples, grad_rgba,
                                    reinterpret_cast<float4 *>(vol->wtab), grad_vox, counter, tiles_x, ntiles);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int n = 4 * p.K, chunk = 64;
    dim3 rgrid((unsigned)((n + 255) / 256), (unsigned)((nrows + chunk - 1) / chunk));
    reduce_rows<<<rgrid, 256, 0, s>>>(vol->wtab, nrows, n, grad_tf, chunk);
    return cudaGetLastError();
}

// Largest table the backward supports (the staged kernel keeps eight warps of
// bins in shared memory).
int backward_max_tf_size() { return (int)(200 * 1024 / (sizeof(float) * 4 * 8)); }

cudaError_t launch_backward(const VolDev &v, vr_volume *vol, const CamDev &c, const ParamDev &p, const float4 *rgba,
                            const uint32_t *nsamples, const float4 *grad_rgba, double *grad_tf, float *grad_vox,
                            long long nvox, bool accumulate, unsigned *counter, cudaStream_t s)
{
    return visit_layout(
        v, vol->store_dtype,
        [&](auto lay) {
            using Y = decltype(lay);
            return launch_bwd_t<typename Y::type, Y::log2b, Y::order>(v, vol, c, p, rgba, nsamples, grad_rgba,
                                                                       grad_tf, grad_vox, nvox, accumulate, counter,
                                                                       s);
        },
        cudaErrorInvalidValue);
}

}  // namespace vr
