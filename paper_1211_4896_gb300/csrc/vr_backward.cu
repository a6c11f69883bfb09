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
// forward.  Each warp accumulates its tile's table gradient in private FP32
// bins in shared memory, then adds the non-zero bins into the FP64 output
// with FP64 atomics (the only FP64 arithmetic: the final cross-block sum).
// The voxel gradient is scattered with float atomics into the dense layout.
#include "vr_device.cuh"

namespace vr {

constexpr int kBwdThreads = 256;
constexpr int kBwdWarps = kBwdThreads / 32;

template <typename VT, int LOG2B>
__global__ void __launch_bounds__(kBwdThreads) bwd_kernel(VolDev v, CamDev c, ParamDev p,
                                                           const float4 *__restrict__ rgba,
                                                           const uint32_t *__restrict__ nsamples,
                                                           const float4 *__restrict__ grad_rgba, double *grad_tf,
                                                           float *grad_vox, unsigned *counter, int tiles_x,
                                                           unsigned ntiles)
{
    extern __shared__ float sbins[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nb = 4 * p.K;
    float *bins = sbins + warp * nb;
    for (int q = lane; q < nb; q += 32) bins[q] = 0.0f;
    __syncwarp();
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
        // one sample: gradient of (cell, f); the next sample's gathers go to (ncell, nf)
        auto step = [&](const Cell &cell, const Corners &f, Cell &ncell, Corners &nf) {
                const bool more = k + 1 < n;
                if (more) {
                    ncell = locate<LOG2B>(v, sample_pos(ray, k + 1, p.step));
                    fetch_corners<VT, LOG2B>(v, ncell, nf);
                }
                const float val = interp_corners(cell, f);
                TfPos tp;
                const float4 e = tf_lookup_l1(p, val, tp);
                const float a = e.w;
                const float cg = e.x * g.x + e.y * g.y + e.z * g.z;
                const float aT = a * T;
                R = fmaf(-aT, cg, R);                       // R_k = R_{k-1} - T_k a_k (c_k.g)
                const float om = 1.0f - a;
                const float da = T * cg - (om > 0.0f ? R / om : 0.0f);
                const float w1 = tp.w, w0 = 1.0f - tp.w;
                float *g0 = bins + 4 * tp.i0;
                if (aT != 0.0f) {
                    atomicAdd(g0 + 0, w0 * aT * g.x); atomicAdd(g0 + 4, w1 * aT * g.x);
                    atomicAdd(g0 + 1, w0 * aT * g.y); atomicAdd(g0 + 5, w1 * aT * g.y);
                    atomicAdd(g0 + 2, w0 * aT * g.z); atomicAdd(g0 + 6, w1 * aT * g.z);
                }
                if (da != 0.0f) { atomicAdd(g0 + 3, w0 * da); atomicAdd(g0 + 7, w1 * da); }
                if (grad_vox && tp.interior) {
                    const float4 e0 = __ldg(p.tf + tp.i0), e1 = __ldg(p.tf + tp.i0 + 1);
                    const float dv = (aT * (g.x * (e1.x - e0.x) + g.y * (e1.y - e0.y) + g.z * (e1.z - e0.z)) +
                                      da * (e1.w - e0.w)) * vscale;
                    if (dv != 0.0f) {
                        float *gv = grad_vox + ((long long)cell.z0 * nyx + (long long)cell.y0 * v.nx + cell.x0);
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const long long off = ((q & 4) ? nyx : 0) + ((q & 2) ? v.nx : 0) + (q & 1);
                            atomicAdd(gv + off, corner_weight(cell, q) * dv);
                        }
                    }
                }
                T = fmaf(-a, T, T);
                ++k;
                if (!more) active = false;
        };
        Cell c0, c1;
        Corners f0, f1;
        if (active) {
            c0 = locate<LOG2B>(v, sample_pos(ray, 0, p.step));
            fetch_corners<VT, LOG2B>(v, c0, f0);
        }
        for (;;) {      // two register sets in turn (no copy of the prefetched sample)
            if (!__any_sync(kFull, active)) break;
            if (active) step(c0, f0, c1, f1);
            if (!__any_sync(kFull, active)) break;
            if (active) step(c1, f1, c0, f0);
        }
        // Final cross-block sum in FP64: this tile's FP32 partial bins go to
        // the output, and the bins restart from zero.
        __syncwarp();
        for (int q = lane; q < nb; q += 32) {
            const float x = bins[q];
            if (x != 0.0f) {
                atomicAdd(grad_tf + q, (double)x);
                bins[q] = 0.0f;
            }
        }
        __syncwarp();
    }
}

template <typename T, int LOG2B>
static cudaError_t launch_bwd_t(const VolDev &v, const CamDev &c, const ParamDev &p, const float4 *rgba,
                                const uint32_t *nsamples, const float4 *grad_rgba, double *grad_tf, float *grad_vox,
                                long long nvox, bool accumulate, unsigned *counter, cudaStream_t s)
{
    const size_t smem = sizeof(float) * 4 * (size_t)p.K * kBwdWarps;
    auto fn = bwd_kernel<T, LOG2B>;
    cudaError_t e;
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (!accumulate) {
        e = cudaMemsetAsync(grad_tf, 0, sizeof(double) * 4 * (size_t)p.K, s);
        if (e != cudaSuccess) return e;
        if (grad_vox) {
            e = cudaMemsetAsync(grad_vox, 0, sizeof(float) * (size_t)nvox, s);
            if (e != cudaSuccess) return e;
        }
    }
    const int tiles_x = (c.W + 7) / 8, tiles_y = (c.H + 3) / 4;
    const unsigned ntiles = (unsigned)tiles_x * (unsigned)tiles_y;
    const int per_sm = occupancy_blocks((const void *)fn, kBwdThreads, smem);
    unsigned grid = (unsigned)(per_sm * sm_count());
    const unsigned max_useful = (ntiles + kBwdWarps - 1) / kBwdWarps;
    if (grid > max_useful) grid = max_useful;
    if (grid < 1) grid = 1;
    e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    fn<<<grid, kBwdThreads, smem, s>>>(v, c, p, rgba, nsamples, grad_rgba, grad_tf, grad_vox, counter, tiles_x,
                                       ntiles);
    return cudaGetLastError();
}

// Largest table the backward supports: eight warps of private FP32 bins must
// fit in shared memory.
int backward_max_tf_size() { return (int)(200 * 1024 / (sizeof(float) * 4 * kBwdWarps)); }

cudaError_t launch_backward(const VolDev &v, vr_dtype dt, const CamDev &c, const ParamDev &p, const float4 *rgba,
                            const uint32_t *nsamples, const float4 *grad_rgba, double *grad_tf, float *grad_vox,
                            long long nvox, bool accumulate, unsigned *counter, cudaStream_t s)
{
#define VR_BWD_CASE(TT, LB) \
    return launch_bwd_t<TT, LB>(v, c, p, rgba, nsamples, grad_rgba, grad_tf, grad_vox, nvox, accumulate, counter, s)
#define VR_BWD_DT(TT)                      \
    switch (v.log2b) {                     \
    case 4: VR_BWD_CASE(TT, 4);            \
    case 5: VR_BWD_CASE(TT, 5);            \
    case 6: VR_BWD_CASE(TT, 6);            \
    default: return cudaErrorInvalidValue; \
    }
    switch (dt) {
    case VR_F32: VR_BWD_DT(float);
    case VR_F16: VR_BWD_DT(__half);
    case VR_BF16: VR_BWD_DT(__nv_bfloat16);
    }
    return cudaErrorInvalidValue;
#undef VR_BWD_DT
#undef VR_BWD_CASE
}

}  // namespace vr
