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
// The table gradient is accumulated per CTA in shared memory (FP32) and the
// CTA partials are summed across blocks in FP64; the voxel gradient is
// scattered with float atomics into the dense layout.
#include "vr_device.cuh"

namespace vr {

constexpr int kBwdThreads = 256;   // one CTA renders a 16x16 pixel tile (8 warps of 8x4)

template <typename VT, int LOG2B>
__global__ void __launch_bounds__(kBwdThreads) bwd_kernel(VolDev v, CamDev c, ParamDev p,
                                                           const float4 *__restrict__ rgba,
                                                           const uint32_t *__restrict__ nsamples,
                                                           const float4 *__restrict__ grad_rgba,
                                                           float *__restrict__ partials, float *grad_vox,
                                                           int tiles_x16)
{
    extern __shared__ float4 smem[];
    float4 *tfs = smem;
    float *gtf = reinterpret_cast<float *>(smem + p.K);
    load_tf_shared(tfs, p.tf, p.K);
    for (int q = threadIdx.x; q < 4 * p.K; q += blockDim.x) gtf[q] = 0.0f;
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = (int)(blockIdx.x % tiles_x16) * 16 + (warp & 1) * 8 + (lane & 7);
    const int j = (int)(blockIdx.x / tiles_x16) * 16 + (warp >> 1) * 4 + (lane >> 3);
    const bool inside = i < c.W && j < c.H;
    Ray ray;
    int n = 0;
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    float Tn = 1.0f, R = 0.0f;
    if (inside) {
        const long long px = (long long)j * c.W + i;
        n = (int)nsamples[px];
        if (n > 0 && setup_ray(c, v.nx, v.ny, v.nz, p.step, i, j, ray)) {
            n = min(n, ray.n);
            const float4 out = rgba[px];
            g = grad_rgba[px];
            Tn = (1.0f - out.w) / (1.0f - p.bg.w);
            const float Cg = (out.x - Tn * p.bg.x) * g.x + (out.y - Tn * p.bg.y) * g.y + (out.z - Tn * p.bg.z) * g.z;
            const float gT = g.x * p.bg.x + g.y * p.bg.y + g.z * p.bg.z - g.w * (1.0f - p.bg.w);
            R = Cg + gT * Tn;            // R_{-1}: (C - C_<=-1).g + gT T_n
        } else {
            n = 0;
        }
    }
    const float vscale = p.km1 * p.scale01;    // du/dv inside the range
    const int nyx = v.ny * v.nx;
    float T = 1.0f;
    int k = 0;
    bool active = n > 0;
    while (__any_sync(kFull, active)) {
        if (active) {
            const float3 pos = sample_pos(ray, k, p.step);
            const Cell cell = locate<LOG2B>(v, pos);
            const float val = trilinear<VT, LOG2B>(v, cell);
            TfPos tp;
            const float4 e = tf_lookup(tfs, p, val, tp);
            const float a = e.w;
            const float cg = e.x * g.x + e.y * g.y + e.z * g.z;
            const float aT = a * T;
            R = fmaf(-aT, cg, R);                       // R_k = R_{k-1} - T_k a_k (c_k.g)
            const float om = 1.0f - a;
            const float da = T * cg - (om > 0.0f ? R / om : 0.0f);
            const float4 dr = make_float4(aT * g.x, aT * g.y, aT * g.z, da);
            const float w1 = tp.w, w0 = 1.0f - tp.w;
            float *g0 = gtf + 4 * tp.i0;
            if (aT != 0.0f) {
                atomicAdd(g0 + 0, w0 * dr.x); atomicAdd(g0 + 4, w1 * dr.x);
                atomicAdd(g0 + 1, w0 * dr.y); atomicAdd(g0 + 5, w1 * dr.y);
                atomicAdd(g0 + 2, w0 * dr.z); atomicAdd(g0 + 6, w1 * dr.z);
            }
            if (da != 0.0f) { atomicAdd(g0 + 3, w0 * da); atomicAdd(g0 + 7, w1 * da); }
            if (grad_vox && tp.interior) {
                const float4 e0 = tfs[tp.i0], e1 = tfs[tp.i0 + 1];
                const float dv = (dr.x * (e1.x - e0.x) + dr.y * (e1.y - e0.y) + dr.z * (e1.z - e0.z) +
                                  dr.w * (e1.w - e0.w)) * vscale;
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
            if (k >= n) active = false;
        }
    }
    __syncthreads();
    float *dst = partials + (long long)blockIdx.x * 4 * p.K;
    for (int q = threadIdx.x; q < 4 * p.K; q += blockDim.x) dst[q] = gtf[q];
}

// Final cross-block sum of the table-gradient partials, in FP64.
__global__ void __launch_bounds__(256) reduce_partials(const float *__restrict__ partials, int nblocks, int n,
                                                        double *out, int chunk)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int b0 = blockIdx.y * chunk, b1 = min(b0 + chunk, nblocks);
    double acc = 0.0;
    for (int b = b0; b < b1; ++b) acc += (double)partials[(long long)b * n + q];
    atomicAdd(out + q, acc);
}

int backward_blocks(const CamDev &c)
{
    return ((c.W + 15) / 16) * ((c.H + 15) / 16);
}

template <typename T, int LOG2B>
static cudaError_t launch_bwd_t(const VolDev &v, const CamDev &c, const ParamDev &p, const float4 *rgba,
                                const uint32_t *nsamples, const float4 *grad_rgba, float *partials, int nblocks,
                                double *grad_tf, float *grad_vox, long long nvox, bool accumulate, cudaStream_t s)
{
    const size_t smem = sizeof(float4) * (size_t)p.K * 2;
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
    fn<<<nblocks, kBwdThreads, smem, s>>>(v, c, p, rgba, nsamples, grad_rgba, partials, grad_vox,
                                          (c.W + 15) / 16);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int n = 4 * p.K;
    const int chunk = 64;
    dim3 grid((unsigned)((n + 255) / 256), (unsigned)((nblocks + chunk - 1) / chunk));
    reduce_partials<<<grid, 256, 0, s>>>(partials, nblocks, n, grad_tf, chunk);
    return cudaGetLastError();
}

cudaError_t launch_backward(const VolDev &v, vr_dtype dt, const CamDev &c, const ParamDev &p,
                            const float4 *rgba, const uint32_t *nsamples, const float4 *grad_rgba,
                            float *partials, int nblocks, double *grad_tf, float *grad_vox, long long nvox,
                            bool accumulate, cudaStream_t s)
{
#define VR_BWD_CASE(TT, LB) \
    return launch_bwd_t<TT, LB>(v, c, p, rgba, nsamples, grad_rgba, partials, nblocks, grad_tf, grad_vox, nvox, \
                                accumulate, s)
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
