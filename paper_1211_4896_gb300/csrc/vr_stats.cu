// vr_stats.cu -- global statistics of the resident cube (Sections 4.1-4.3):
// count, mean, standard deviation, minimum and maximum; a histogram; the
// exact median.  Each is a streaming pass over the x-fastest bricks (every
// voxel counted once: an apron element is skipped unless it is the cube's
// last layer), so the passes run at HBM bandwidth.  NULL (NaN) voxels are
// left out.
//
// Mean and deviation follow the paper's mixed precision (Section 4.2): short
// runs of values are summed in FP32, the runs with compensated FP32 sums,
// the threads' totals in FP64, all about a shift (the first voxel) to keep
// the squares small.  (FP64 arithmetic is slow on this part, so it stays out
// of the per-voxel loop.)  The median is the value of
// rank (n + 1) / 2, found by a radix select on order-preserving 32-bit keys
// (three counting passes of 11, 11 and 10 bits, the selection on the device)
// instead of the paper's Torben bisection, which needs a pass per halving
// of the value range: the same rank, in three passes.
#include "vr_device.cuh"

#include <cmath>

namespace vr {

constexpr int kStatThreads = 256;

// 16-byte chunks of brick elements: four floats or eight 16-bit values.
template <typename T> struct Chunk {
    static constexpr int n = 16 / sizeof(T);
};

__device__ __forceinline__ void widen_chunk(const uint4 &c, float (&out)[4], float)
{
    out[0] = __uint_as_float(c.x), out[1] = __uint_as_float(c.y);
    out[2] = __uint_as_float(c.z), out[3] = __uint_as_float(c.w);
}
__device__ __forceinline__ void widen_chunk(const uint4 &c, float (&out)[8], __half)
{
    const unsigned w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w[q]));
        out[2 * q] = f.x, out[2 * q + 1] = f.y;
    }
}
__device__ __forceinline__ void widen_chunk(const uint4 &c, float (&out)[8], __nv_bfloat16)
{
    const unsigned w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w[q]));
        out[2 * q] = f.x, out[2 * q + 1] = f.y;
    }
}

// Calls f(value) for every non-NaN voxel of the bricks handed to this CTA
// (bricks blockIdx.x, blockIdx.x + gridDim.x, ...).  Threads stride over the
// brick in 16-byte chunks (coalesced) with four chunks in flight per thread;
// an element counts when it is a voxel of the cube and not an apron copy (the
// apron of the last brick of an axis holds the cube's last layer).
template <typename T, int LOG2B, typename F>
__device__ __forceinline__ void for_each_voxel(const VolDev &v, F &&f)
{
    constexpr int B = 1 << LOG2B, B1 = B + 1, V = Chunk<T>::n, U = 4;
    // brick indices fit 32 bits (the volume limits keep nbx*nby*nbz < 2^31): 32-bit
    // division instead of the much slower 64-bit one
    const unsigned nbx = (unsigned)v.nbx, nbxy = (unsigned)v.nbx * (unsigned)v.nby;
    const unsigned nbricks = nbxy * (unsigned)v.nbz;
    const int nchunks = (int)(v.stride / V);                // bricks are padded to 64 elements
    for (unsigned brick = blockIdx.x; brick < nbricks; brick += gridDim.x) {
        const unsigned bz_ = brick / nbxy, rem = brick - bz_ * nbxy, by_ = rem / nbx;
        const int bx = (int)(rem - by_ * nbx), by = (int)by_, bz = (int)bz_;
        const int ex = min(B1, v.nx - bx * B) - ((bx < v.nbx - 1) ? 1 : 0);
        const int ey = min(B1, v.ny - by * B) - ((by < v.nby - 1) ? 1 : 0);
        const int ez = min(B1, v.nz - bz * B) - ((bz < v.nbz - 1) ? 1 : 0);
        const int used = min(nchunks, (B1 * B1 * ez + V - 1) / V);
        const uint4 *b = reinterpret_cast<const uint4 *>(static_cast<const T *>(v.data) + (long long)brick * v.stride);
        for (int c0 = threadIdx.x; c0 < used; c0 += U * blockDim.x) {
            uint4 raw[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int c = c0 + u * blockDim.x;
                if (c < used) raw[u] = __ldg(b + c);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int c = c0 + u * blockDim.x;
                if (c >= used) break;
                float val[V];
                widen_chunk(raw[u], val, T());
                // element coordinates: decoded once per chunk, then stepped
                const int e0 = c * V;
                int lz = e0 / (B1 * B1), r = e0 - lz * (B1 * B1), ly = r / B1, lx = r - ly * B1;
#pragma unroll
                for (int q = 0; q < V; ++q) {
                    if (lz < ez && ly < ey && lx < ex && val[q] == val[q]) f(val[q]);
                    if (++lx == B1) {
                        lx = 0;
                        if (++ly == B1) {
                            ly = 0;
                            ++lz;
                        }
                    }
                }
            }
        }
    }
}

__device__ __forceinline__ double warp_sum(double x)
{
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

// ---------------------------------------------------------------------------
// Moments
// ---------------------------------------------------------------------------

struct MomentPartial {
    double n, s1, s2;
    float mn, mx;
};

// Compensated FP32 accumulation (Kahan): the running error of the sum is
// carried along, so per-thread totals keep about FP32 precision relative to
// the sum however many runs they add.
struct Kahan {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = x - c, t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

template <typename T, int LOG2B>
__global__ void __launch_bounds__(kStatThreads) moments_kernel(VolDev v, MomentPartial *part)
{
    // shift: the first voxel (every thread reads the same element), 0 if NULL
    const float s0 = to_f(static_cast<const T *>(v.data)[0]);
    const float shift = s0 == s0 ? s0 : 0.0f;
    unsigned long long cnt = 0;
    Kahan k1, k2;
    float r1 = 0.0f, r2 = 0.0f, mn = INFINITY, mx = -INFINITY;
    int run = 0;
    for_each_voxel<T, LOG2B>(v, [&](float a) {
        const float d = a - shift;
        r1 += d;
        r2 = fmaf(d, d, r2);
        mn = fminf(mn, a);
        mx = fmaxf(mx, a);
        if (++run == 16) {               // runs of 16 values in plain FP32, the runs compensated
            cnt += 16;
            k1.add(r1);
            k2.add(r2);
            r1 = r2 = 0.0f;
            run = 0;
        }
    });
    cnt += run;
    k1.add(r1);
    k2.add(r2);
    double n = warp_sum((double)cnt);
    double s1 = warp_sum((double)k1.s - (double)k1.c);
    double s2 = warp_sum((double)k2.s - (double)k2.c);
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(kFull, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
    }
    __shared__ MomentPartial w[kStatThreads / 32];
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) w[warp] = MomentPartial{n, s1, s2, mn, mx};
    __syncthreads();
    if (threadIdx.x == 0) {
        MomentPartial t = w[0];
        for (int q = 1; q < kStatThreads / 32; ++q) {
            t.n += w[q].n;
            t.s1 += w[q].s1;
            t.s2 += w[q].s2;
            t.mn = fminf(t.mn, w[q].mn);
            t.mx = fmaxf(t.mx, w[q].mx);
        }
        part[blockIdx.x] = t;
    }
}

template <typename T>
__global__ void moments_final(VolDev v, const MomentPartial *part, int nparts, double *out)
{
    if (threadIdx.x != 0) return;
    const float s0 = to_f(static_cast<const T *>(v.data)[0]);
    const double shift = s0 == s0 ? (double)s0 : 0.0;
    double n = 0.0, s1 = 0.0, s2 = 0.0;
    float mn = INFINITY, mx = -INFINITY;
    for (int q = 0; q < nparts; ++q) {         // fixed order: deterministic
        n += part[q].n;
        s1 += part[q].s1;
        s2 += part[q].s2;
        mn = fminf(mn, part[q].mn);
        mx = fmaxf(mx, part[q].mx);
    }
    const double m1 = n > 0.0 ? s1 / n : 0.0;
    out[0] = n;
    out[1] = n > 0.0 ? shift + m1 : NAN;
    out[2] = n > 0.0 ? sqrt(fmax(s2 / n - m1 * m1, 0.0)) : NAN;
    out[3] = n > 0.0 ? (double)mn : NAN;
    out[4] = n > 0.0 ? (double)mx : NAN;
}

// ---------------------------------------------------------------------------
// Histogram: per-CTA shared counters, added to the global counts at the end.
// Bin b of n covers [lo + b (hi - lo)/n, lo + (b+1) (hi - lo)/n), the top
// value hi in the last bin.  When `fast` (the host has bounded the FP32
// estimate's error below 0.02 bin widths) the bin is estimated in FP32 and
// decided again in FP64 only within `band` (4x that bound) of an edge;
// otherwise in FP64.
// ---------------------------------------------------------------------------

// With `copies` = 32 each lane of a warp counts into its own copy of the
// shared histogram (row stride nbins + 1, so equal bins of different lanes
// sit in different banks): lanes never contend on one counter.
template <typename T, int LOG2B>
__global__ void __launch_bounds__(kStatThreads) histogram_kernel(VolDev v, double lo, double hi, float flo_in,
                                                                   float fhi_in, int nbins, int fast, float band,
                                                                   int copies, unsigned long long *counts)
{
    extern __shared__ unsigned sh[];
    const int pitch = nbins + 1;
    for (int b = threadIdx.x; b < copies * pitch; b += blockDim.x) sh[b] = 0u;
    __syncthreads();
    unsigned *mine = sh + (copies > 1 ? (threadIdx.x & 31) * pitch : 0);
    const float flo = (float)lo, fscale = (float)((double)nbins / (hi - lo));
    const double range = hi - lo;          // the FP64 decision: (a - lo) / (hi - lo) * nbins, in this order
    for_each_voxel<T, LOG2B>(v, [&](float a) {
        // flo_in / fhi_in: the least float >= lo and the greatest float <= hi, so
        // the FP32 test equals the FP64 one for every float a
        if (!(a >= flo_in && a <= fhi_in)) return;
        int b;
        if (fast) {
            const float u = (a - flo) * fscale;
            b = (int)floorf(u);
            const float fr = u - floorf(u);
            if (fr < band || fr > 1.0f - band) b = (int)floor(((double)a - lo) / range * (double)nbins);
        } else {
            b = (int)floor(((double)a - lo) / range * (double)nbins);
        }
        b = min(max(b, 0), nbins - 1);
        atomicAdd(&mine[b], 1u);
    });
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        unsigned long long t = 0;
        for (int q = 0; q < copies; ++q) t += sh[q * pitch + b];
        if (t) atomicAdd(&counts[b], t);
    }
}

// ---------------------------------------------------------------------------
// Median: radix select on keys that order like the values.
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned order_key(float a)
{
    const unsigned u = __float_as_uint(a);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float key_value(unsigned k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

struct SelectState {
    unsigned prefix;           // key bits fixed so far (high bits)
    unsigned long long n;      // values counted (non-NaN)
    unsigned long long k;      // rank still to find among the values matching the prefix (1-based)
};

template <typename T, int LOG2B>
__global__ void __launch_bounds__(kStatThreads) digit_hist_kernel(VolDev v, int pass, const SelectState *st,
                                                                    unsigned long long *hist)
{
    __shared__ unsigned sh[2048];
    const int bits = pass == 2 ? 10 : 11, shift = pass == 0 ? 21 : (pass == 1 ? 10 : 0);
    const int nb = 1 << bits;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) sh[b] = 0u;
    __syncthreads();
    const int fixed = 32 - (shift + bits);                 // high bits already selected
    const unsigned prefix = pass == 0 ? 0u : st->prefix;
    for_each_voxel<T, LOG2B>(v, [&](float a) {
        const unsigned key = order_key(a);
        if (fixed > 0 && (key >> (32 - fixed)) != (prefix >> (32 - fixed))) return;
        atomicAdd(&sh[(key >> shift) & (unsigned)(nb - 1)], 1u);
    });
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        if (sh[b]) atomicAdd(&hist[b], (unsigned long long)sh[b]);
}

// One thread: picks the digit that holds rank k, narrows the prefix and the
// rank, clears the histogram for the next pass; after the last pass writes
// the median (NaN without values).
__global__ void select_digit_kernel(int pass, SelectState *st, unsigned long long *hist, double *median)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int bits = pass == 2 ? 10 : 11, shift = pass == 0 ? 21 : (pass == 1 ? 10 : 0);
    const int nb = 1 << bits;
    if (pass == 0) {
        unsigned long long n = 0;
        for (int b = 0; b < nb; ++b) n += hist[b];
        st->n = n;
        st->k = (n + 1) / 2;
        st->prefix = 0u;
    }
    if (st->n == 0) {
        for (int b = 0; b < nb; ++b) hist[b] = 0ull;
        if (pass == 2) *median = NAN;
        return;
    }
    unsigned long long below = 0;
    int d = nb - 1;
    for (int b = 0; b < nb; ++b) {
        if (below + hist[b] >= st->k) {
            d = b;
            break;
        }
        below += hist[b];
    }
    st->k -= below;
    st->prefix |= (unsigned)d << shift;
    for (int b = 0; b < nb; ++b) hist[b] = 0ull;
    if (pass == 2) *median = (double)key_value(st->prefix);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

static unsigned stat_grid(long long nbricks)
{
    const long long g = (long long)sm_count() * 8;
    return (unsigned)(nbricks < g ? (nbricks > 0 ? nbricks : 1) : g);
}

template <typename F>
static cudaError_t by_storage(const VolDev &v, vr_dtype dt, F &&f)
{
    // the x-fastest bricks: element type = storage type, order 0
    return visit_layout(
        v, dt,
        [&](auto lay) {
            using Y = decltype(lay);
            if constexpr (Y::order == 0 && !is_pair<typename Y::type>::value)
                return f(lay);
            else
                return cudaErrorInvalidValue;
        },
        cudaErrorInvalidValue);
}

size_t stats_scratch_bytes() { return sizeof(MomentPartial) * 152 * 8 * 4 + 2048 * 8 + 64; }

cudaError_t launch_moments(const VolDev &v, vr_dtype dt, void *scratch, double *out, cudaStream_t s)
{
    const unsigned grid = stat_grid((long long)v.nbx * v.nby * v.nbz);
    if ((size_t)grid * sizeof(MomentPartial) > sizeof(MomentPartial) * 152 * 8 * 4) return cudaErrorInvalidValue;
    MomentPartial *part = static_cast<MomentPartial *>(scratch);
    return by_storage(v, dt, [&](auto lay) {
        using Y = decltype(lay);
        moments_kernel<typename Y::type, Y::log2b><<<grid, kStatThreads, 0, s>>>(v, part);
        moments_final<typename Y::type><<<1, 32, 0, s>>>(v, part, (int)grid, out);
        return cudaGetLastError();
    });
}

cudaError_t launch_histogram(const VolDev &v, vr_dtype dt, double lo, double hi, int nbins,
                             unsigned long long *counts, cudaStream_t s)
{
    const unsigned grid = stat_grid((long long)v.nbx * v.nby * v.nbz);
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * (size_t)nbins, s);
    if (e != cudaSuccess) return e;
    const int copies = (size_t)32 * (nbins + 1) * sizeof(unsigned) <= 96 * 1024 ? 32 : 1;
    const size_t smem = sizeof(unsigned) * (size_t)copies * (nbins + 1);
    // FP32 estimate error in bins: rounding of lo and of a - lo (each within
    // one ulp of max(|lo|, |hi|)) times the scale, plus the scale's rounding
    const double m = std::fmax(std::fabs(lo), std::fabs(hi));
    const double ulp = m > 0.0 ? std::ldexp(1.0, std::ilogb(m) - 23) : 0.0;
    const double err = 2.0 * ulp * (double)nbins / (hi - lo) + 4.0 * 6e-8 * (double)nbins;   // bins
    const int fast = err <= 0.02 ? 1 : 0;
    const float band = (float)std::fmax(4.0 * err, 1e-3);       // decide again in FP64 this close to an edge
    float flo_in = (float)lo, fhi_in = (float)hi;
    if ((double)flo_in < lo) flo_in = std::nextafterf(flo_in, INFINITY);
    if ((double)fhi_in > hi) fhi_in = std::nextafterf(fhi_in, -INFINITY);
    return by_storage(v, dt, [&](auto lay) {
        using Y = decltype(lay);
        auto fn = histogram_kernel<typename Y::type, Y::log2b>;
        if (smem > 48 * 1024) {
            cudaError_t a = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (a != cudaSuccess) return a;
        }
        fn<<<grid, kStatThreads, smem, s>>>(v, lo, hi, flo_in, fhi_in, nbins, fast, band, copies, counts);
        return cudaGetLastError();
    });
}

cudaError_t launch_median(const VolDev &v, vr_dtype dt, void *scratch, double *median, cudaStream_t s)
{
    const unsigned grid = stat_grid((long long)v.nbx * v.nby * v.nbz);
    unsigned char *base = static_cast<unsigned char *>(scratch) + sizeof(MomentPartial) * 152 * 8 * 4;
    unsigned long long *hist = reinterpret_cast<unsigned long long *>(base);
    SelectState *st = reinterpret_cast<SelectState *>(base + 2048 * 8);
    cudaError_t e = cudaMemsetAsync(hist, 0, 2048 * 8, s);
    if (e != cudaSuccess) return e;
    return by_storage(v, dt, [&](auto lay) {
        using Y = decltype(lay);
        for (int pass = 0; pass < 3; ++pass) {
            digit_hist_kernel<typename Y::type, Y::log2b><<<grid, kStatThreads, 0, s>>>(v, pass, st, hist);
            select_digit_kernel<<<1, 32, 0, s>>>(pass, st, hist, median);
        }
        return cudaGetLastError();
    });
}

}  // namespace vr
