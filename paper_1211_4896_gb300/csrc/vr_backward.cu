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
// with two fire-and-forget 16-byte vector reductions.  Samples of zero
// opacity (a = 0: no colour gradient, only the two opacity bins change) whose
// bins lie in the table's longest run of zero-opacity entries -- where
// transfer functions put the noise floor -- go instead to lane-private
// columns of 32 opacity bins in shared memory (plain loads and stores, no
// conflicts), summed into the warp's row when it has no tiles left.  One
// final kernel sums the warps' rows in FP64 (the only FP64 arithmetic: the
// cross-block sum).  The table itself is copied into shared memory when the
// kernel starts, so its two entries per sample do not wait behind the
// volume gathers in the L1/texture pipeline.
// The voxel gradient is scattered with reductions.  A ray's pending sums for
// the eight corners of its current cell are kept as two planes of four
// corners across the carry axis (the view's dominant axis); when the ray
// steps to the next cell along that axis the shared plane is carried in
// registers instead of being written, so a straight run writes one plane per
// cell.  A plane goes either into the dense gradient (x-neighbour pairs as
// 8-byte reductions when aligned) or, where many samples fall in each voxel,
// into a quad scratch holding per voxel position the plane's four corners as
// one float4 (one 16-byte reduction per plane); a gather pass then adds the
// four quads that hold each voxel into the dense gradient.
#include "vr_device.cuh"

namespace vr {

// Four warps per CTA: at 90 registers five CTAs (20 warps) fit an SM, where
// eight-warp CTAs fit two (16 warps); measured 6% faster on the 512^3
// four-view workload.
constexpr int kBwdThreads = 128;
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

// A ray's pending table-gradient contributions: bins b and b+1 of this
// thread's row.  A sample adds w0 dr to bin i0 and w1 dr to bin i0+1, with
// dr = (aT g.rgb, da); g is the ray's own, so the colour part is kept as the
// scalar sum of w aT and multiplied by g when the bin is written.
// Consecutive samples whose bin pair coincides or overlaps are added here and
// reach memory once.
struct BinRun {
    int b = -1;
    float s0 = 0.f, d0 = 0.f, s1 = 0.f, d1 = 0.f;     // bin b: (s0 g.rgb, d0); bin b+1: (s1 g.rgb, d1)
    __device__ __forceinline__ static void put(float4 *row, int bin, float sc, float d, const float4 &g)
    {
        red_add_v4(row + bin, make_float4(sc * g.x, sc * g.y, sc * g.z, d));
    }
    __device__ __forceinline__ void add(float4 *row, int i0, float w0, float w1, float aT, float da, const float4 &g)
    {
        if (i0 == b) {
            s0 = fmaf(w0, aT, s0);
            d0 = fmaf(w0, da, d0);
            s1 = fmaf(w1, aT, s1);
            d1 = fmaf(w1, da, d1);
            return;
        }
        if (i0 == b + 1) {                 // new lower bin == pending upper bin
            put(row, b, s0, d0, g);
            s0 = fmaf(w0, aT, s1);
            d0 = fmaf(w0, da, d1);
        } else if (i0 + 1 == b) {          // new upper bin == pending lower bin
            put(row, b + 1, s1, d1, g);
            s1 = fmaf(w1, aT, s0);
            d1 = fmaf(w1, da, d0);
            s0 = w0 * aT;
            d0 = w0 * da;
            b = i0;
            return;
        } else {
            flush(row, g);
            s0 = w0 * aT;
            d0 = w0 * da;
        }
        s1 = w1 * aT;
        d1 = w1 * da;
        b = i0;
    }
    __device__ __forceinline__ void flush(float4 *row, const float4 &g)
    {
        if (b >= 0) {
            put(row, b, s0, d0, g);
            put(row, b + 1, s1, d1, g);
        }
        b = -1;
    }
};

// Lane-private opacity bins for zero-opacity samples: kWin bins [lo, lo +
// kWin) over the table's longest run of zero-opacity entries; bin lo + q of
// lane l is col[q * 32] with col = window + l (bank l: no conflicts).
constexpr int kWin = 32;
struct OpacityWindow {
    float *col;
    int lo;
    // Adds w0 da to bin i0 and w1 da to bin i0 + 1 when both are in the window.
    __device__ __forceinline__ bool add(int i0, float w0, float w1, float da) const
    {
        const int q = i0 - lo;
        if ((unsigned)q >= (unsigned)(kWin - 1)) return false;
        col[q * 32] += w0 * da;
        col[(q + 1) * 32] += w1 * da;
        return true;
    }
};

// First entry of the longest run of table entries with zero opacity (kWin
// entries from there, moved down to fit the table), or a value that puts
// every bin outside the window when no two neighbouring entries have zero
// opacity.  Called by one whole warp.
__device__ int zero_opacity_window(const ParamDev &p, int lane)
{
    int run = 0, best = 0, best_lo = 0;
    for (int base = 0; base < p.K; base += 32) {
        const int q = base + lane;
        const unsigned m = __ballot_sync(kFull, q < p.K && __ldg(&p.tf[q].w) == 0.0f);
        for (int b = 0; b < 32 && base + b < p.K; ++b) {
            if ((m >> b) & 1u) {
                if (++run > best) best = run, best_lo = base + b - run + 1;
            } else {
                run = 0;
            }
        }
    }
    if (best < 2) return -2 * kWin;
    return max(0, min(best_lo, p.K - kWin));
}

// Where the voxel gradient goes.  Axes u, v, w: w is the carry axis, u and
// v the other two in x, y, z order; su, sv, sw their strides in the dense
// layout.  quad (or NULL): the scratch, quad[i] = the corners i, i + su,
// i + sv, i + su + sv of one plane.
struct GradDev {
    float *vox;
    float4 *quad;
    long long su, sv, sw;
    int axis;
    long long n;              // voxels (the bounds-check build tests indices against it)
    unsigned *status;
};

// A ray's pending voxel-gradient sums for the cell whose corner (x0, y0, z0)
// has dense index idx: plane p0 at w0 and p1 at w0 + 1, each in corner order
// (u, v) = (0, 0), (1, 0), (0, 1), (1, 1).
struct CellRun {
    long long idx = -1;
    float p0[4], p1[4];
    __device__ __forceinline__ void add(const GradDev &g, long long cell, float fu, float fv, float fw, float dv)
    {
        if (cell != idx) {
            if (idx >= 0 && cell == idx + g.sw) {            // step +1 along w: p1 becomes the new p0
                plane(g, idx, p0);
#pragma unroll
                for (int q = 0; q < 4; ++q) p0[q] = p1[q], p1[q] = 0.0f;
            } else if (idx >= 0 && cell == idx - g.sw) {     // step -1 along w: p0 becomes the new p1
                plane(g, idx + g.sw, p1);
#pragma unroll
                for (int q = 0; q < 4; ++q) p1[q] = p0[q], p0[q] = 0.0f;
            } else {
                flush(g);
#pragma unroll
                for (int q = 0; q < 4; ++q) p0[q] = 0.0f, p1[q] = 0.0f;
            }
            idx = cell;
        }
        const float wu0 = 1.0f - fu, wv0 = 1.0f - fv;
        const float d0 = (1.0f - fw) * dv, d1 = fw * dv;
        const float c[4] = {wu0 * wv0, fu * wv0, wu0 * fv, fu * fv};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            p0[q] = fmaf(c[q], d0, p0[q]);
            p1[q] = fmaf(c[q], d1, p1[q]);
        }
    }
    __device__ __forceinline__ static void plane(const GradDev &g, long long base, const float (&p)[4])
    {
        if constexpr (kBoundsCheck) {
            if (!index_ok(g.status, base, g.n) || !index_ok(g.status, base + (g.quad ? 0 : g.su + g.sv), g.n))
                return;
        }
        if (g.quad) {
            red_add_v4(g.quad + base, make_float4(p[0], p[1], p[2], p[3]));
        } else if (g.su == 1) {                               // (0,0)-(1,0) and (0,1)-(1,1) are x-neighbours
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float *b = g.vox + base + (h ? g.sv : 0);
                if ((reinterpret_cast<uintptr_t>(b) & 7u) == 0) {
                    red_add_v2(b, p[2 * h], p[2 * h + 1]);
                } else {
                    red_add_f32(b, p[2 * h]);
                    red_add_f32(b + 1, p[2 * h + 1]);
                }
            }
        } else {
            red_add_f32(g.vox + base, p[0]);
            red_add_f32(g.vox + base + g.su, p[1]);
            red_add_f32(g.vox + base + g.sv, p[2]);
            red_add_f32(g.vox + base + g.su + g.sv, p[3]);
        }
    }
    __device__ __forceinline__ void flush(const GradDev &g)
    {
        if (idx < 0) return;
        plane(g, idx, p0);
        plane(g, idx + g.sw, p1);
        idx = -1;
    }
};

// Resident CTAs the register budget is sized for: six for the texture layers
// (80 registers, a few spilled, against 90 at five: the eight 1080p views of
// the 1024^3 cube 2.82 against 3.10 ms per view; the layers' gathers need no
// brick addressing, so they keep fewer values live); the compiler's choice
// otherwise (six CTAs measured slower for the bricks).
template <typename T> struct BwdMinBlocks { static constexpr int value = 0; };   // 0: no minimum
template <> struct BwdMinBlocks<TexLayers<float>> { static constexpr int value = 6; };

template <typename VT, int LOG2B, int L>
__global__ void __launch_bounds__(kBwdThreads, BwdMinBlocks<VT>::value) bwd_kernel(VolDev v, CamDev c, ParamDev p,
                                                           const float4 *__restrict__ rgba,
                                                           const uint32_t *__restrict__ nsamples,
                                                           const float4 *__restrict__ grad_rgba, float4 *wtab,
                                                           GradDev gd, unsigned *counter, int tiles_x,
                                                           unsigned ntiles)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4 *row = wtab + ((size_t)blockIdx.x * kBwdWarps + warp) * (size_t)p.K;     // this warp's bins
    const float vscale = p.km1 * p.scale01;    // du/dv inside the range
    const long long nyx = (long long)v.ny * v.nx;
    __shared__ float window[kBwdWarps][kWin][32];
    __shared__ int window_lo;
    for (int q = threadIdx.x; q < kBwdWarps * kWin * 32; q += blockDim.x) (&window[0][0][0])[q] = 0.0f;
    if (warp == 0) {
        const int lo = zero_opacity_window(p, lane);
        if (lane == 0) window_lo = lo;
    }
    stage_tf(p);              // (its barrier also publishes the window)
    const OpacityWindow win{&window[warp][0][lane], window_lo};

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
                ncell = locate_t<VT, LOG2B, L, false>(v, sample_pos(ray, k + 1, p.step));
                fetch_corners<VT, LOG2B, L>(v, ncell, nf);
            }
            const float val = interp_corners(cell, f);
            TfPos tp;
            float4 de;
            const float4 e = tf_lookup_l1<true>(p, val, tp, de);
            const float a = e.w;
            const float cg = e.x * g.x + e.y * g.y + e.z * g.z;
            const float aT = a * T;
            R = fmaf(-aT, cg, R);                       // R_k = R_{k-1} - T_k a_k (c_k.g)
            const float om = 1.0f - a;
            // om is in (0, 1] where it divides: the fast reciprocal-based division is
            // within 2 ulp there
            const float da = T * cg - (om > 0.0f ? __fdividef(R, om) : 0.0f);
            bool bins_ok = true;                        // bins i0 and i0 + 1 exist
            if constexpr (kBoundsCheck) bins_ok = index_ok(v.status, tp.i0, p.K - 1);
            if (bins_ok && (aT != 0.0f || da != 0.0f)) {
                if (aT != 0.0f || !win.add(tp.i0, 1.0f - tp.w, tp.w, da))
                    bins.add(row, tp.i0, 1.0f - tp.w, tp.w, aT, da, g);
                if (gd.vox && tp.interior && (aT != 0.0f || de.w != 0.0f)) {
                    // dr . de with dr = (aT g.rgb, da); zero for a transparent sample
                    // between two zero-opacity entries
                    const float dv = fmaf(aT, de.x * g.x + de.y * g.y + de.z * g.z, da * de.w) * vscale;
                    if (dv != 0.0f) {
                        const float fu = gd.axis == 0 ? cell.fy : cell.fx;
                        const float fv = gd.axis == 2 ? cell.fy : cell.fz;
                        const float fw = gd.axis == 0 ? cell.fx : (gd.axis == 1 ? cell.fy : cell.fz);
                        cells.add(gd, (long long)cell.z0 * nyx + (long long)cell.y0 * v.nx + cell.x0, fu, fv, fw, dv);
                    }
                }
            }
            T = fmaf(-a, T, T);
            ++k;
            if (!more) active = false;
        };
        Cell c0, c1;
        Gathered<VT, L> f0, f1;
        if (active) {
            c0 = locate_t<VT, LOG2B, L, false>(v, sample_pos(ray, 0, p.step));
            fetch_corners<VT, LOG2B, L>(v, c0, f0);
        }
        for (;;) {      // two register sets in turn (no copy of the prefetched sample)
            if (!__any_sync(kFull, active)) break;
            if (active) step(c0, f0, c1, f1);
            if (!__any_sync(kFull, active)) break;
            if (active) step(c1, f1, c0, f0);
        }
        bins.flush(row, g);
        cells.flush(gd);
    }
    // the warp's opacity window into its row: lane l sums bin lo + l over the
    // 32 lanes' columns (skewed so that the lanes read distinct banks)
    __syncwarp();
    float sum = 0.0f;
#pragma unroll 8
    for (int j = 0; j < 32; ++j) sum += window[warp][lane][(j + lane) & 31];
    const int bin = window_lo + lane;
    if (sum != 0.0f && bin >= 0 && bin < p.K) red_add_f32(&row[bin].w, sum);
}

// Dense voxel gradient from the quad scratch: the voxel at (u, v) of its
// plane is corner (0, 0) of quad (u, v), (1, 0) of (u-1, v), (0, 1) of
// (u, v-1) and (1, 1) of (u-1, v-1).  Quads at u = nu-1 or v = nv-1 are never
// written and stay zero.  One CTA per (y, z) row.
__global__ void __launch_bounds__(256) quad_gather(const float4 *__restrict__ quad, float *grad_vox, int nx, int ny,
                                                    int axis, int accumulate)
{
    const unsigned row = blockIdx.x;                       // z * ny + y
    const int y = (int)(row % (unsigned)ny);
    const int z = (int)(row / (unsigned)ny);
    const long long base = (long long)row * nx, nyx = (long long)nx * ny;
    const long long su = axis == 0 ? nx : 1, sv = axis == 2 ? nx : nyx;
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
        const long long q = base + x;
        const bool u1 = (axis == 0 ? y : x) > 0, v1 = (axis == 2 ? y : z) > 0;
        float s = __ldg(&quad[q].x);
        if (u1) s += __ldg(&quad[q - su].y);
        if (v1) {
            s += __ldg(&quad[q - sv].z);
            if (u1) s += __ldg(&quad[q - su - sv].w);
        }
        grad_vox[q] = accumulate ? grad_vox[q] + s : s;
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

static GradDev grad_dev(const VolDev &v, float *grad_vox, float4 *grad_quad, int axis)
{
    const long long nx = v.nx, nyx = (long long)v.nx * v.ny;
    GradDev gd;
    gd.vox = grad_vox;
    gd.quad = grad_quad;
    gd.axis = axis;
    gd.su = axis == 0 ? nx : 1;
    gd.sv = axis == 2 ? nx : nyx;
    gd.sw = axis == 0 ? 1 : (axis == 1 ? nx : nyx);
    gd.n = nyx * v.nz;
    gd.status = v.status;
    return gd;
}

// Persistent grid of one view's backward kernel: the resident CTAs, but no
// more than its tiles need (smem: the staged table).
static unsigned view_grid(const void *fn, const CamDev &c, size_t smem)
{
    const unsigned ntiles = (unsigned)((c.W + 7) / 8) * (unsigned)((c.H + 3) / 4);
    unsigned grid = (unsigned)(occupancy_blocks(fn, kBwdThreads, smem) * sm_count());
    const unsigned max_useful = (ntiles + kBwdWarps - 1) / kBwdWarps;
    if (grid > max_useful) grid = max_useful;
    return grid < 1 ? 1 : grid;
}

static cudaError_t view_kernel(const BwdView &bv, vr_dtype dt, const void **fn_out)
{
    return visit_layout_tex(
        bv.v, dt,
        [&](auto lay) {
            using Y = decltype(lay);
            *fn_out = (const void *)bwd_kernel<typename Y::type, Y::log2b, Y::order>;
            return cudaSuccess;
        },
        cudaErrorInvalidValue);
}

// The two streams and three events with which a backward of several views
// overlaps each view's last tiles with the next view's first, created on
// first use (on the volume's device) and kept with the volume.
static cudaError_t ensure_aux_streams(vr_volume *vol)
{
    for (cudaStream_t &a : vol->aux)
        if (!a) {
            cudaError_t e = cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking);
            if (e != cudaSuccess) {
                a = nullptr;
                return e;
            }
        }
    for (cudaEvent_t &ev : vol->aux_ev)
        if (!ev) {
            cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e != cudaSuccess) {
                ev = nullptr;
                return e;
            }
        }
    return cudaSuccess;
}

// One view's backward kernel on stream s (its work counter cleared first).
static cudaError_t launch_view(const BwdView &bv, vr_dtype dt, const ParamDev &p, float4 *wtab, const GradDev &gd,
                               unsigned *counter, cudaStream_t s)
{
    const int tiles_x = (bv.c.W + 7) / 8;
    const unsigned ntiles = (unsigned)tiles_x * (unsigned)((bv.c.H + 3) / 4);
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    return visit_layout_tex(
        bv.v, dt,
        [&](auto lay) {
            using Y = decltype(lay);
            auto fn = bwd_kernel<typename Y::type, Y::log2b, Y::order>;
            const size_t smem = tf_shared_bytes(p);
            fn<<<view_grid((const void *)fn, bv.c, smem), kBwdThreads, smem, s>>>(bv.v, bv.c, p, bv.rgba, bv.nsamples,
                                                                        bv.grad_rgba, wtab, gd, counter, tiles_x,
                                                                        ntiles);
            return cudaGetLastError();
        },
        cudaErrorInvalidValue);
}

// The backward of a loss summed over n views: every view's kernel adds into
// the same per-warp table rows and voxel gradient (all reductions), then one
// FP64 row sum and (with the quad scratch) one gather finish all of them.
// With several views the kernels alternate between two streams forked from
// s, each with its own work counter: a view's grid holds every resident CTA
// slot, so the next view's CTAs take the slots its first CTAs to run out of
// tiles leave, instead of waiting for its last one.
cudaError_t launch_backward(vr_volume *vol, const BwdView *views, int n, const ParamDev &p, double *grad_tf,
                            float *grad_vox, float4 *grad_quad, int quad_axis, long long nvox, bool accumulate,
                            unsigned *counter, cudaStream_t s)
{
    const vr_dtype dt = vol->store_dtype;
    unsigned max_grid = 1;
    for (int q = 0; q < n; ++q) {
        const void *fn = nullptr;
        cudaError_t e = view_kernel(views[q], dt, &fn);
        if (e != cudaSuccess) return e;
        const unsigned g = view_grid(fn, views[q].c, tf_shared_bytes(p));
        if (g > max_grid) max_grid = g;
    }
    const int nrows = (int)max_grid * kBwdWarps;
    const size_t need = (size_t)nrows * 4 * (size_t)p.K;          // floats
    cudaError_t e = ensure_wtab(vol, need, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(vol->wtab, 0, need * sizeof(float), s);
    if (e != cudaSuccess) return e;
    if (!grad_vox) grad_quad = nullptr;
    if (!accumulate) {
        e = cudaMemsetAsync(grad_tf, 0, sizeof(double) * 4 * (size_t)p.K, s);
        if (e == cudaSuccess && grad_vox && !grad_quad)
            e = cudaMemsetAsync(grad_vox, 0, sizeof(float) * (size_t)nvox, s);
        if (e != cudaSuccess) return e;
    }
    if (grad_quad) {
        e = cudaMemsetAsync(grad_quad, 0, sizeof(float4) * (size_t)nvox, s);
        if (e != cudaSuccess) return e;
    }
    float4 *wtab = reinterpret_cast<float4 *>(vol->wtab);
    // direct reductions carry along each view's own axis; the quads have one
    // orientation for the whole call
    auto view_gd = [&](const BwdView &bv) {
        return grad_dev(bv.v, grad_vox, grad_quad, grad_quad ? quad_axis : bv.carry_axis);
    };
    if (n == 1) {
        e = launch_view(views[0], dt, p, wtab, view_gd(views[0]), counter, s);
    } else {
        unsigned *counter2 = nullptr;
        next_counter(vol, &counter2);
        e = ensure_aux_streams(vol);
        if (e != cudaSuccess) return e;
        e = cudaEventRecord(vol->aux_ev[0], s);
        if (e != cudaSuccess) return e;
        for (cudaStream_t a : vol->aux) {
            e = cudaStreamWaitEvent(a, vol->aux_ev[0], 0);
            if (e != cudaSuccess) return e;
        }
        for (int q = 0; q < n && e == cudaSuccess; ++q)
            e = launch_view(views[q], dt, p, wtab, view_gd(views[q]), (q & 1) ? counter2 : counter, vol->aux[q & 1]);
        // join both streams back into s, also after a failed launch
        for (int k = 0; k < 2; ++k) {
            cudaError_t j = cudaEventRecord(vol->aux_ev[1 + k], vol->aux[k]);
            if (j == cudaSuccess) j = cudaStreamWaitEvent(s, vol->aux_ev[1 + k], 0);
            if (e == cudaSuccess) e = j;
        }
    }
    if (e != cudaSuccess) return e;
    const int nb = 4 * p.K, chunk = 64;
    dim3 rgrid((unsigned)((nb + 255) / 256), (unsigned)((nrows + chunk - 1) / chunk));
    reduce_rows<<<rgrid, 256, 0, s>>>(vol->wtab, nrows, nb, grad_tf, chunk);
    e = cudaGetLastError();
    if (e != cudaSuccess || !grad_quad) return e;
    const VolDev &v = views[0].v;
    const unsigned rows = (unsigned)((long long)v.ny * v.nz);
    const unsigned threads = v.nx >= 256 ? 256u : (unsigned)((v.nx + 31) / 32 * 32);
    quad_gather<<<rows, threads, 0, s>>>(grad_quad, grad_vox, v.nx, v.ny, quad_axis, accumulate ? 1 : 0);
    return cudaGetLastError();
}

// Largest table the backward supports (the staged kernel keeps eight warps of
// bins in shared memory).
int backward_max_tf_size() { return (int)(200 * 1024 / (sizeof(float) * 4 * 8)); }

}  // namespace vr
