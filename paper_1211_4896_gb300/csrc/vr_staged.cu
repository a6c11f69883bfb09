// vr_staged.cu -- forward and adjoint ray casting with the volume staged in
// shared memory, slab by slab (same method as vr_forward.cu / vr_backward.cu:
// Sections 3.3-3.4 and 4.4 of Hassan et al. 2012).
//
// A CTA owns a 16x16 ray tile.  Its rays are marched together through slabs
// of cells along the tile's principal axis a (the axis along which the tile
// centre ray moves fastest); a sample belongs to the slab that holds its cell
// index along a, so slab after slab preserves every ray's front-to-back
// order.  For each slab the CTA copies into shared memory the box of voxels
// that the tile's rays can touch there -- bounded by the four corner rays,
// which are extreme for a pinhole or orthographic bundle crossing a plane --
// with 16-byte cp.async copies from a dense row-padded copy of the volume,
// double buffered so the next slab streams in while this one is composited.
// The eight trilinear corners then come from shared memory (bank-conflict
// cost, independent of the view direction) instead of scattered L1 lines.
// A sample whose cell lies outside the staged box (rounding at the box
// margin, an oversized box, an eye inside the slab) reads global memory, so
// the result never depends on the box.
#include "vr_device.cuh"

#include <climits>
#include <cstdlib>

namespace vr {

constexpr int kStThreads = 256;
constexpr int kStWarps = kStThreads / 32;
constexpr int kStTile = 16;            // 16 x 16 rays per CTA
constexpr int kStSlabMax = 8;          // cells per slab along a (halved until the box fits)

struct Box {
    int x0, y0, z0;    // first voxel of the box
    int lx, ly, lz;    // extent in voxels (lx a multiple of 8)
    int sp;            // shared-memory row pitch in elements
    int valid;
};

struct Slab {
    int lo, hi;        // cell range along a, inclusive
    int next;          // first cell of the following slab
    int last;          // 1 if this is the last slab of the tile
    Box box;
};

struct StageCtl {
    unsigned tile;
    int cmin, cmax;            // cell range along a over the tile's rays
    float cq[4][3], cd[4][3];  // corner rays (anchor, direction), voxel space
    float seye[4];             // ray parameter of the eye (perspective); -inf otherwise
    Slab slab[2];
};

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (the copy engine moves whole rows into shared
// memory and reports completion on an mbarrier) and bounded mbarrier waits.
// ---------------------------------------------------------------------------
constexpr unsigned kWaitSpins = 1u << 22;   // bound on one wait; a timeout sets the status word

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Waits for the phase of `bar` with the given parity; gives up after
// `spins` polls and records the timeout in *status.
__device__ __forceinline__ void mbar_wait(uint64_t *bar, unsigned parity, unsigned *status,
                                          unsigned spins = kWaitSpins)
{
    const unsigned a = smem_u32(bar);
    for (unsigned spin = 0; spin < spins; ++spin) {
        unsigned done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return;
    }
    atomicOr(status, kStatusTimeout);
}

// Failure-detection self-test: one thread waits, with the bounded wait of the
// staged kernels, on a barrier that expects one arrival that never comes; the
// wait gives up after `spins` polls and sets the status word.  Nothing faults
// and no copy is in flight.
__global__ void wait_selftest_kernel(unsigned *status, unsigned spins)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_wait(&bar, 0u, status, spins);
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_u32(&bar)) : "memory");
    }
}

// Failure-detection self-test of the bounds-check report: tests an index one
// past the end of an n-element range (nothing is accessed), so the volume's
// status word records a caught violation.
__global__ void bounds_selftest_kernel(unsigned *status)
{
    if (threadIdx.x == 0) index_ok(status, 1, 1);
}

cudaError_t launch_bounds_selftest(unsigned *status, cudaStream_t s)
{
    bounds_selftest_kernel<<<1, 32, 0, s>>>(status);
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(unsigned *status, cudaStream_t s)
{
    wait_selftest_kernel<<<1, 32, 0, s>>>(status, 256u);
    return cudaGetLastError();
}

__device__ __forceinline__ void bulk_copy(void *smem_dst, const void *gmem_src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 ::"r"(smem_u32(smem_dst)), "l"(gmem_src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

// Unclipped ray of pixel (i, j): anchor q, direction d (voxel space), and the
// ray parameter of the eye (perspective) -- the same arithmetic as setup_ray.
__device__ __forceinline__ void pixel_ray(const CamDev &c, int i, int j, float q[3], float d[3], float &seye)
{
    const float hi = (float)i - 0.5f * (float)(c.W - 1);
    const float hj = (float)j - 0.5f * (float)(c.H - 1);
    q[0] = fmaf(hi, c.qa.x, fmaf(hj, c.qb.x, c.q0.x));
    q[1] = fmaf(hi, c.qa.y, fmaf(hj, c.qb.y, c.q0.y));
    q[2] = fmaf(hi, c.qa.z, fmaf(hj, c.qb.z, c.q0.z));
    float3 w;
    if (c.persp) {
        w.x = fmaf(hi, c.wa.x, fmaf(hj, c.wb.x, c.wf.x));
        w.y = fmaf(hi, c.wa.y, fmaf(hj, c.wb.y, c.wf.y));
        w.z = fmaf(hi, c.wa.z, fmaf(hj, c.wb.z, c.wf.z));
        const float len = sqrtf(w.x * w.x + w.y * w.y + w.z * w.z);
        const float il = 1.0f / len;
        w.x *= il; w.y *= il; w.z *= il;
        seye = -c.dist * len;
    } else {
        w = c.wf;
        seye = -INFINITY;
    }
    d[0] = w.x * c.inv_sp.x;
    d[1] = w.y * c.inv_sp.y;
    d[2] = w.z * c.inv_sp.z;
}

__device__ __forceinline__ float comp(const float3 &v, int a) { return a == 0 ? v.x : (a == 1 ? v.y : v.z); }

// Cell of a sample in the dense grid (clamped origin, fractional offsets).
struct DCell {
    int x0, y0, z0;
    float fx, fy, fz;
};

__device__ __forceinline__ DCell locate_dense(const DenseDev &d, float3 p)
{
    DCell c;
    c.x0 = min(max(__float2int_rd(p.x), 0), d.nx - 2);
    c.y0 = min(max(__float2int_rd(p.y), 0), d.ny - 2);
    c.z0 = min(max(__float2int_rd(p.z), 0), d.nz - 2);
    c.fx = p.x - (float)c.x0;
    c.fy = p.y - (float)c.y0;
    c.fz = p.z - (float)c.z0;
    return c;
}

__device__ __forceinline__ int cell_axis(const DCell &c, int a) { return a == 0 ? c.x0 : (a == 1 ? c.y0 : c.z0); }

// The eight corners, from the staged box when the whole cell is inside it,
// else from the dense copy in global memory.
template <typename T>
__device__ __forceinline__ void fetch_staged(const DenseDev &d, const T *buf, const Box b, const DCell &c, Corners &f)
{
    const int lx = c.x0 - b.x0, ly = c.y0 - b.y0, lz = c.z0 - b.z0;
    if (b.valid && lx >= 0 && ly >= 0 && lz >= 0 && lx + 1 < b.lx && ly + 1 < b.ly && lz + 1 < b.lz) {
        const int ps = b.sp * b.ly;
        const T *s = buf + (lz * b.ly + ly) * b.sp + lx;
        f.v[0] = to_f(s[0]);
        f.v[1] = to_f(s[1]);
        f.v[2] = to_f(s[b.sp]);
        f.v[3] = to_f(s[b.sp + 1]);
        f.v[4] = to_f(s[ps]);
        f.v[5] = to_f(s[ps + 1]);
        f.v[6] = to_f(s[ps + b.sp]);
        f.v[7] = to_f(s[ps + b.sp + 1]);
    } else {
        const long long px = d.px, pxy = (long long)d.px * d.ny;
        const T *g = static_cast<const T *>(d.data) + ((long long)c.z0 * d.ny + c.y0) * px + c.x0;
        f.v[0] = ldv(g);
        f.v[1] = ldv(g + 1);
        f.v[2] = ldv(g + px);
        f.v[3] = ldv(g + px + 1);
        f.v[4] = ldv(g + pxy);
        f.v[5] = ldv(g + pxy + 1);
        f.v[6] = ldv(g + pxy + px);
        f.v[7] = ldv(g + pxy + px + 1);
    }
}

__device__ __forceinline__ float interp_dcell(const DCell &c, const Corners &f)
{
    const float c00 = fmaf(c.fx, f.v[1] - f.v[0], f.v[0]), c10 = fmaf(c.fx, f.v[3] - f.v[2], f.v[2]);
    const float c01 = fmaf(c.fx, f.v[5] - f.v[4], f.v[4]), c11 = fmaf(c.fx, f.v[7] - f.v[6], f.v[6]);
    const float c0 = fmaf(c.fy, c10 - c00, c00), c1 = fmaf(c.fy, c11 - c01, c01);
    return fmaf(c.fz, c1 - c0, c0);
}

// ---------------------------------------------------------------------------
// Slab planning (warp 0): lanes 0..7 intersect the four corner rays with the
// slab's two bounding planes; the box is the bounding box of those points,
// one voxel of margin on each side, clamped to the volume, x aligned to 16
// bytes.  Slab thickness starts at kStSlabMax cells and halves until the box
// fits.  Lane 0 publishes the slab and, for a staged box, arms the slot's
// mbarrier with the number of bytes the row copies will deliver.
// ---------------------------------------------------------------------------
template <typename T>
__device__ void plan_slab(StageCtl &ctl, uint64_t *bars, int slot, int start, int endc, int axis, int dir,
                          const DenseDev &d, int buf_bytes)
{
    const int lane = threadIdx.x & 31;
    const int b1 = axis == 0 ? 1 : 0, b2 = axis == 2 ? 1 : 2;    // lateral axes
    const int n1 = b1 == 0 ? d.nx : (b1 == 1 ? d.ny : d.nz);
    const int n2 = b2 == 1 ? d.ny : d.nz;
    Slab sl;
    bool done = false;
    for (int S = kStSlabMax; S >= 1 && !done; S >>= 1) {
        int lo, hi;
        if (dir > 0) { lo = start; hi = min(start + S - 1, endc); }
        else { hi = start; lo = max(start - S + 1, endc); }
        // lane r + 4*plane: corner r against plane lo (plane 0) or hi + 1 (plane 1)
        float mn1 = INFINITY, mx1 = -INFINITY, mn2 = INFINITY, mx2 = -INFINITY;
        int ok = 1;
        if (lane < 8) {
            const int r = lane & 3;
            const float P = (float)((lane >> 2) ? hi + 1 : lo);
            const float s = (P - ctl.cq[r][axis]) / ctl.cd[r][axis];
            ok = s >= ctl.seye[r];
            const float v1 = fmaf(s, ctl.cd[r][b1], ctl.cq[r][b1]);
            const float v2 = fmaf(s, ctl.cd[r][b2], ctl.cq[r][b2]);
            mn1 = mx1 = v1;
            mn2 = mx2 = v2;
            if (!(isfinite(v1) && isfinite(v2))) ok = 0;
        }
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            mn1 = fminf(mn1, __shfl_xor_sync(kFull, mn1, o));
            mx1 = fmaxf(mx1, __shfl_xor_sync(kFull, mx1, o));
            mn2 = fminf(mn2, __shfl_xor_sync(kFull, mn2, o));
            mx2 = fmaxf(mx2, __shfl_xor_sync(kFull, mx2, o));
            ok &= __shfl_xor_sync(kFull, ok, o);
        }
        // lanes 0..7 now hold the reduction; every lane takes lane 0's values
        // so the whole warp makes the same decisions below
        mn1 = __shfl_sync(kFull, mn1, 0);
        mx1 = __shfl_sync(kFull, mx1, 0);
        mn2 = __shfl_sync(kFull, mn2, 0);
        mx2 = __shfl_sync(kFull, mx2, 0);
        ok = __shfl_sync(kFull, ok, 0);
        // +-1 voxel margin for rounding, +1 for the upper trilinear corner
        const int l1 = (int)fminf(fmaxf(floorf(mn1) - 1.0f, 0.0f), (float)(n1 - 1));
        const int h1 = (int)fminf(fmaxf(floorf(mx1) + 2.0f, 0.0f), (float)(n1 - 1));
        const int l2 = (int)fminf(fmaxf(floorf(mn2) - 1.0f, 0.0f), (float)(n2 - 1));
        const int h2 = (int)fminf(fmaxf(floorf(mx2) + 2.0f, 0.0f), (float)(n2 - 1));
        // (axis, b1, b2) -> (x, y, z)
        int xl, xh, yl, yh, zl, zh;
        if (axis == 0) { xl = lo; xh = hi + 1; yl = l1; yh = h1; zl = l2; zh = h2; }
        else if (axis == 1) { xl = l1; xh = h1; yl = lo; yh = hi + 1; zl = l2; zh = h2; }
        else { xl = l1; xh = h1; yl = l2; yh = h2; zl = lo; zh = hi + 1; }
        constexpr int G = 16 / (int)sizeof(T);                    // elements per 16 bytes
        Box bx;
        bx.x0 = xl & ~(G - 1);
        bx.y0 = yl;
        bx.z0 = zl;
        bx.lx = ((xh - bx.x0 + 1) + G - 1) & ~(G - 1);
        bx.ly = yh - yl + 1;
        bx.lz = zh - zl + 1;
        int sp = bx.lx;
        if (((sp * (int)sizeof(T)) / 4) % 32 == 0) sp += G;      // rows not all on one bank
        bx.sp = sp;
        const long long bytes = (long long)sp * bx.ly * bx.lz * (long long)sizeof(T);
        bx.valid = ok && bx.ly > 0 && bx.lz > 0 && bytes <= buf_bytes;
        sl.lo = lo;
        sl.hi = hi;
        sl.next = dir > 0 ? hi + 1 : lo - 1;
        sl.last = dir > 0 ? (hi >= endc) : (lo <= endc);
        sl.box = bx;
        done = bx.valid || S == 1 || !ok;
    }
    if (lane == 0) {
        ctl.slab[slot] = sl;
        if (sl.box.valid) mbar_expect_tx(&bars[slot], (unsigned)(sl.box.lx * sl.box.ly * sl.box.lz * (int)sizeof(T)));
    }
}

// All threads issue the box's row copies (one bulk copy per x-row of the box).
template <typename T>
__device__ __forceinline__ void stage_box(const DenseDev &d, const Box &b, T *buf, uint64_t *bar)
{
    if (!b.valid) return;
    const int rows = b.ly * b.lz;
    const unsigned bytes = (unsigned)(b.lx * (int)sizeof(T));
    const T *src0 = static_cast<const T *>(d.data);
    // order this thread's earlier generic reads of the buffer before the copy engine's writes
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    for (int r = threadIdx.x; r < rows; r += kStThreads) {
        const int cz = r / b.ly, cy = r - cz * b.ly;
        bulk_copy(buf + (cz * b.ly + cy) * b.sp, src0 + ((long long)(b.z0 + cz) * d.ny + (b.y0 + cy)) * d.px + b.x0,
                  bytes, bar);
    }
}

// Marches the tile's rays slab by slab.  `step(cell, corners)` composites one
// sample and clears `active` when the ray ends.  Buffers alternate between the
// two slots; while slab s is marched the rows of slab s+1 are in flight.
template <typename T, typename Step>
__device__ __forceinline__ void run_slabs(StageCtl &ctl, uint64_t *bars, unsigned &parity, unsigned char *smem_raw,
                                          int buf_bytes, const DenseDev &d, const ParamDev &p, const Ray &ray, int &k,
                                          bool &active, int axis, int dir, unsigned *status, Step step)
{
    const int t = threadIdx.x;
    const int first = dir > 0 ? ctl.cmin : ctl.cmax, endc = dir > 0 ? ctl.cmax : ctl.cmin;
    auto bufp = [&](int slot) { return reinterpret_cast<T *>(smem_raw + (size_t)slot * buf_bytes); };
    if (t < 32) plan_slab<T>(ctl, bars, 0, first, endc, axis, dir, d, buf_bytes);
    __syncthreads();
    stage_box<T>(d, ctl.slab[0].box, bufp(0), &bars[0]);
    for (int s = 0;; ++s) {
        const int slot = s & 1;
        const Slab cur = ctl.slab[slot];
        if (!cur.last && t < 32) plan_slab<T>(ctl, bars, slot ^ 1, cur.next, endc, axis, dir, d, buf_bytes);
        __syncthreads();
        const Box nxt = ctl.slab[slot ^ 1].box;
        if (!cur.last) stage_box<T>(d, nxt, bufp(slot ^ 1), &bars[slot ^ 1]);
        if (cur.box.valid) {
            mbar_wait(&bars[slot], (parity >> slot) & 1u, status);
            parity ^= 1u << slot;
        }
        const T *buf = bufp(slot);
        while (active) {
            const DCell cell = locate_dense(d, sample_pos(ray, k, p.step));
            const int ca = cell_axis(cell, axis);
            if (dir > 0 ? ca > cur.hi : ca < cur.lo) break;      // belongs to a later slab
            Corners f;
            fetch_staged<T>(d, buf, cur.box, cell, f);
            step(cell, f);
        }
        const int any = __syncthreads_or(active);
        if (cur.last || !any) {
            if (!cur.last && nxt.valid) {          // the next slab's rows are in flight: let them land
                mbar_wait(&bars[slot ^ 1], (parity >> (slot ^ 1)) & 1u, status);
                parity ^= 1u << (slot ^ 1);
            }
            break;
        }
    }
}

// Per-tile set-up shared by both kernels: principal axis and direction from
// the tile centre ray, corner rays, and the cell range along the axis.
// Returns false when the tile must be marched without staging (some ray
// moves against the principal direction).
template <typename T>
__device__ __forceinline__ bool tile_setup(StageCtl &ctl, const DenseDev &d, const CamDev &c, const ParamDev &p,
                                           int tx0, int ty0, bool hit, const Ray &ray, int nsamp, int &axis,
                                           int &dir)
{
    const int t = threadIdx.x;
    {
        float q[3], dd[3], se;
        pixel_ray(c, min(tx0 + kStTile / 2, c.W - 1), min(ty0 + kStTile / 2, c.H - 1), q, dd, se);
        const float ax = fabsf(dd[0]), ay = fabsf(dd[1]), az = fabsf(dd[2]);
        axis = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
        dir = dd[axis] >= 0.0f ? 1 : -1;
    }
    bool ok = true;
    if (t < 4) {
        const int ci = min(tx0 + ((t & 1) ? kStTile - 1 : 0), c.W - 1);
        const int cj = min(ty0 + ((t & 2) ? kStTile - 1 : 0), c.H - 1);
        float q[3], dd[3], se;
        pixel_ray(c, ci, cj, q, dd, se);
        for (int a = 0; a < 3; ++a) { ctl.cq[t][a] = q[a]; ctl.cd[t][a] = dd[a]; }
        ctl.seye[t] = se;
        ok = dir > 0 ? dd[axis] > 0.0f : dd[axis] < 0.0f;
    }
    if (hit) {
        const float da = comp(ray.d, axis);
        ok = ok && (dir > 0 ? da > 0.0f : da < 0.0f);
        const int c0 = cell_axis(locate_dense(d, sample_pos(ray, 0, p.step)), axis);
        const int c1 = cell_axis(locate_dense(d, sample_pos(ray, nsamp - 1, p.step)), axis);
        atomicMin(&ctl.cmin, min(c0, c1));
        atomicMax(&ctl.cmax, max(c0, c1));
    }
    return __syncthreads_and(ok) != 0;
}

// ---------------------------------------------------------------------------
// Forward
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kStThreads, 2) staged_fwd_kernel(DenseDev d, CamDev c, ParamDev p, float4 *out,
                                                                 uint32_t *nsamples, unsigned *counter, int tiles_x,
                                                                 unsigned ntiles, int buf_bytes, unsigned *status)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ StageCtl ctl;
    __shared__ uint64_t bars[2];
    const int t = threadIdx.x;
    if (t == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    unsigned parity = 0;
    const Box nobox{0, 0, 0, 0, 0, 0, 0, 0};
    for (;;) {
        if (t == 0) {
            ctl.tile = atomicAdd(counter, 1u);
            ctl.cmin = INT_MAX;
            ctl.cmax = INT_MIN;
        }
        __syncthreads();
        const unsigned tile = ctl.tile;
        if (tile >= ntiles) break;
        const int tx0 = (int)(tile % tiles_x) * kStTile, ty0 = (int)(tile / tiles_x) * kStTile;
        const int i = tx0 + (t & (kStTile - 1)), j = ty0 + t / kStTile;
        const bool inside = i < c.W && j < c.H;
        Ray ray;
        const bool hit = inside && setup_ray(c, d.nx, d.ny, d.nz, p.step, i, j, ray);
        int axis, dir;
        const bool staged = tile_setup<T>(ctl, d, c, p, tx0, ty0, hit, ray, hit ? ray.n : 0, axis, dir);
        Composite acc{0.0f, 0.0f, 0.0f, 1.0f};
        int k = 0;
        bool active = hit;
        auto step = [&](const DCell &cell, const Corners &f) {
            const float val = interp_dcell(cell, f);
            TfPos tp;
            const float4 e = tf_lookup_l1(p, val, tp);
            const float aT = e.w * acc.T;
            acc.r = fmaf(aT, e.x, acc.r);
            acc.g = fmaf(aT, e.y, acc.g);
            acc.b = fmaf(aT, e.z, acc.b);
            acc.T = fmaf(-e.w, acc.T, acc.T);
            ++k;
            if (k >= ray.n || acc.T <= p.t_stop) active = false;
        };
        if (!staged) {
            while (active) {
                const DCell cell = locate_dense(d, sample_pos(ray, k, p.step));
                Corners f;
                fetch_staged<T>(d, nullptr, nobox, cell, f);
                step(cell, f);
            }
        } else if (ctl.cmin <= ctl.cmax) {
            run_slabs<T>(ctl, bars, parity, smem_raw, buf_bytes, d, p, ray, k, active, axis, dir, status, step);
        }
        if (inside) write_pixel(p, acc, hit ? k : 0, out, nsamples, (long long)j * c.W + i);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Backward (same adjoint as vr_backward.cu, on the staged march)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kStThreads, 2) staged_bwd_kernel(DenseDev d, CamDev c, ParamDev p,
                                                                 const float4 *__restrict__ rgba,
                                                                 const uint32_t *__restrict__ nsamples,
                                                                 const float4 *__restrict__ grad_rgba,
                                                                 double *grad_tf, float *grad_vox, unsigned *counter,
                                                                 int tiles_x, unsigned ntiles, int buf_bytes,
                                                                 unsigned *status)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ StageCtl ctl;
    __shared__ uint64_t bars[2];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int nb = 4 * p.K;
    float *bins = reinterpret_cast<float *>(smem_raw + 2 * (size_t)buf_bytes) + warp * nb;
    for (int q = lane; q < nb; q += 32) bins[q] = 0.0f;
    if (t == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    unsigned parity = 0;
    const Box nobox{0, 0, 0, 0, 0, 0, 0, 0};
    const float vscale = p.km1 * p.scale01;
    const long long nyx = (long long)d.ny * d.nx;
    for (;;) {
        if (t == 0) {
            ctl.tile = atomicAdd(counter, 1u);
            ctl.cmin = INT_MAX;
            ctl.cmax = INT_MIN;
        }
        __syncthreads();
        const unsigned tile = ctl.tile;
        if (tile >= ntiles) break;
        const int tx0 = (int)(tile % tiles_x) * kStTile, ty0 = (int)(tile / tiles_x) * kStTile;
        const int i = tx0 + (t & (kStTile - 1)), j = ty0 + t / kStTile;
        Ray ray;
        int n = 0;
        float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
        float R = 0.0f;
        if (i < c.W && j < c.H) {
            const long long px = (long long)j * c.W + i;
            n = (int)nsamples[px];
            if (n > 0 && setup_ray(c, d.nx, d.ny, d.nz, p.step, i, j, ray)) {
                n = min(n, ray.n);
                const float4 o = rgba[px];
                g = grad_rgba[px];
                const float Tn = (1.0f - o.w) / (1.0f - p.bg.w);
                const float Cg = (o.x - Tn * p.bg.x) * g.x + (o.y - Tn * p.bg.y) * g.y + (o.z - Tn * p.bg.z) * g.z;
                const float gT = g.x * p.bg.x + g.y * p.bg.y + g.z * p.bg.z - g.w * (1.0f - p.bg.w);
                R = Cg + gT * Tn;
            } else {
                n = 0;
            }
        }
        const bool hit = n > 0;
        int axis, dir;
        const bool staged = tile_setup<T>(ctl, d, c, p, tx0, ty0, hit, ray, n, axis, dir);
        float Tr = 1.0f;
        int k = 0;
        bool active = hit;
        auto step = [&](const DCell &cell, const Corners &f) {
            const float val = interp_dcell(cell, f);
            TfPos tp;
            const float4 e = tf_lookup_l1(p, val, tp);
            const float a = e.w;
            const float cg = e.x * g.x + e.y * g.y + e.z * g.z;
            const float aT = a * Tr;
            R = fmaf(-aT, cg, R);
            const float om = 1.0f - a;
            const float da = Tr * cg - (om > 0.0f ? R / om : 0.0f);
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
                    float *gv = grad_vox + ((long long)cell.z0 * nyx + (long long)cell.y0 * d.nx + cell.x0);
                    const float wx1 = cell.fx, wx0 = 1.0f - cell.fx, wy1 = cell.fy, wy0 = 1.0f - cell.fy;
                    const float wz1 = cell.fz, wz0 = 1.0f - cell.fz;
                    atomicAdd(gv, wx0 * wy0 * wz0 * dv);
                    atomicAdd(gv + 1, wx1 * wy0 * wz0 * dv);
                    atomicAdd(gv + d.nx, wx0 * wy1 * wz0 * dv);
                    atomicAdd(gv + d.nx + 1, wx1 * wy1 * wz0 * dv);
                    atomicAdd(gv + nyx, wx0 * wy0 * wz1 * dv);
                    atomicAdd(gv + nyx + 1, wx1 * wy0 * wz1 * dv);
                    atomicAdd(gv + nyx + d.nx, wx0 * wy1 * wz1 * dv);
                    atomicAdd(gv + nyx + d.nx + 1, wx1 * wy1 * wz1 * dv);
                }
            }
            Tr = fmaf(-a, Tr, Tr);
            ++k;
            if (k >= n) active = false;
        };
        if (!staged) {
            while (active) {
                const DCell cell = locate_dense(d, sample_pos(ray, k, p.step));
                Corners f;
                fetch_staged<T>(d, nullptr, nobox, cell, f);
                step(cell, f);
            }
        } else if (ctl.cmin <= ctl.cmax) {
            run_slabs<T>(ctl, bars, parity, smem_raw, buf_bytes, d, p, ray, k, active, axis, dir, status, step);
        }
        // this tile's FP32 bins -> FP64 output (the final cross-block sum)
        __syncwarp();
        for (int q = lane; q < nb; q += 32) {
            const float x = bins[q];
            if (x != 0.0f) {
                atomicAdd(grad_tf + q, (double)x);
                bins[q] = 0.0f;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Dense copy (row-padded) and launchers
// ---------------------------------------------------------------------------
template <typename S, typename D>
__global__ void __launch_bounds__(256) densify_kernel(const S *__restrict__ src, D *__restrict__ dst, int nx, int ny,
                                                       int px)
{
    const long long row = blockIdx.x;       // z * ny + y
    const S *s = src + row * nx;
    D *o = dst + row * px;
    for (int x = threadIdx.x; x < px; x += blockDim.x) o[x] = x < nx ? to_dtype<D>(to_f(s[x])) : to_dtype<D>(0.0f);
}

template <typename S>
static cudaError_t densify_src(const void *src, vr_volume *vol, cudaStream_t s)
{
    const long long rows = vol->dims[1] * vol->dims[2];
    const int nx = (int)vol->dims[0], ny = (int)vol->dims[1], px = vol->dense_px;
    const S *sp = static_cast<const S *>(src);
    for (long long r0 = 0; r0 < rows; r0 += 1ll << 30) {      // grid.x <= 2^31 - 1
        const long long nr = rows - r0 < (1ll << 30) ? rows - r0 : (1ll << 30);
        switch (vol->store_dtype) {
        case VR_F32:
            densify_kernel<S, float><<<(unsigned)nr, 256, 0, s>>>(sp + r0 * nx, static_cast<float *>(vol->dense) + r0 * px,
                                                                 nx, ny, px);
            break;
        case VR_F16:
            densify_kernel<S, __half><<<(unsigned)nr, 256, 0, s>>>(sp + r0 * nx, static_cast<__half *>(vol->dense) + r0 * px,
                                                                  nx, ny, px);
            break;
        case VR_BF16:
            densify_kernel<S, __nv_bfloat16><<<(unsigned)nr, 256, 0, s>>>(
                sp + r0 * nx, static_cast<__nv_bfloat16 *>(vol->dense) + r0 * px, nx, ny, px);
            break;
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_densify(const void *src, vr_dtype src_dtype, vr_volume *vol, cudaStream_t s)
{
    switch (src_dtype) {
    case VR_F32: return densify_src<float>(src, vol, s);
    case VR_F16: return densify_src<__half>(src, vol, s);
    case VR_BF16: return densify_src<__nv_bfloat16>(src, vol, s);
    }
    return cudaErrorInvalidValue;
}

// Dense copy rebuilt from the bricks (first staged call on a volume).
template <typename D>
__global__ void __launch_bounds__(256) dense_from_bricks_kernel(VolDev v, D *__restrict__ dst, int px)
{
    const int y = blockIdx.x % v.ny, z = blockIdx.x / v.ny;
    const int B = 1 << v.log2b, B1 = B + 1;
    const int by = min(y >> v.log2b, v.nby - 1), bz = min(z >> v.log2b, v.nbz - 1);
    const int ly = y - by * B, lz = z - bz * B;
    D *o = dst + ((long long)z * v.ny + y) * px;
    for (int x = threadIdx.x; x < px; x += blockDim.x) {
        if (x >= v.nx) { o[x] = to_dtype<D>(0.0f); continue; }
        const int bx = min(x >> v.log2b, v.nbx - 1), lx = x - bx * B;
        const long long brick = ((long long)bz * v.nby + by) * v.nbx + bx;
        o[x] = static_cast<const D *>(v.data)[brick * v.stride + ((long long)lz * B1 + ly) * B1 + lx];
    }
}

cudaError_t launch_dense_from_bricks(vr_volume *vol, cudaStream_t s)
{
    const VolDev v = vol_dev(vol);
    const unsigned rows = (unsigned)(vol->dims[1] * vol->dims[2]);
    switch (vol->store_dtype) {
    case VR_F32: dense_from_bricks_kernel<float><<<rows, 256, 0, s>>>(v, static_cast<float *>(vol->dense), vol->dense_px); break;
    case VR_F16: dense_from_bricks_kernel<__half><<<rows, 256, 0, s>>>(v, static_cast<__half *>(vol->dense), vol->dense_px); break;
    case VR_BF16:
        dense_from_bricks_kernel<__nv_bfloat16><<<rows, 256, 0, s>>>(v, static_cast<__nv_bfloat16 *>(vol->dense), vol->dense_px);
        break;
    }
    return cudaGetLastError();
}

DenseDev dense_dev(const vr_volume *vol)
{
    DenseDev d;
    d.data = vol->dense;
    d.nx = (int)vol->dims[0];
    d.ny = (int)vol->dims[1];
    d.nz = (int)vol->dims[2];
    d.px = vol->dense_px;
    return d;
}

static int env_int(const char *name, int dflt)
{
    const char *s = std::getenv(name);
    return s ? std::atoi(s) : dflt;
}

// Shared-memory budget per CTA: two slab buffers (+ the backward's bins).
// VR_STAGED_BUF_KB overrides the buffer size (a tuning knob).
static int staged_buf_bytes(size_t extra)
{
    static const int env_kb = env_int("VR_STAGED_BUF_KB", 0);
    if (env_kb > 0) return env_kb * 1024;
    // two CTAs per SM when they fit (227 KB per SM, 1 KB reserved per CTA)
    const long long per_cta = 113 * 1024 - 2048 - (long long)extra;
    int b = (int)(per_cta / 2) & ~127;
    if (b < 16 * 1024) b = (int)((225 * 1024 - (long long)extra - 2048) / 2) & ~127;      // one CTA per SM
    return b;
}

template <typename T>
static cudaError_t launch_fwd_staged_t(const DenseDev &d, const CamDev &c, const ParamDev &p, float4 *out,
                                       uint32_t *nsamples, unsigned *counter, unsigned *status, cudaStream_t s)
{
    const int tiles_x = (c.W + kStTile - 1) / kStTile, tiles_y = (c.H + kStTile - 1) / kStTile;
    const unsigned ntiles = (unsigned)tiles_x * (unsigned)tiles_y;
    const int buf = staged_buf_bytes(0);
    const size_t smem = 2 * (size_t)buf;
    auto fn = staged_fwd_kernel<T>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int per_sm = occupancy_blocks((const void *)fn, kStThreads, smem);
    unsigned grid = (unsigned)(per_sm * sm_count());
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    fn<<<grid, kStThreads, smem, s>>>(d, c, p, out, nsamples, counter, tiles_x, ntiles, buf, status);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_bwd_staged_t(const DenseDev &d, const CamDev &c, const ParamDev &p, const float4 *rgba,
                                       const uint32_t *nsamples, const float4 *grad_rgba, double *grad_tf,
                                       float *grad_vox, long long nvox, bool accumulate, unsigned *counter,
                                       unsigned *status, cudaStream_t s)
{
    const int tiles_x = (c.W + kStTile - 1) / kStTile, tiles_y = (c.H + kStTile - 1) / kStTile;
    const unsigned ntiles = (unsigned)tiles_x * (unsigned)tiles_y;
    const size_t bins = sizeof(float) * 4 * (size_t)p.K * kStWarps;
    const int buf = staged_buf_bytes(bins);
    const size_t smem = 2 * (size_t)buf + bins;
    auto fn = staged_bwd_kernel<T>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (!accumulate) {
        e = cudaMemsetAsync(grad_tf, 0, sizeof(double) * 4 * (size_t)p.K, s);
        if (e == cudaSuccess && grad_vox) e = cudaMemsetAsync(grad_vox, 0, sizeof(float) * (size_t)nvox, s);
        if (e != cudaSuccess) return e;
    }
    const int per_sm = occupancy_blocks((const void *)fn, kStThreads, smem);
    unsigned grid = (unsigned)(per_sm * sm_count());
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    fn<<<grid, kStThreads, smem, s>>>(d, c, p, rgba, nsamples, grad_rgba, grad_tf, grad_vox, counter, tiles_x, ntiles,
                                      buf, status);
    return cudaGetLastError();
}

cudaError_t launch_forward_staged(const DenseDev &d, vr_dtype dt, const CamDev &c, const ParamDev &p, float4 *out,
                                  uint32_t *nsamples, unsigned *counter, unsigned *status, cudaStream_t s)
{
    switch (dt) {
    case VR_F32: return launch_fwd_staged_t<float>(d, c, p, out, nsamples, counter, status, s);
    case VR_F16: return launch_fwd_staged_t<__half>(d, c, p, out, nsamples, counter, status, s);
    case VR_BF16: return launch_fwd_staged_t<__nv_bfloat16>(d, c, p, out, nsamples, counter, status, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_backward_staged(const DenseDev &d, vr_dtype dt, const CamDev &c, const ParamDev &p,
                                   const float4 *rgba, const uint32_t *nsamples, const float4 *grad_rgba,
                                   double *grad_tf, float *grad_vox, long long nvox, bool accumulate,
                                   unsigned *counter, unsigned *status, cudaStream_t s)
{
    switch (dt) {
    case VR_F32:
        return launch_bwd_staged_t<float>(d, c, p, rgba, nsamples, grad_rgba, grad_tf, grad_vox, nvox, accumulate,
                                          counter, status, s);
    case VR_F16:
        return launch_bwd_staged_t<__half>(d, c, p, rgba, nsamples, grad_rgba, grad_tf, grad_vox, nvox, accumulate,
                                           counter, status, s);
    case VR_BF16:
        return launch_bwd_staged_t<__nv_bfloat16>(d, c, p, rgba, nsamples, grad_rgba, grad_tf, grad_vox, nvox,
                                                  accumulate, counter, status, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace vr
