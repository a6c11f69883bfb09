// vr_device.cuh -- device helpers shared by the forward, backward and batched
// kernels: ray setup (camera + box clipping), trilinear interpolation from the
// bricked layout, and the transfer-function lookup.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "vr_internal.h"

namespace vr {

constexpr unsigned kFull = 0xffffffffu;

// Bounds-check build (-DVR_BOUNDS_CHECK, a stand-in for a memory checker):
// every voxel gather, gradient scatter, table-bin and per-brick index is
// tested against its buffer before the access; a failing index sets
// kStatusOutOfBounds in the volume's status word (vr_check reports it) and the
// access is skipped.  The normal build compiles the tests away.
#ifdef VR_BOUNDS_CHECK
constexpr bool kBoundsCheck = true;
#else
constexpr bool kBoundsCheck = false;
#endif

// True when 0 <= i < n; otherwise records the violation in *status.
__device__ __forceinline__ bool index_ok(unsigned *status, long long i, long long n)
{
    if (i >= 0 && i < n) return true;
    if (status) atomicOr(status, kStatusOutOfBounds);
    return false;
}

// ---------------------------------------------------------------------------
// Voxel loads (read-only path), widened to float.
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ float ldv(const T *p);
template <> __device__ __forceinline__ float ldv<float>(const float *p) { return __ldg(p); }
template <> __device__ __forceinline__ float ldv<__half>(const __half *p) { return __half2float(__ldg(p)); }
template <> __device__ __forceinline__ float ldv<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    return __bfloat162float(__ldg(p));
}

// Element of a paired brick copy of a 16-bit volume: the element's own value
// and the value one step further along the copy's fastest axis, loaded
// together (4 bytes), so that four loads fetch the eight corners of a cell.  The last layer along
// that axis (the apron, never a cell origin) repeats its own value.
template <typename S> struct Pair;
template <> struct Pair<__half> {
    using V = __half2;
    static __device__ __forceinline__ V pack(__half a, __half b) { return __halves2half2(a, b); }
};
template <> struct Pair<__nv_bfloat16> {
    using V = __nv_bfloat162;
    static __device__ __forceinline__ V pack(__nv_bfloat16 a, __nv_bfloat16 b) { return __halves2bfloat162(a, b); }
};

template <typename T> struct is_pair { static constexpr bool value = false; };
template <typename S> struct is_pair<Pair<S>> { static constexpr bool value = true; };

// Element of a blocked brick copy (storage type S), for views whose rays are
// far apart: inside each brick the voxels sit in blocks of 2 x 2 x BW that
// fill one 32-byte sector (BW = 2 for float, 4 for 16-bit storage), deep
// along the copy's axis w, the axis the view's rays advance along most.  A
// ray that shares no sector with its neighbours then fetches a new sector
// only every BW / 2 ... BW steps of a cell's 2 x 2 columns, where a
// row-ordered brick costs two sectors per step whatever the voxel size; so
// a 16-bit volume moves half the sectors of a float one.  Blocks follow each
// other across u first: a 128-byte line then holds a ray's neighbouring
// columns, so each ray keeps fewer lines live in L1 and L2.  (Blocks of one
// column made contiguous along w moved 10-20% fewer DRAM bytes per sample
// but were 15% slower on the 4096 x 4096 x 1024 cube: every column a ray
// reads then holds a line of its own for 16 steps.)
template <typename S> struct Blocked {
    using storage = S;
};
template <typename T> struct is_blocked { static constexpr bool value = false; };
template <typename S> struct is_blocked<Blocked<S>> { static constexpr bool value = true; };

// Element of a texture-layer copy of a float volume (Section 4.3 keeps the
// sub-cubes in texture memory): a 2D layered texture, one layer per voxel
// plane across axis A (the copy's order), whose in-layer (u, v) axes are
// given by LayerUV; read with tld4, the texture unit's four-texel
// gather, two per sample (the cell's corners in layer a0 and a0 + 1) at the
// cell's exact integer corner, so the values are the stored texels and the
// interpolation stays the software one (bit-identical to the bricks).  The
// texture's block-linear tiling keeps both in-layer axes local, and the
// texture unit does the addressing that the bricks cost in instructions.
// VolDev.data holds the cudaTextureObject_t.
template <typename S> struct TexLayers {
    using storage = S;
};
template <typename T> struct is_layers { static constexpr bool value = false; };
template <typename S> struct is_layers<TexLayers<S>> { static constexpr bool value = true; };

// In-layer texel axes (u, v) of a layer copy across axis A: layers across z
// hold (x, y), across x hold (z, y), across y hold (x, z).
template <int A> struct LayerUV {
    static constexpr int u = A == 0 ? 2 : 0;
    static constexpr int v = A == 1 ? 2 : 1;
};

// Geometry of a blocked brick of B^3 cells (B + 1 voxels per axis with the
// apron, padded to whole blocks).  Axes (u, v, w): w is the copy's axis, u
// and v the other two in x, y, z order.  Element (lu, lv, lw) of a brick is
//   (((lw / BW) NV + lv / 2) NU + lu / 2) BS + (lw % BW) 4 + (lv % 2) 2 + lu % 2.
template <int ELEM_BYTES, int LOG2B> struct BlockGeom {
    static constexpr int B = 1 << LOG2B;
    static constexpr int BW = ELEM_BYTES == 4 ? 2 : 4;         // block depth along w
    static constexpr int BS = 4 * BW;                          // elements per block (32 bytes)
    static constexpr int NU = (B + 2) / 2, NV = (B + 2) / 2;   // blocks across u and v
    static constexpr int NW = (B + BW) / BW;                   // blocks along w (B + 1 voxels, padded)
    static constexpr long long stride = (long long)NU * NV * NW * BS;
    static __host__ __device__ __forceinline__ int index(int lu, int lv, int lw)
    {
        return (((lw / BW) * NV + (lv >> 1)) * NU + (lu >> 1)) * BS + (lw % BW) * 4 + (lv & 1) * 2 + (lu & 1);
    }
};

// ---------------------------------------------------------------------------
// Brick layouts a kernel can read (host-side dispatch).  Every volume has its
// x-fastest bricks (element type = storage type, order 0).  Copies for views
// along other axes: plain copies in order 1 or 2 (element type = storage
// type); for 16-bit storage also paired copies in any order (element type
// Pair<S>, as many bytes as float bricks).
// ---------------------------------------------------------------------------
template <typename T, int LOG2B_, int L_> struct Layout {
    using type = T;
    static constexpr int log2b = LOG2B_, order = L_;
};

// Calls f(Layout<...>{}) for the layout of v (storage type S); returns
// `none` for a layout no volume builds.
template <typename S, int LOG2B, typename F, typename R>
R visit_layout_b(const VolDev &v, F &&f, R none)
{
    if (!v.paired && v.order == 0) return f(Layout<S, LOG2B, 0>{});
    if (!v.paired && v.order == 1) return f(Layout<S, LOG2B, 1>{});
    if (!v.paired && v.order == 2) return f(Layout<S, LOG2B, 2>{});
    if constexpr (!std::is_same<S, float>::value) {
        if (v.paired == 1 && v.order == 0) return f(Layout<Pair<S>, LOG2B, 0>{});
        if (v.paired == 1 && v.order == 1) return f(Layout<Pair<S>, LOG2B, 1>{});
        if (v.paired == 1 && v.order == 2) return f(Layout<Pair<S>, LOG2B, 2>{});
    }
    return none;
}

template <typename S, typename F, typename R>
R visit_layout_s(const VolDev &v, F &&f, R none)
{
    if (v.paired >= 2) return none;                 // blocked and layer copies: see below
    switch (v.log2b) {
    case 4: return visit_layout_b<S, 4>(v, f, none);
    case 5: return visit_layout_b<S, 5>(v, f, none);
    case 6: return visit_layout_b<S, 6>(v, f, none);
    }
    return none;
}

template <typename F, typename R>
R visit_layout(const VolDev &v, vr_dtype dt, F &&f, R none)
{
    switch (dt) {
    case VR_F32: return visit_layout_s<float>(v, f, none);
    case VR_F16: return visit_layout_s<__half>(v, f, none);
    case VR_BF16: return visit_layout_s<__nv_bfloat16>(v, f, none);
    }
    return none;
}

// Texture-layer copies (float storage only): the brick size plays no part in
// them, so one instance (LOG2B 4) serves every volume.
template <typename F, typename R>
R visit_layers(const VolDev &v, vr_dtype dt, F &&f, R none)
{
    if (dt != VR_F32) return none;
    if (v.order == 0) return f(Layout<TexLayers<float>, 4, 0>{});
    if (v.order == 1) return f(Layout<TexLayers<float>, 4, 1>{});
    if (v.order == 2) return f(Layout<TexLayers<float>, 4, 2>{});
    return none;
}

// visit_layout, texture-layer copies included (the backward).
template <typename F, typename R>
R visit_layout_tex(const VolDev &v, vr_dtype dt, F &&f, R none)
{
    if (v.paired == 3) return visit_layers(v, dt, f, none);
    return visit_layout(v, dt, f, none);
}

// visit_layout, blocked and texture-layer copies included (the kernels that
// read them: the forward and the batched forward).
template <typename S, int LOG2B, typename F, typename R>
R visit_blocked_b(const VolDev &v, F &&f, R none)
{
    if (v.order == 0) return f(Layout<Blocked<S>, LOG2B, 0>{});
    if (v.order == 1) return f(Layout<Blocked<S>, LOG2B, 1>{});
    if (v.order == 2) return f(Layout<Blocked<S>, LOG2B, 2>{});
    return none;
}

template <typename S, typename F, typename R>
R visit_layout_all_s(const VolDev &v, F &&f, R none)
{
    if (v.paired != 2) return visit_layout_s<S>(v, f, none);
    switch (v.log2b) {
    case 4: return visit_blocked_b<S, 4>(v, f, none);
    case 5: return visit_blocked_b<S, 5>(v, f, none);
    case 6: return visit_blocked_b<S, 6>(v, f, none);
    }
    return none;
}

template <typename F, typename R>
R visit_layout_all(const VolDev &v, vr_dtype dt, F &&f, R none)
{
    if (v.paired == 3) return visit_layers(v, dt, f, none);
    switch (dt) {
    case VR_F32: return visit_layout_all_s<float>(v, f, none);
    case VR_F16: return visit_layout_all_s<__half>(v, f, none);
    case VR_BF16: return visit_layout_all_s<__nv_bfloat16>(v, f, none);
    }
    return none;
}

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

// float -> storage type, round to nearest even
template <typename D> __device__ __forceinline__ D to_dtype(float v);
template <> __device__ __forceinline__ float to_dtype<float>(float v) { return v; }
template <> __device__ __forceinline__ __half to_dtype<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 to_dtype<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// ---------------------------------------------------------------------------
// Ray setup: camera model of Section 3.1's user-controlled viewport (pinhole
// or orthographic projection), clipped to the closed box [0, n-1]^3 by the
// slab method.  Samples sit at s_in + (k + 1/2) step, k = 0 .. n-1, i.e.
// n = floor((s_out - s_in)/step + 1/2) (constant sampling step, Section 4.4).
// ---------------------------------------------------------------------------
struct Ray {
    float3 q, d;      // anchor and direction, voxel space (d per world unit)
    float s_in;
    int n;
};

__device__ __forceinline__ bool slab_axis(float q, float d, float hi, float &s0, float &s1)
{
    if (d != 0.0f) {
        float rd = 1.0f / d;
        float ta = (0.0f - q) * rd, tb = (hi - q) * rd;
        s0 = fmaxf(s0, fminf(ta, tb));
        s1 = fminf(s1, fmaxf(ta, tb));
        return true;
    }
    return q >= 0.0f && q <= hi;     // parallel: inside the slab or a miss
}

__device__ __forceinline__ bool setup_ray(const CamDev &c, int nx, int ny, int nz, float step, int i, int j,
                                          Ray &r)
{
    const float hi = (float)i - 0.5f * (float)(c.W - 1);
    const float hj = (float)j - 0.5f * (float)(c.H - 1);
    r.q.x = fmaf(hi, c.qa.x, fmaf(hj, c.qb.x, c.q0.x));
    r.q.y = fmaf(hi, c.qa.y, fmaf(hj, c.qb.y, c.q0.y));
    r.q.z = fmaf(hi, c.qa.z, fmaf(hj, c.qb.z, c.q0.z));
    float3 w;
    float smin;
    if (c.persp) {
        w.x = fmaf(hi, c.wa.x, fmaf(hj, c.wb.x, c.wf.x));
        w.y = fmaf(hi, c.wa.y, fmaf(hj, c.wb.y, c.wf.y));
        w.z = fmaf(hi, c.wa.z, fmaf(hj, c.wb.z, c.wf.z));
        const float len = sqrtf(w.x * w.x + w.y * w.y + w.z * w.z);
        const float il = 1.0f / len;
        w.x *= il; w.y *= il; w.z *= il;
        smin = -c.dist * len;                  // the eye: samples only in front of it
    } else {
        w = c.wf;
        smin = -INFINITY;
    }
    r.d = make_float3(w.x * c.inv_sp.x, w.y * c.inv_sp.y, w.z * c.inv_sp.z);
    float s0 = smin, s1 = INFINITY;
    if (!slab_axis(r.q.x, r.d.x, (float)(nx - 1), s0, s1)) return false;
    if (!slab_axis(r.q.y, r.d.y, (float)(ny - 1), s0, s1)) return false;
    if (!slab_axis(r.q.z, r.d.z, (float)(nz - 1), s0, s1)) return false;
    if (!(s0 < s1)) return false;
    r.s_in = s0;
    r.n = (int)floorf((s1 - s0) / step + 0.5f);
    return r.n > 0;
}

__device__ __forceinline__ float3 sample_pos(const Ray &r, int k, float step)
{
    const float s = fmaf((float)k + 0.5f, step, r.s_in);
    return make_float3(fmaf(s, r.d.x, r.q.x), fmaf(s, r.d.y, r.q.y), fmaf(s, r.d.z, r.q.z));
}

// ---------------------------------------------------------------------------
// Trilinear interpolation (Section 4.4) from the bricked layout.  The cell
// origin is clamp(floor(p), 0, n-2) per axis; with the +1 apron all eight
// corners of the cell lie in one brick at constant offsets.
// ---------------------------------------------------------------------------
struct Cell {
    long long base;   // element index of corner (x0, y0, z0)
    float fx, fy, fz;
    int x0, y0, z0;
};

// Element order inside a brick.  Order 0 is x fastest, then y, then z; order
// 1 is y fastest, then x, then z; order 2 is z fastest, then y, then x.  A
// render reads the paired copy whose fastest axis runs closest to the image's
// horizontal axis, so the lanes of a warp's row of rays read neighbouring
// elements whatever the view direction.
template <int LOG2B, int L> struct BrickOrder {
    static constexpr int B1 = (1 << LOG2B) + 1;
    static constexpr int SX = L == 0 ? 1 : (L == 1 ? B1 : B1 * B1);
    static constexpr int SY = L == 1 ? 1 : B1;
    static constexpr int SZ = L == 2 ? 1 : B1 * B1;
};

// NARROW: the brick index in 32 bits and one widening multiply (fewer than
// 2^31 bricks of fewer than 2^31 elements, checked at creation).  Measured on
// the 1024^3 views: 9% faster for the issue-bound 16-bit march, but 4% slower
// for the batched float march (its schedule changes), so the float march
// keeps the 64-bit form.
template <int LOG2B, int L = 0, bool NARROW = false>
__device__ __forceinline__ Cell locate(const VolDev &v, float3 p)
{
    Cell c;
    c.x0 = min(max(__float2int_rd(p.x), 0), v.nx - 2);
    c.y0 = min(max(__float2int_rd(p.y), 0), v.ny - 2);
    c.z0 = min(max(__float2int_rd(p.z), 0), v.nz - 2);
    c.fx = p.x - (float)c.x0;
    c.fy = p.y - (float)c.y0;
    c.fz = p.z - (float)c.z0;
    using O = BrickOrder<LOG2B, L>;
    constexpr int B = 1 << LOG2B;
    const int bx = c.x0 >> LOG2B, by = c.y0 >> LOG2B, bz = c.z0 >> LOG2B;
    const int lx = c.x0 & (B - 1), ly = c.y0 & (B - 1), lz = c.z0 & (B - 1);
    if constexpr (NARROW) {
        const unsigned brick = ((unsigned)bz * (unsigned)v.nby + (unsigned)by) * (unsigned)v.nbx + (unsigned)bx;
        c.base = (long long)((unsigned long long)brick * (unsigned)v.stride) + (lx * O::SX + ly * O::SY + lz * O::SZ);
    } else {
        const long long brick = ((long long)bz * v.nby + by) * v.nbx + bx;
        c.base = brick * v.stride + (lx * O::SX + ly * O::SY + lz * O::SZ);
    }
    return c;
}

// The cell of a sample in a blocked copy (storage S, copy axis W): base is
// the element of corner (0, 0, 0); the corners' parities (the low bits of x0,
// y0, z0, which B keeps inside the brick) give the other seven.
template <typename S, int LOG2B, int W>
__device__ __forceinline__ Cell locate_blocked(const VolDev &v, float3 p)
{
    Cell c;
    c.x0 = min(max(__float2int_rd(p.x), 0), v.nx - 2);
    c.y0 = min(max(__float2int_rd(p.y), 0), v.ny - 2);
    c.z0 = min(max(__float2int_rd(p.z), 0), v.nz - 2);
    c.fx = p.x - (float)c.x0;
    c.fy = p.y - (float)c.y0;
    c.fz = p.z - (float)c.z0;
    using G = BlockGeom<(int)sizeof(S), LOG2B>;
    constexpr int B = 1 << LOG2B;
    const int bx = c.x0 >> LOG2B, by = c.y0 >> LOG2B, bz = c.z0 >> LOG2B;
    const int lx = c.x0 & (B - 1), ly = c.y0 & (B - 1), lz = c.z0 & (B - 1);
    const int lu = W == 0 ? ly : lx, lv = W == 2 ? ly : lz, lw = W == 0 ? lx : (W == 1 ? ly : lz);
    const unsigned brick = ((unsigned)bz * (unsigned)v.nby + (unsigned)by) * (unsigned)v.nbx + (unsigned)bx;
    c.base = (long long)((unsigned long long)brick * (unsigned)v.stride) + G::index(lu, lv, lw);
    return c;
}

// The cell of a sample in a texture-layer copy: the corner and fractions
// only (the texture unit addresses the texels).
__device__ __forceinline__ Cell locate_cell(const VolDev &v, float3 p)
{
    Cell c;
    c.x0 = min(max(__float2int_rd(p.x), 0), v.nx - 2);
    c.y0 = min(max(__float2int_rd(p.y), 0), v.ny - 2);
    c.z0 = min(max(__float2int_rd(p.z), 0), v.nz - 2);
    c.fx = p.x - (float)c.x0;
    c.fy = p.y - (float)c.y0;
    c.fz = p.z - (float)c.z0;
    c.base = 0;
    return c;
}

// The cell of a sample in the layout of element type T.
template <typename T, int LOG2B, int L, bool NARROW>
__device__ __forceinline__ Cell locate_t(const VolDev &v, float3 p)
{
    if constexpr (is_layers<T>::value) return locate_cell(v, p);
    else if constexpr (is_blocked<T>::value) return locate_blocked<typename T::storage, LOG2B, L>(v, p);
    else return locate<LOG2B, L, NARROW>(v, p);
}

// The eight corners of a cell as floats (index bit 0: +x, bit 1: +y, bit 2: +z).
struct Corners {
    float v[8];
};

__device__ __forceinline__ float2 widen2(__half2 w) { return __half22float2(w); }
__device__ __forceinline__ float2 widen2(__nv_bfloat162 w) { return __bfloat1622float2(w); }

// The eight corners of a cell as loaded from a brick copy of element type T
// and order L.  They are widened to float only where they are interpolated,
// so the loads of a sample can be issued several samples ahead of its use
// (16-bit pairs stay packed, two corners per register, while in flight).
template <typename T, int L> struct Gathered {
    T v[8];
    __device__ __forceinline__ float at(int q) const { return to_f(v[q]); }
};
template <typename S, int L> struct Gathered<Pair<S>, L> {
    typename Pair<S>::V p[4];     // pairs along the fastest axis of order L
    __device__ __forceinline__ float at(int q) const
    {
        const int i = L == 0 ? (q >> 1) : (L == 1 ? ((q & 1) | ((q >> 2) << 1)) : (q & 3));
        const int h = L == 0 ? (q & 1) : (L == 1 ? ((q >> 1) & 1) : (q >> 2));
        const float2 w = widen2(p[i]);
        return h ? w.y : w.x;
    }
};

template <typename S, int L> struct Gathered<Blocked<S>, L> {
    S v[8];
    __device__ __forceinline__ float at(int q) const { return to_f(v[q]); }
};
template <typename S, int L> struct Gathered<TexLayers<S>, L> {
    float v[8];
    __device__ __forceinline__ float at(int q) const { return v[q]; }
};

// tld4 on layer `layer` of a 2D layered texture at unnormalised (u, v): the
// red channel of the 2 x 2 texels whose centres surround (u, v), in the
// order (u0, v1), (u1, v1), (u1, v0), (u0, v0) with u0 = floor(u - 1/2).
// At u = a + 1, v = b + 1 (integers a, b) that is texels a, a + 1 and b, b + 1
// exactly, whatever the unit's fixed-point rounding.
__device__ __forceinline__ float4 gather_layer(cudaTextureObject_t t, int layer, float u, float v)
{
    float4 r;
    asm("tld4.r.a2d.v4.f32.f32 {%0, %1, %2, %3}, [%4, {%5, %6, %7, %7}];"
        : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
        : "l"(t), "r"(layer), "f"(u), "f"(v));
    return r;
}

template <typename T, int LOG2B, int L>
__device__ __forceinline__ void fetch_corners_mem(const VolDev &v, const Cell &c, Gathered<T, L> &f);

// T is the stored element: float / __half / __nv_bfloat16 (eight loads) or
// Pair<...> (four paired loads; each returns a corner and its neighbour along
// the fastest axis of order L).
template <typename T, int LOG2B, int L>
__device__ __forceinline__ void fetch_corners(const VolDev &v, const Cell &c, Gathered<T, L> &f)
{
    if constexpr (is_layers<T>::value) {
        // corners q (bit 0 +x, bit 1 +y, bit 2 +z) of layers a0 and a0 + 1; a
        // clamped cell keeps every texel inside the texture
        const cudaTextureObject_t tex = static_cast<cudaTextureObject_t>(reinterpret_cast<uintptr_t>(v.data));
        using UV = LayerUV<L>;
        const int c3[3] = {c.x0, c.y0, c.z0};
        const float u = (float)c3[UV::u] + 1.0f, w = (float)c3[UV::v] + 1.0f;
        constexpr int bu = 1 << UV::u, bv = 1 << UV::v, ba = 1 << L;      // corner bits of u, v, layer
        const float4 g0 = gather_layer(tex, c3[L], u, w);
        const float4 g1 = gather_layer(tex, c3[L] + 1, u, w);
        f.v[bv] = g0.x;
        f.v[bu | bv] = g0.y;
        f.v[bu] = g0.z;
        f.v[0] = g0.w;
        f.v[ba | bv] = g1.x;
        f.v[ba | bu | bv] = g1.y;
        f.v[ba | bu] = g1.z;
        f.v[ba] = g1.w;
    } else {
        fetch_corners_mem<T, LOG2B, L>(v, c, f);
    }
}

// The memory-copy layouts (bricks and their copies).
template <typename T, int LOG2B, int L>
__device__ __forceinline__ void fetch_corners_mem(const VolDev &v, const Cell &c, Gathered<T, L> &f)
{
    using O = BrickOrder<LOG2B, L>;
    if constexpr (kBoundsCheck && !is_blocked<T>::value) {
        constexpr long long span = is_pair<T>::value ? (L == 0 ? O::SY : O::SX) + (L == 2 ? O::SY : O::SZ)
                                                     : O::SX + O::SY + O::SZ;
        if (!index_ok(v.status, c.base, v.nelem) || !index_ok(v.status, c.base + span, v.nelem)) {
            f = Gathered<T, L>{};
            return;
        }
    }
    if constexpr (is_blocked<T>::value) {
        using S = typename T::storage;
        using G = BlockGeom<(int)sizeof(S), LOG2B>;
        // steps to the +u, +v, +w neighbour of corner (0, 0, 0): inside its block,
        // or into the next block across that axis
        const int pu = L == 0 ? c.y0 : c.x0, pv = L == 2 ? c.y0 : c.z0, pw = L == 0 ? c.x0 : (L == 1 ? c.y0 : c.z0);
        const int du = (pu & 1) ? G::BS - 1 : 1;
        const int dv = (pv & 1) ? G::NU * G::BS - 2 : 2;
        const int dw = (pw % G::BW == G::BW - 1) ? G::NV * G::NU * G::BS - (G::BW - 1) * 4 : 4;
        const int dx = L == 0 ? dw : du, dy = L == 0 ? du : (L == 1 ? dw : dv), dz = L == 2 ? dw : dv;
        if constexpr (kBoundsCheck) {
            if (!index_ok(v.status, c.base, v.nelem) || !index_ok(v.status, c.base + dx + dy + dz, v.nelem)) {
                f = Gathered<T, L>{};
                return;
            }
        }
        const S *b = static_cast<const S *>(v.data) + c.base;
        f.v[0] = __ldg(b);
        f.v[1] = __ldg(b + dx);
        f.v[2] = __ldg(b + dy);
        f.v[3] = __ldg(b + dx + dy);
        f.v[4] = __ldg(b + dz);
        f.v[5] = __ldg(b + dz + dx);
        f.v[6] = __ldg(b + dz + dy);
        f.v[7] = __ldg(b + dz + dx + dy);
    } else if constexpr (is_pair<T>::value) {
        using V = typename T::V;
        const V *b = static_cast<const V *>(v.data) + c.base;
        // the three pair bases besides b: the two non-fastest axes and both
        constexpr int A1 = L == 0 ? O::SY : O::SX;
        constexpr int A2 = L == 2 ? O::SY : O::SZ;
        f.p[0] = __ldg(b);
        f.p[1] = __ldg(b + A1);
        f.p[2] = __ldg(b + A2);
        f.p[3] = __ldg(b + A1 + A2);
    } else {
        const T *b = static_cast<const T *>(v.data) + c.base;
        f.v[0] = __ldg(b);
        f.v[1] = __ldg(b + O::SX);
        f.v[2] = __ldg(b + O::SY);
        f.v[3] = __ldg(b + O::SX + O::SY);
        f.v[4] = __ldg(b + O::SZ);
        f.v[5] = __ldg(b + O::SZ + O::SX);
        f.v[6] = __ldg(b + O::SZ + O::SY);
        f.v[7] = __ldg(b + O::SZ + O::SX + O::SY);
    }
}

// Trilinear interpolation, always along x, then y, then z (so every copy
// gives the same bits).
template <typename G>
__device__ __forceinline__ float interp_corners(const Cell &c, const G &f)
{
    const float v0 = f.at(0), v1 = f.at(1), v2 = f.at(2), v3 = f.at(3);
    const float v4 = f.at(4), v5 = f.at(5), v6 = f.at(6), v7 = f.at(7);
    const float c00 = fmaf(c.fx, v1 - v0, v0), c10 = fmaf(c.fx, v3 - v2, v2);
    const float c01 = fmaf(c.fx, v5 - v4, v4), c11 = fmaf(c.fx, v7 - v6, v6);
    const float c0 = fmaf(c.fy, c10 - c00, c00), c1 = fmaf(c.fy, c11 - c01, c01);
    return fmaf(c.fz, c1 - c0, c0);
}

// Dense index of corner q (bit 0: +x, bit 1: +y, bit 2: +z) and its weight.
__device__ __forceinline__ float corner_weight(const Cell &c, int q)
{
    const float wx = (q & 1) ? c.fx : 1.0f - c.fx;
    const float wy = (q & 2) ? c.fy : 1.0f - c.fy;
    const float wz = (q & 4) ? c.fz : 1.0f - c.fz;
    return wx * wy * wz;
}

// ---------------------------------------------------------------------------
// Transfer function (Section 3.3): the value range is partitioned into K-1
// levels between K table entries; u = clamp((v-vmin)/(vmax-vmin),0,1)(K-1),
// entries floor(u) and floor(u)+1 blended linearly.
// ---------------------------------------------------------------------------
struct TfPos {
    int i0;
    float w;
    bool interior;    // vmin < v < vmax: the lookup has a slope in v
};

__device__ __forceinline__ float4 tf_lookup(const float4 *tfs, const ParamDev &p, float v, TfPos &pos)
{
    float s = (v - p.vmin) * p.scale01;
    pos.interior = (s > 0.0f) && (s < 1.0f);
    s = fminf(fmaxf(s, 0.0f), 1.0f);          // fmaxf maps NaN to 0
    const float u = s * p.km1;
    const int i0 = min(__float2int_rd(u), p.K - 2);
    const float w = u - (float)i0;
    pos.i0 = i0;
    pos.w = w;
    const float4 e0 = tfs[i0], e1 = tfs[i0 + 1];
    return make_float4(fmaf(w, e1.x - e0.x, e0.x), fmaf(w, e1.y - e0.y, e0.y), fmaf(w, e1.z - e0.z, e0.z),
                       fmaf(w, e1.w - e0.w, e0.w));
}

__device__ __forceinline__ void load_tf_shared(float4 *tfs, const float4 *tf, int K)
{
    for (int q = threadIdx.x; q < K; q += blockDim.x) tfs[q] = __ldg(tf + q);
}

// Table lookup through the read-only L1 path.  The lanes of a warp mostly hit
// a handful of neighbouring entries (one or two 128-byte lines), which costs
// fewer L1 wavefronts than a 128-bit shared-memory load (4 wavefronts).
// The same lookup, also returning the slope of the blend between the two
// entries (e1 - e0) for the adjoint.
// The transfer-function table staged in a kernel's dynamic shared memory (K
// float4 entries, copied by stage_tf when the kernel starts).  A sample's two
// entries are then shared-memory loads: a global load, even one that hits
// L1, waits in the L1/texture pipeline behind the volume gathers in flight.
// The backward stages its table (the eight 1080p views of the 1024^3 cube:
// 22.2 -> 21.7 ms); the forward kernels read theirs through L1 (staged, they
// measured 2-4% slower, probably because the texture gathers lose the L1
// capacity the table takes).
extern __shared__ float4 vr_tf_shared[];

// All threads of the CTA copy the table; ends with a CTA barrier.
__device__ __forceinline__ void stage_tf(const ParamDev &p)
{
    for (int q = threadIdx.x; q < p.K; q += blockDim.x) vr_tf_shared[q] = __ldg(p.tf + q);
    __syncthreads();
}

// Dynamic shared memory a kernel that stages the table needs.
inline size_t tf_shared_bytes(const ParamDev &p) { return (size_t)p.K * sizeof(float4); }

// Table entry i: from the staged copy (SH) or through L1.
template <bool SH> __device__ __forceinline__ float4 tf_entry(const ParamDev &p, int i)
{
    if constexpr (SH) return vr_tf_shared[i];
    else return __ldg(p.tf + i);
}

template <bool SH = false>
__device__ __forceinline__ float4 tf_lookup_l1(const ParamDev &p, float v, TfPos &pos, float4 &de)
{
    float u = fmaf(v, p.su, p.ou);
    pos.interior = (u > 0.0f) && (u < p.km1);
    u = fminf(fmaxf(u, 0.0f), p.km1);
    const int i0 = min(__float2int_rd(u), p.K - 2);
    const float w = u - (float)i0;
    pos.i0 = i0;
    pos.w = w;
    const float4 e0 = tf_entry<SH>(p, i0), e1 = tf_entry<SH>(p, i0 + 1);
    de = make_float4(e1.x - e0.x, e1.y - e0.y, e1.z - e0.z, e1.w - e0.w);
    return make_float4(fmaf(w, de.x, e0.x), fmaf(w, de.y, e0.y), fmaf(w, de.z, e0.z), fmaf(w, de.w, e0.w));
}

template <bool SH = false>
__device__ __forceinline__ float4 tf_lookup_l1(const ParamDev &p, float v, TfPos &pos)
{
    float u = fmaf(v, p.su, p.ou);               // (v - vmin) (K-1)/(vmax - vmin)
    pos.interior = (u > 0.0f) && (u < p.km1);
    u = fminf(fmaxf(u, 0.0f), p.km1);            // fmaxf maps NaN to 0
    const int i0 = min(__float2int_rd(u), p.K - 2);
    const float w = u - (float)i0;
    pos.i0 = i0;
    pos.w = w;
    const float4 e0 = tf_entry<SH>(p, i0), e1 = tf_entry<SH>(p, i0 + 1);
    return make_float4(fmaf(w, e1.x - e0.x, e0.x), fmaf(w, e1.y - e0.y, e0.y), fmaf(w, e1.z - e0.z, e0.z),
                       fmaf(w, e1.w - e0.w, e0.w));
}

// ---------------------------------------------------------------------------
// One ray, marched front to back with early termination (Section 3.4's
// front-to-back composition): C += T a rgb, T *= 1 - a.  The warp keeps
// marching while any lane's ray is live and leaves together (warp vote).
// Loads for sample k+1 are issued before sample k is composited.
// ---------------------------------------------------------------------------
struct Composite {
    float r, g, b, T;
};

// Samples whose gathers are in flight ahead of the one being composited (1
// or 2).  A deeper pipeline keeps more gathers in flight per warp but costs a
// Cell and a Gathered set of registers per stage, and so resident warps.
// Measured on the 1024^3 eight-view workload: 16-bit layouts gain from depth
// 2 (oblique views 10% faster; packed pairs keep the register cost low),
// float loses from it (axis views 3% slower), so float keeps depth 1 (the
// single-view kernel of the texture layers asks for 2, vr_forward.cu).
template <typename T> struct Pipeline { static constexpr int depth = 2; };
template <> struct Pipeline<float> { static constexpr int depth = 1; };
template <> struct Pipeline<TexLayers<float>> { static constexpr int depth = 1; };

// The value the transfer function sees for a sample: the interpolated value
// itself (generic transfer function), or a transform of it at the sample's
// cell (the sigma-clipping transfer function, vr_modes.cu).
struct IdentityMap {
    __device__ __forceinline__ float operator()(float v, const Cell &) const { return v; }
};

// One sample: composites (cur, fc) and, while the ray goes on, issues the
// gathers of sample k + depth into (nxt, fn).
template <typename T, int LOG2B, int L, typename Map = IdentityMap, int D = Pipeline<T>::depth>
__device__ __forceinline__ void march_step(const VolDev &v, const ParamDev &p, const Ray &ray, int &k, bool &active,
                                           Composite &acc, const Cell &cur, const Gathered<T, L> &fc, Cell &nxt,
                                           Gathered<T, L> &fn, const Map &map = Map())
{
    constexpr bool N = !std::is_same<T, float>::value;
    const bool more = k + 1 < ray.n;
    if (D == 1 ? more : k + D < ray.n) {
        nxt = locate_t<T, LOG2B, L, N>(v, sample_pos(ray, k + D, p.step));
        fetch_corners<T, LOG2B, L>(v, nxt, fn);
    }
    const float val = map(interp_corners(cur, fc), cur);
    TfPos tp;
    const float4 e = tf_lookup_l1(p, val, tp);
    const float aT = e.w * acc.T;
    acc.r = fmaf(aT, e.x, acc.r);
    acc.g = fmaf(aT, e.y, acc.g);
    acc.b = fmaf(aT, e.z, acc.b);
    acc.T = fmaf(-e.w, acc.T, acc.T);
    ++k;
    if (!more || acc.T <= p.t_stop) active = false;
}

// The loop body is unrolled over depth + 1 register sets that take turns, so
// a prefetched sample is never copied.
template <typename T, int LOG2B, int L, typename Map = IdentityMap, int D = Pipeline<T>::depth>
__device__ __forceinline__ int march_ray(const VolDev &v, const ParamDev &p, const Ray &ray, bool active,
                                         Composite &acc, const Map &map = Map())
{
    static_assert(D == 1 || D == 2, "pipeline depth 1 or 2");
    constexpr bool N = !std::is_same<T, float>::value;
    int k = 0;
    Cell c0, c1, c2;
    Gathered<T, L> f0, f1, f2;
    if (active) {
        c0 = locate_t<T, LOG2B, L, N>(v, sample_pos(ray, 0, p.step));
        fetch_corners<T, LOG2B, L>(v, c0, f0);
        if (D == 2 && ray.n > 1) {
            c1 = locate_t<T, LOG2B, L, N>(v, sample_pos(ray, 1, p.step));
            fetch_corners<T, LOG2B, L>(v, c1, f1);
        }
    }
    if constexpr (D == 1) {
        for (;;) {
            if (!__any_sync(kFull, active)) break;
            if (active) march_step<T, LOG2B, L, Map, D>(v, p, ray, k, active, acc, c0, f0, c1, f1, map);
            if (!__any_sync(kFull, active)) break;
            if (active) march_step<T, LOG2B, L, Map, D>(v, p, ray, k, active, acc, c1, f1, c0, f0, map);
        }
    } else {
        // one warp vote per round of register sets (measured faster for the
        // issue-bound 16-bit march): a lane that finishes inside a round skips
        // the rest of it on its own `active`
        for (;;) {
            if (!__any_sync(kFull, active)) break;
            if (active) march_step<T, LOG2B, L, Map, D>(v, p, ray, k, active, acc, c0, f0, c2, f2, map);
            if (active) march_step<T, LOG2B, L, Map, D>(v, p, ray, k, active, acc, c1, f1, c0, f0, map);
            if (active) march_step<T, LOG2B, L, Map, D>(v, p, ray, k, active, acc, c2, f2, c1, f1, map);
        }
    }
    return k;
}

__device__ __forceinline__ void write_pixel(const ParamDev &p, const Composite &acc, int used, float4 *out,
                                            uint32_t *nsamples, long long px)
{
    const float T = acc.T;
    out[px] = make_float4(fmaf(T, p.bg.x, acc.r), fmaf(T, p.bg.y, acc.g), fmaf(T, p.bg.z, acc.b),
                          fmaf(T, p.bg.w, 1.0f - T));
    if (nsamples) nsamples[px] = (uint32_t)used;
}

}  // namespace vr
