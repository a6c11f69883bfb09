// vr_volume.cu -- volume residency: the dense cube is copied once into a
// bricked layout that stays in HBM (the paper keeps the whole data set
// resident in GPU memory, Section 2, in texture memory, Section 4.3).
//
// Brick (bx, by, bz) stores voxels [bx*B, bx*B+B] x [by*B, by*B+B] x
// [bz*B, bz*B+B]: B^3 cells plus a one-voxel apron on the high side, so the
// eight corners of any cell are in one brick.  Apron voxels past the end of
// the volume replicate the last voxel (they are never read by a sample).
#include "vr_device.cuh"

namespace vr {

template <typename S, typename D> __device__ __forceinline__ D convert_voxel(S s);
template <> __device__ __forceinline__ float convert_voxel<float, float>(float s) { return s; }
template <> __device__ __forceinline__ __half convert_voxel<float, __half>(float s) { return __float2half_rn(s); }
template <> __device__ __forceinline__ __nv_bfloat16 convert_voxel<float, __nv_bfloat16>(float s)
{
    return __float2bfloat16_rn(s);
}
template <> __device__ __forceinline__ float convert_voxel<__half, float>(__half s) { return __half2float(s); }
template <> __device__ __forceinline__ __half convert_voxel<__half, __half>(__half s) { return s; }
template <> __device__ __forceinline__ __nv_bfloat16 convert_voxel<__half, __nv_bfloat16>(__half s)
{
    return __float2bfloat16_rn(__half2float(s));
}
template <> __device__ __forceinline__ float convert_voxel<__nv_bfloat16, float>(__nv_bfloat16 s)
{
    return __bfloat162float(s);
}
template <> __device__ __forceinline__ __half convert_voxel<__nv_bfloat16, __half>(__nv_bfloat16 s)
{
    return __float2half_rn(__bfloat162float(s));
}
template <> __device__ __forceinline__ __nv_bfloat16 convert_voxel<__nv_bfloat16, __nv_bfloat16>(__nv_bfloat16 s)
{
    return s;
}

// One CTA per (brick, z-layer of the brick): threads sweep the (B+1)^2 plane,
// reading rows of the dense cube and writing the brick plane contiguously.
template <typename S, typename D>
__global__ void __launch_bounds__(256) brick_kernel(const S *__restrict__ src, D *__restrict__ dst, int nx,
                                                     int ny, int nz, int nbx, int nby, int log2b,
                                                     long long stride)
{
    const long long brick = blockIdx.x;
    const int lz = blockIdx.y;
    const int B = 1 << log2b, B1 = B + 1;
    const int bx = (int)(brick % nbx);
    const int by = (int)((brick / nbx) % nby);
    const int bz = (int)(brick / ((long long)nbx * nby));
    const int z = min(bz * B + lz, nz - 1);
    D *out = dst + brick * stride + (long long)lz * B1 * B1;
    for (int e = threadIdx.x; e < B1 * B1; e += blockDim.x) {
        const int ly = e / B1, lx = e - ly * B1;
        const int x = min(bx * B + lx, nx - 1), y = min(by * B + ly, ny - 1);
        out[e] = convert_voxel<S, D>(src[((long long)z * ny + y) * nx + x]);
    }
    // zero the padding after the last layer so the brick is fully defined
    if (lz == B1 - 1) {
        D *pad = dst + brick * stride + (long long)B1 * B1 * B1;
        const long long npad = stride - (long long)B1 * B1 * B1;
        for (long long e = threadIdx.x; e < npad; e += blockDim.x) pad[e] = convert_voxel<float, D>(0.0f);
    }
}

template <typename S, typename D>
static cudaError_t launch_brick_t(const void *src, vr_volume *vol, cudaStream_t s)
{
    const long long nbricks = vol->nb[0] * vol->nb[1] * vol->nb[2];
    dim3 grid((unsigned)nbricks, (unsigned)(vol->brick + 1));
    brick_kernel<S, D><<<grid, 256, 0, s>>>(static_cast<const S *>(src), static_cast<D *>(vol->bricks),
                                            (int)vol->dims[0], (int)vol->dims[1], (int)vol->dims[2],
                                            (int)vol->nb[0], (int)vol->nb[1], vol->log2b, vol->stride);
    return cudaGetLastError();
}

template <typename S>
static cudaError_t launch_brick_src(const void *src, vr_volume *vol, cudaStream_t s)
{
    switch (vol->store_dtype) {
    case VR_F32: return launch_brick_t<S, float>(src, vol, s);
    case VR_F16: return launch_brick_t<S, __half>(src, vol, s);
    case VR_BF16: return launch_brick_t<S, __nv_bfloat16>(src, vol, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_brick(const void *src, vr_dtype src_dtype, vr_volume *vol, cudaStream_t s)
{
    switch (src_dtype) {
    case VR_F32: return launch_brick_src<float>(src, vol, s);
    case VR_F16: return launch_brick_src<__half>(src, vol, s);
    case VR_BF16: return launch_brick_src<__nv_bfloat16>(src, vol, s);
    }
    return cudaErrorInvalidValue;
}

// Re-bricking: the voxels of a volume's bricks (src) in bricks of another
// size, without a dense copy.  One CTA per (destination brick, z-layer);
// voxel (x, y, z) is read from the source brick that holds it.
template <typename D>
__global__ void __launch_bounds__(256) rebrick_kernel(VolDev src, D *__restrict__ dst, int log2b, int nbx, int nby,
                                                      long long stride)
{
    const long long brick = blockIdx.x;
    const int lz = blockIdx.y;
    const int B = 1 << log2b, B1 = B + 1;
    const int bx = (int)(brick % nbx);
    const int by = (int)((brick / nbx) % nby);
    const int bz = (int)(brick / ((long long)nbx * nby));
    const int z = min(bz * B + lz, src.nz - 1);
    const int SB1 = (1 << src.log2b) + 1;
    const int sbz = min(z >> src.log2b, src.nbz - 1), slz = z - (sbz << src.log2b);
    const D *sv = static_cast<const D *>(src.data);
    D *out = dst + brick * stride + (long long)lz * B1 * B1;
    for (int e = threadIdx.x; e < B1 * B1; e += blockDim.x) {
        const int ly = e / B1, lx = e - ly * B1;
        const int x = min(bx * B + lx, src.nx - 1), y = min(by * B + ly, src.ny - 1);
        const int sbx = min(x >> src.log2b, src.nbx - 1), sby = min(y >> src.log2b, src.nby - 1);
        const int slx = x - (sbx << src.log2b), sly = y - (sby << src.log2b);
        const long long sb = ((long long)sbz * src.nby + sby) * src.nbx + sbx;
        out[e] = sv[sb * src.stride + ((long long)slz * SB1 + sly) * SB1 + slx];
    }
    if (lz == B1 - 1) {
        D *pad = dst + brick * stride + (long long)B1 * B1 * B1;
        const long long npad = stride - (long long)B1 * B1 * B1;
        for (long long e = threadIdx.x; e < npad; e += blockDim.x) pad[e] = convert_voxel<float, D>(0.0f);
    }
}

cudaError_t launch_rebrick(const vr_volume *src, vr_volume *dst, cudaStream_t s)
{
    const long long nbricks = dst->nb[0] * dst->nb[1] * dst->nb[2];
    dim3 grid((unsigned)nbricks, (unsigned)(dst->brick + 1));
    const VolDev v = vol_dev(src);
    switch (dst->store_dtype) {
    case VR_F32:
        rebrick_kernel<float><<<grid, 256, 0, s>>>(v, static_cast<float *>(dst->bricks), dst->log2b, (int)dst->nb[0],
                                                   (int)dst->nb[1], dst->stride);
        break;
    case VR_F16:
        rebrick_kernel<__half><<<grid, 256, 0, s>>>(v, static_cast<__half *>(dst->bricks), dst->log2b,
                                                    (int)dst->nb[0], (int)dst->nb[1], dst->stride);
        break;
    case VR_BF16:
        rebrick_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(v, static_cast<__nv_bfloat16 *>(dst->bricks), dst->log2b,
                                                           (int)dst->nb[0], (int)dst->nb[1], dst->stride);
        break;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Hardware-filter copy: a 3D CUDA array written from the bricks through a
// surface, sampled with cudaFilterModeLinear (the measured alternative).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void surface_store(float v, cudaSurfaceObject_t s, int x, int y, int z)
{
    surf3Dwrite(v, s, x * (int)sizeof(float), y, z);
}
__device__ __forceinline__ void surface_store(__half v, cudaSurfaceObject_t s, int x, int y, int z)
{
    surf3Dwrite(__half_as_ushort(v), s, x * (int)sizeof(unsigned short), y, z);
}

template <typename D>
__global__ void __launch_bounds__(256) unbrick_to_surface(VolDev v, cudaSurfaceObject_t surf)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= v.nx) return;
    const int B = 1 << v.log2b, B1 = B + 1;
    const int bx = min(x >> v.log2b, v.nbx - 1), by = min(y >> v.log2b, v.nby - 1),
              bz = min(z >> v.log2b, v.nbz - 1);
    const int lx = x - bx * B, ly = y - by * B, lz = z - bz * B;
    const long long brick = ((long long)bz * v.nby + by) * v.nbx + bx;
    const D val = static_cast<const D *>(v.data)[brick * v.stride + ((long long)lz * B1 + ly) * B1 + lx];
    surface_store(val, surf, x, y, z);
}

vr_status build_texture(vr_volume *vol, cudaStream_t s)
{
    if (vol->tex) return VR_OK;
    if (vol->store_dtype == VR_BF16) {
        set_error("texture filter: bfloat16 storage has no hardware-filtered texture format");
        return VR_ERR_UNSUPPORTED;
    }
    int mx = 0, my = 0, mz = 0;
    cudaDeviceGetAttribute(&mx, cudaDevAttrMaxTexture3DWidth, vol->device);
    cudaDeviceGetAttribute(&my, cudaDevAttrMaxTexture3DHeight, vol->device);
    cudaDeviceGetAttribute(&mz, cudaDevAttrMaxTexture3DDepth, vol->device);
    if (vol->dims[0] > mx || vol->dims[1] > my || vol->dims[2] > mz) {
        set_error("texture filter: volume exceeds the device's 3D texture extent");
        return VR_ERR_UNSUPPORTED;
    }
    cudaChannelFormatDesc fd = vol->store_dtype == VR_F32 ? cudaCreateChannelDesc<float>()
                                                          : cudaCreateChannelDescHalf();
    cudaExtent ext = make_cudaExtent((size_t)vol->dims[0], (size_t)vol->dims[1], (size_t)vol->dims[2]);
    cudaError_t e = cudaMalloc3DArray(&vol->tex_array, &fd, ext, cudaArraySurfaceLoadStore);
    if (e != cudaSuccess) {
        vol->tex_array = nullptr;
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? (set_error("texture filter: out of device memory"), VR_ERR_OOM)
                                              : cuda_fail(e, "cudaMalloc3DArray");
    }
    cudaResourceDesc rd{};
    rd.resType = cudaResourceTypeArray;
    rd.res.array.array = vol->tex_array;
    cudaSurfaceObject_t surf = 0;
    e = cudaCreateSurfaceObject(&surf, &rd);
    if (e != cudaSuccess) return cuda_fail(e, "cudaCreateSurfaceObject");
    VolDev v = vol_dev(vol);
    dim3 grid((unsigned)((vol->dims[0] + 255) / 256), (unsigned)vol->dims[1], (unsigned)vol->dims[2]);
    if (vol->store_dtype == VR_F32)
        unbrick_to_surface<float><<<grid, 256, 0, s>>>(v, surf);
    else
        unbrick_to_surface<__half><<<grid, 256, 0, s>>>(v, surf);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaDestroySurfaceObject(surf);
    if (e != cudaSuccess) return cuda_fail(e, "texture build");
    cudaTextureDesc td{};
    td.addressMode[0] = td.addressMode[1] = td.addressMode[2] = cudaAddressModeClamp;
    td.filterMode = cudaFilterModeLinear;
    td.readMode = cudaReadModeElementType;
    td.normalizedCoords = 0;
    e = cudaCreateTextureObject(&vol->tex, &rd, &td, nullptr);
    if (e != cudaSuccess) {
        vol->tex = 0;
        return cuda_fail(e, "cudaCreateTextureObject");
    }
    return VR_OK;
}

// ---------------------------------------------------------------------------
// Brick copies in element order L (see BrickOrder), built brick by brick from
// the x-fastest bricks, one CTA per brick; reads are coalesced, writes follow
// the new order.  Plain copies (any storage type) in order 1 or 2; paired
// copies (16-bit storage) in any order: element (lx, ly, lz) holds its own
// value and the next one along the order's fastest axis, so that four loads
// fetch a cell's eight corners.
// ---------------------------------------------------------------------------
template <typename D, int LOG2B, int L>
__global__ void __launch_bounds__(256) reorder_kernel(const D *__restrict__ src, D *__restrict__ dst, long long stride)
{
    using O = BrickOrder<LOG2B, L>;
    constexpr int B1 = O::B1;
    const D *s = src + (long long)blockIdx.x * stride;
    D *o = dst + (long long)blockIdx.x * stride;
    for (int e = threadIdx.x; e < (int)stride; e += blockDim.x) {
        if (e >= B1 * B1 * B1) {      // padding
            o[e] = s[e];
            continue;
        }
        const int lz = e / (B1 * B1), r = e - lz * B1 * B1, ly = r / B1, lx = r - ly * B1;
        o[lx * O::SX + ly * O::SY + lz * O::SZ] = s[e];
    }
}

template <typename D, int LOG2B, int L>
__global__ void __launch_bounds__(256) pair_kernel(const D *__restrict__ src, typename Pair<D>::V *__restrict__ dst,
                                                   long long stride)
{
    using O = BrickOrder<LOG2B, L>;
    constexpr int B1 = O::B1;
    constexpr int NB = L == 0 ? 1 : (L == 1 ? B1 : B1 * B1);   // next element along the fastest axis (source)
    const D *s = src + (long long)blockIdx.x * stride;
    typename Pair<D>::V *o = dst + (long long)blockIdx.x * stride;
    for (int e = threadIdx.x; e < (int)stride; e += blockDim.x) {
        if (e >= B1 * B1 * B1) {      // padding
            o[e] = Pair<D>::pack(convert_voxel<float, D>(0.0f), convert_voxel<float, D>(0.0f));
            continue;
        }
        const int lz = e / (B1 * B1), r = e - lz * B1 * B1, ly = r / B1, lx = r - ly * B1;
        const int la = L == 0 ? lx : (L == 1 ? ly : lz);
        const D a = s[e];
        const D nxt = la + 1 < B1 ? s[e + NB] : a;
        o[lx * O::SX + ly * O::SY + lz * O::SZ] = Pair<D>::pack(a, nxt);
    }
}

// Blocked copy (see Blocked in vr_device.cuh): one CTA per brick, writes in
// the blocked order (coalesced), each element read from the x-fastest brick;
// padding elements (past the apron) are zero.
template <typename D, int LOG2B, int W>
__global__ void __launch_bounds__(256) block_kernel(const D *__restrict__ src, D *__restrict__ dst,
                                                    long long src_stride)
{
    using G = BlockGeom<(int)sizeof(D), LOG2B>;
    constexpr int B1 = (1 << LOG2B) + 1;
    const D *s = src + (long long)blockIdx.x * src_stride;
    D *o = dst + (long long)blockIdx.x * G::stride;
    for (int e = threadIdx.x; e < (int)G::stride; e += blockDim.x) {
        const int blk = e / G::BS, in = e - blk * G::BS;
        const int bu = blk % G::NU, bv = (blk / G::NU) % G::NV, bw = blk / (G::NU * G::NV);
        const int lu = 2 * bu + (in & 1), lv = 2 * bv + ((in >> 1) & 1), lw = bw * G::BW + (in >> 2);
        const int lx = W == 0 ? lw : lu, ly = W == 0 ? lu : (W == 1 ? lw : lv), lz = W == 2 ? lw : lv;
        o[e] = (lx < B1 && ly < B1 && lz < B1) ? s[((long long)lz * B1 + ly) * B1 + lx]
                                               : convert_voxel<float, D>(0.0f);
    }
}

long long blocked_stride(int log2b, int elem_bytes)
{
    switch (log2b) {
    case 4: return elem_bytes == 4 ? BlockGeom<4, 4>::stride : BlockGeom<2, 4>::stride;
    case 5: return elem_bytes == 4 ? BlockGeom<4, 5>::stride : BlockGeom<2, 5>::stride;
    default: return elem_bytes == 4 ? BlockGeom<4, 6>::stride : BlockGeom<2, 6>::stride;
    }
}

template <typename D, int LOG2B, int L, bool PAIRED>
static void copy_t(vr_volume *vol, void *dst, cudaStream_t s)
{
    const unsigned nbricks = (unsigned)(vol->nb[0] * vol->nb[1] * vol->nb[2]);
    const D *src = static_cast<const D *>(vol->bricks);
    if constexpr (PAIRED) {
        if constexpr (!std::is_same<D, float>::value)
            pair_kernel<D, LOG2B, L><<<nbricks, 256, 0, s>>>(src, static_cast<typename Pair<D>::V *>(dst),
                                                             vol->stride);
    } else if constexpr (L != 0) {
        reorder_kernel<D, LOG2B, L><<<nbricks, 256, 0, s>>>(src, static_cast<D *>(dst), vol->stride);
    }
}

template <typename D, int LOG2B>
static void copy_b(vr_volume *vol, int copy, cudaStream_t s)
{
    void *dst = vol->copies[copy];
    const unsigned nbricks = (unsigned)(vol->nb[0] * vol->nb[1] * vol->nb[2]);
    const D *src = static_cast<const D *>(vol->bricks);
    switch (copy) {
    case 1: copy_t<D, LOG2B, 1, false>(vol, dst, s); break;
    case 2: copy_t<D, LOG2B, 2, false>(vol, dst, s); break;
    case 3: copy_t<D, LOG2B, 0, true>(vol, dst, s); break;
    case 4: copy_t<D, LOG2B, 1, true>(vol, dst, s); break;
    case 5: copy_t<D, LOG2B, 2, true>(vol, dst, s); break;
    case 6: block_kernel<D, LOG2B, 0><<<nbricks, 256, 0, s>>>(src, static_cast<D *>(dst), vol->stride); break;
    case 7: block_kernel<D, LOG2B, 1><<<nbricks, 256, 0, s>>>(src, static_cast<D *>(dst), vol->stride); break;
    default: block_kernel<D, LOG2B, 2><<<nbricks, 256, 0, s>>>(src, static_cast<D *>(dst), vol->stride); break;
    }
}

template <typename D>
static void copy_d(vr_volume *vol, int copy, cudaStream_t s)
{
    switch (vol->log2b) {
    case 4: copy_b<D, 4>(vol, copy, s); break;
    case 5: copy_b<D, 5>(vol, copy, s); break;
    default: copy_b<D, 6>(vol, copy, s); break;
    }
}

// ---------------------------------------------------------------------------
// Texture-layer copies (float storage): voxel (x, y, z) is texel (u, v) of
// layer a, with a the voxel's coordinate across the copy's axis A and (u, v)
// its in-layer coordinates (LayerUV<A>).  One thread per voxel, reading the
// bricks in x order and writing through the layered surface.
// ---------------------------------------------------------------------------
// Voxel (x, y, z) of a float volume's bricks.
__device__ __forceinline__ float brick_voxel(const VolDev &v, int x, int y, int z)
{
    const int B = 1 << v.log2b, B1 = B + 1;
    const int bx = min(x >> v.log2b, v.nbx - 1), by = min(y >> v.log2b, v.nby - 1),
              bz = min(z >> v.log2b, v.nbz - 1);
    const int lx = x - bx * B, ly = y - by * B, lz = z - bz * B;
    const long long brick = ((long long)bz * v.nby + by) * v.nbx + bx;
    return static_cast<const float *>(v.data)[brick * v.stride + ((long long)lz * B1 + ly) * B1 + lx];
}

// Layers across z (u = x) or y (u = x): threads along x read and write
// neighbouring voxels.
template <int A>
__global__ void __launch_bounds__(256) unbrick_to_layers(VolDev v, cudaSurfaceObject_t surf)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= v.nx) return;
    const float val = brick_voxel(v, x, y, z);
    const int c[3] = {x, y, z};
    surf2DLayeredwrite(val, surf, c[LayerUV<A>::u] * (int)sizeof(float), c[LayerUV<A>::v], c[A]);
}

// Layers across x (u = z): a 32 x 32 tile of (x, z) at one y goes through
// shared memory, read along x and written along z.
__global__ void __launch_bounds__(256) unbrick_to_x_layers(VolDev v, cudaSurfaceObject_t surf)
{
    __shared__ float tile[32][33];
    const int x0 = blockIdx.x * 32, z0 = blockIdx.z * 32, y = blockIdx.y;
    const int tx = threadIdx.x, ty = threadIdx.y;                 // 32 x 8 threads
    for (int r = ty; r < 32; r += 8) {
        const int x = x0 + tx, z = z0 + r;
        if (x < v.nx && z < v.nz) tile[r][tx] = brick_voxel(v, x, y, z);
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int z = z0 + tx, x = x0 + r;
        if (x < v.nx && z < v.nz) surf2DLayeredwrite(tile[tx][r], surf, z * (int)sizeof(float), y, x);
    }
}

static cudaError_t fill_layers(vr_volume *vol, int axis, cudaStream_t s)
{
    const VolDev v = vol_dev(vol);
    const cudaSurfaceObject_t surf = vol->layers[axis].surf;
    if (axis == 0) {
        const dim3 grid((unsigned)((vol->dims[0] + 31) / 32), (unsigned)vol->dims[1], (unsigned)((vol->dims[2] + 31) / 32));
        unbrick_to_x_layers<<<grid, dim3(32, 8), 0, s>>>(v, surf);
        return cudaGetLastError();
    }
    const dim3 grid((unsigned)((vol->dims[0] + 255) / 256), (unsigned)vol->dims[1], (unsigned)vol->dims[2]);
    if (axis == 1) unbrick_to_layers<1><<<grid, 256, 0, s>>>(v, surf);
    else unbrick_to_layers<2><<<grid, 256, 0, s>>>(v, surf);
    return cudaGetLastError();
}

static void destroy_layers(vr_volume::Layers &l)
{
    if (l.tex) cudaDestroyTextureObject(l.tex);
    if (l.surf) cudaDestroySurfaceObject(l.surf);
    if (l.array) cudaFreeArray(l.array);
    l = vr_volume::Layers();
}

void free_layers(vr_volume *vol)
{
    for (vr_volume::Layers &l : vol->layers) destroy_layers(l);
}

cudaError_t build_layers(vr_volume *vol, int axis, cudaStream_t s)
{
    if (vol->store_dtype != VR_F32 || axis < 0 || axis > 2) return cudaErrorInvalidValue;
    if (vol->layers[axis].tex) return cudaSuccess;
    const int64_t ext[3] = {vol->dims[0], vol->dims[1], vol->dims[2]};
    const int u = (int)ext[axis == 0 ? 2 : 0], v = (int)ext[axis == 1 ? 2 : 1], n = (int)ext[axis];
    int mw = 0, mh = 0, ml = 0;
    cudaDeviceGetAttribute(&mw, cudaDevAttrMaxTexture2DLayeredWidth, vol->device);
    cudaDeviceGetAttribute(&mh, cudaDevAttrMaxTexture2DLayeredHeight, vol->device);
    cudaDeviceGetAttribute(&ml, cudaDevAttrMaxTexture2DLayeredLayers, vol->device);
    if (u > mw || v > mh || n > ml) return cudaErrorInvalidValue;        // beyond the texture limits
    vr_volume::Layers &l = vol->layers[axis];
    cudaError_t e = dev_alloc_layers(&l.array, u, v, n);
    if (e != cudaSuccess) {
        l.array = nullptr;
        return e;
    }
    cudaResourceDesc rd{};
    rd.resType = cudaResourceTypeArray;
    rd.res.array.array = l.array;
    e = cudaCreateSurfaceObject(&l.surf, &rd);
    if (e == cudaSuccess) e = fill_layers(vol, axis, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
        cudaTextureDesc td{};
        td.addressMode[0] = td.addressMode[1] = td.addressMode[2] = cudaAddressModeClamp;
        td.filterMode = cudaFilterModePoint;
        td.readMode = cudaReadModeElementType;
        td.normalizedCoords = 0;
        e = cudaCreateTextureObject(&l.tex, &rd, &td, nullptr);
    }
    if (e != cudaSuccess) {
        l.tex = 0;
        destroy_layers(l);
    }
    return e;
}

size_t copy_bytes(const vr_volume *vol, int copy)
{
    if (copy_layers(copy)) return (size_t)(vol->dims[0] * vol->dims[1] * vol->dims[2]) * sizeof(float);
    if (copy_blocked(copy)) {
        const int eb = vol->store_dtype == VR_F32 ? 4 : 2;
        return (size_t)(vol->nb[0] * vol->nb[1] * vol->nb[2]) * (size_t)blocked_stride(vol->log2b, eb) * (size_t)eb;
    }
    return copy_paired(copy) ? 2 * vol->bytes : vol->bytes;
}

cudaError_t launch_copy(vr_volume *vol, int copy, cudaStream_t s)
{
    if (copy_layers(copy)) return vol->layers[copy - 9].tex ? fill_layers(vol, copy - 9, s) : cudaErrorInvalidValue;
    if (copy < 1 || copy >= 9 || !vol->copies[copy]) return cudaErrorInvalidValue;
    if (vol->store_dtype == VR_F32 && copy_paired(copy)) return cudaErrorInvalidValue;   // no float pairs
    switch (vol->store_dtype) {
    case VR_F32: copy_d<float>(vol, copy, s); break;
    case VR_F16: copy_d<__half>(vol, copy, s); break;
    case VR_BF16: copy_d<__nv_bfloat16>(vol, copy, s); break;
    }
    return cudaGetLastError();
}

}  // namespace vr
