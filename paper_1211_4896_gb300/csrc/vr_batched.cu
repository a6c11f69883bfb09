// vr_batched.cu -- many (volume, camera, transfer function, image) jobs in one
// persistent launch per brick layout (an extension: the paper's future-work
// item on many smaller cubes).  Warps pull ray tiles of all jobs of a layout
// from one global atomic queue; a tile index maps to its job by binary search
// over the per-job tile prefix.  The launches (counter reset + one kernel per
// layout, independent of one another) form a CUDA graph built once and
// replayed while the job list is unchanged.
#include "vr_device.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

namespace vr {

constexpr int kBatThreads = 256;

struct JobDev {
    VolDev v;
    CamDev c;
    ParamDev p;
    float4 *out;
    uint32_t *nsamples;
    int tiles_x;
    unsigned tile_begin;     // first global tile index of this job
};

// One launch serves the jobs that read one brick copy (element type T, order
// L; template parameters, so each instance keeps the register budget of a
// single march; a batch reading several copies launches once per copy).
// CTAs per SM the register budget is sized for: paired 16-bit copies fit
// four (64 registers) without spills and gain from it; the texture layers
// gain from five (48 registers, some spilled to L1; the eight 1080p views of
// the 1024^3 cube 13.0 ms, against 14.7 at four and 17.4 at the compiler's
// three: their gathers wait on the texture unit, and more warps hide it); the other
// kernels keep the compiler's choice (for float bricks, three CTAs measured
// faster than four), so do the kernels whose warps share tiles (their
// hand-over spills at 64).
template <typename T> struct BatMinBlocks { static constexpr int value = 0; };   // 0: no minimum
template <> struct BatMinBlocks<Pair<__half>> { static constexpr int value = 4; };
template <> struct BatMinBlocks<Pair<__nv_bfloat16>> { static constexpr int value = 4; };
template <> struct BatMinBlocks<TexLayers<float>> { static constexpr int value = 5; };

// Warps per tile: 2^log2_wpt warps of a CTA take one tile of tw x (th 2^log2_wpt)
// rays together, each its own tw x th part, so that the neighbouring parts
// run on one SM and share its L1; the group's first lane takes the tile from
// the queue and hands it over through shared memory between two named
// barriers of the group (the second keeps the slot until all have read it).
__device__ __forceinline__ void group_barrier(int id, int threads)
{
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(threads) : "memory");
}

template <typename T, int LOG2B, int L, int LOG2_WPT>
__global__ void __launch_bounds__(kBatThreads, LOG2_WPT ? 0 : BatMinBlocks<T>::value) batched_kernel(const JobDev *__restrict__ jobs, int njobs,
                                                               unsigned total_tiles, unsigned *counter,
                                                               int log2_tw)
{
    __shared__ unsigned handed[kBatThreads / 32];
    const int lane = threadIdx.x & 31;
    const int tw = 1 << log2_tw;
    for (;;) {
        unsigned tile = 0;
        if constexpr (LOG2_WPT == 0) {
            if (lane == 0) tile = atomicAdd(counter, 1u);
            tile = __shfl_sync(kFull, tile, 0);
        } else {
            const int group = (threadIdx.x >> 5) >> LOG2_WPT;
            if ((threadIdx.x & ((32 << LOG2_WPT) - 1)) == 0) handed[group] = atomicAdd(counter, 1u);
            group_barrier(1 + group, 32 << LOG2_WPT);
            tile = handed[group];
            group_barrier(1 + group, 32 << LOG2_WPT);
        }
        if (tile >= total_tiles) break;
        // job = last j with tile_begin <= tile
        int lo = 0, hi = njobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&jobs[mid].tile_begin) <= tile) lo = mid; else hi = mid - 1;
        }
        const JobDev &J = jobs[lo];
        const unsigned local = tile - J.tile_begin;
        const int th = 32 >> log2_tw;
        const int i = (int)(local % J.tiles_x) * tw + (lane & (tw - 1));
        const int part = (threadIdx.x >> 5) & ((1 << LOG2_WPT) - 1);
        const int j = (((int)(local / J.tiles_x) << LOG2_WPT) + part) * th + (lane >> log2_tw);
        const CamDev c = J.c;
        const ParamDev p = J.p;
        const VolDev v = J.v;
        const bool inside = i < c.W && j < c.H;
        Ray ray;
        const bool hit = inside && setup_ray(c, v.nx, v.ny, v.nz, p.step, i, j, ray);
        Composite acc{0.0f, 0.0f, 0.0f, 1.0f};
        const int used = march_ray<T, LOG2B, L>(v, p, ray, hit, acc);
        if (inside) write_pixel(p, acc, hit ? used : 0, J.out, J.nsamples, (long long)j * c.W + i);
    }
}

using BatchFn = void (*)(const JobDev *, int, unsigned, unsigned *, int);

// Kernel for the brick layout v reads (see Layout) and 2^log2_wpt warps per tile.
static BatchFn pick_kernel(const VolDev &v, vr_dtype dt, int log2_wpt)
{
    return visit_layout_all(
        v, dt,
        [&](auto lay) -> BatchFn {
            using Y = decltype(lay);
            switch (log2_wpt) {
            case 0: return batched_kernel<typename Y::type, Y::log2b, Y::order, 0>;
            case 1: return batched_kernel<typename Y::type, Y::log2b, Y::order, 1>;
            case 2: return batched_kernel<typename Y::type, Y::log2b, Y::order, 2>;
            }
            return (BatchFn) nullptr;
        },
        (BatchFn) nullptr);
}

constexpr int kGroups = kCopyIds + 1;    // brick copies a batch may read: the bricks + every copy id

// The jobs reading one brick copy: descriptors [first, first + njobs) of the
// grouped table, tiles numbered from 0 within the group.
struct Segment {
    int first = 0, njobs = 0;
    unsigned total_tiles = 0;
    BatchFn fn = nullptr;
    unsigned grid = 0;
};

// A prepared batch: job descriptors resident on the device, a work counter,
// and (optionally) the instantiated graph of one launch.
struct BatchPlan {
    std::vector<unsigned char> key;
    std::vector<const vr_volume *> vols;   // the volumes its jobs read (dropped with any of them)
    JobDev *djobs = nullptr;
    unsigned *counter = nullptr;       // one work counter per group
    int njobs = 0;
    Segment seg[kGroups];
    int log2_tw = 3;
    int log2_wpt = 0;
    cudaGraphExec_t exec = nullptr;
    int device = 0;
};

static std::mutex g_plans_mu;
static std::map<std::vector<unsigned char>, BatchPlan *> g_plans;
constexpr size_t kMaxPlans = 64;

// Cache key of a job list: the device, the stream, the options and every
// named field of every job (never the raw struct bytes, whose padding a
// caller need not initialise).  The stream is part of the key because a plan
// owns one work counter: two streams replaying one plan at the same time
// would share it.
template <typename V> static void key_put(std::vector<unsigned char> &k, const V &v)
{
    const unsigned char *b = reinterpret_cast<const unsigned char *>(&v);
    k.insert(k.end(), b, b + sizeof(V));
}

static std::vector<unsigned char> plan_key(int dev, cudaStream_t s, int tile_w, int ctas, int wpt, const vr_job *jobs,
                                           int n)
{
    std::vector<unsigned char> k;
    k.reserve(64 + (size_t)n * 200);
    key_put(k, dev);
    key_put(k, s);
    key_put(k, tile_w);
    key_put(k, ctas);
    key_put(k, wpt);
    for (int q = 0; q < n; ++q) {
        const vr_job &J = jobs[q];
        key_put(k, J.vol);
        const vr_camera &c = J.cam;
        key_put(k, c.kind);
        for (int a = 0; a < 3; ++a) key_put(k, c.eye[a]), key_put(k, c.forward[a]), key_put(k, c.up[a]);
        key_put(k, c.fov_y_deg);
        key_put(k, c.ortho_height);
        key_put(k, c.width);
        key_put(k, c.height);
        const vr_params &p = J.params;
        key_put(k, p.tf_rgba);
        key_put(k, p.tf_size);
        key_put(k, p.vmin);
        key_put(k, p.vmax);
        key_put(k, p.step);
        key_put(k, p.ert_threshold);
        for (int a = 0; a < 4; ++a) key_put(k, p.bg_rgba[a]);
        key_put(k, p.filter);
        key_put(k, p.mode);
        key_put(k, J.dev_rgba_out);
        key_put(k, J.dev_nsamples_out);
    }
    return k;
}

static int log2_of(int x)
{
    int l = 0;
    while ((1 << l) < x) ++l;
    return (1 << l) == x ? l : -1;
}

// Builds the descriptors of all jobs into hj[0, n), grouped by the brick copy
// each view reads (group g = copy + 1: the bricks first, then the paired
// copies in order 0, 1, 2; call order within a group), and fills seg[] with
// each group's offset, tile count and kernel.  group_of, order and cost are
// host scratch of n entries.  may_build allows building a missing copy.
static vr_status prepare_jobs(const vr_job *jobs, int n, int tile_w, int wpt, bool may_build, cudaStream_t s,
                              JobDev *hj, int *group_of, int *order, double *cost, Segment seg[kGroups],
                              const char *who)
{
    const int tile_h = 32 / tile_w * wpt;           // rows of one group's tile
    vr_dtype dt = VR_F32;
    int log2b = 5;
    for (int g = 0; g < kGroups; ++g) seg[g] = Segment();
    for (int q = 0; q < n; ++q) {
        const vr_job &J = jobs[q];
        if (!J.vol) return (set_error("jobs[" + std::to_string(q) + "].vol is NULL"), VR_ERR_INVALID_ARG);
        if (!J.dev_rgba_out || !is_aligned16(J.dev_rgba_out))
            return (set_error("jobs[" + std::to_string(q) + "].dev_rgba_out must be non-NULL and 16-byte aligned"),
                    VR_ERR_INVALID_ARG);
        if (J.params.filter != VR_FILTER_SOFTWARE)
            return (set_error(std::string(who) + ": software filter only"), VR_ERR_UNSUPPORTED);
        if (q == 0) {
            dt = J.vol->store_dtype;
            log2b = J.vol->log2b;
        } else if (J.vol->store_dtype != dt || J.vol->log2b != log2b) {
            return (set_error(std::string(who) + ": all volumes of a batch must share store dtype and brick size"),
                    VR_ERR_UNSUPPORTED);
        }
        group_of[q] = preferred_copy(J.vol, &J.cam, may_build, s, kReadsBlocked | kReadsLayers) + 1;
        ++seg[group_of[q]].njobs;
    }
    int fill[kGroups];
    for (int g = 0, first = 0; g < kGroups; first += seg[g].njobs, ++g) fill[g] = seg[g].first = first;
    // Within a group the most expensive jobs come first (pixels x samples along
    // the box diagonal), so that the last tiles handed out are cheap ones and
    // the launch ends with a short tail; ties keep the call order.
    for (int q = 0; q < n; ++q) {
        const vr_job &J = jobs[q];
        double d2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double ext = (double)(J.vol->dims[a] - 1) * J.vol->spacing[a];
            d2 += ext * ext;
        }
        cost[q] = (double)J.cam.width * (double)J.cam.height * std::sqrt(d2) / (double)J.params.step;
        order[q] = q;
    }
    std::sort(order, order + n, [&](int a, int b) {
        if (group_of[a] != group_of[b]) return group_of[a] < group_of[b];
        if (cost[a] != cost[b]) return cost[a] > cost[b];
        return a < b;
    });
    for (int k = 0; k < n; ++k) {
        const int q = order[k];
        const vr_job &J = jobs[q];
        Segment &g = seg[group_of[q]];
        JobDev &d = hj[fill[group_of[q]]++];
        prepare_camera(J.vol, &J.cam, &d.c);
        prepare_params(&J.params, &d.p);
        d.v = vol_dev_copy(J.vol, group_of[q] - 1);
        d.out = reinterpret_cast<float4 *>(J.dev_rgba_out);
        d.nsamples = J.dev_nsamples_out;
        d.tiles_x = (J.cam.width + tile_w - 1) / tile_w;
        const unsigned tiles_y = (unsigned)((J.cam.height + tile_h - 1) / tile_h);
        d.tile_begin = g.total_tiles;
        const unsigned long long t = (unsigned long long)g.total_tiles + (unsigned long long)d.tiles_x * tiles_y;
        if (t > 0xFFFFFFF0ull) return (set_error(std::string(who) + ": too many ray tiles"), VR_ERR_INVALID_ARG);
        g.total_tiles = (unsigned)t;
    }
    for (int g = 0; g < kGroups; ++g) {
        if (!seg[g].njobs) continue;
        seg[g].fn = pick_kernel(hj[seg[g].first].v, dt, log2_of(wpt));     // one layout per group
        if (!seg[g].fn) return (set_error(std::string(who) + ": unsupported brick size"), VR_ERR_UNSUPPORTED);
    }
    return VR_OK;
}

// Persistent grid of each group: ctas_per_sm (0: the occupancy limit) x SMs,
// capped at one warp per part of a tile.
static void size_grids(Segment seg[kGroups], int ctas, int wpt)
{
    for (int o = 0; o < kGroups; ++o) {
        Segment &g = seg[o];
        if (!g.njobs) continue;
        const int per_sm = ctas > 0 ? ctas : occupancy_blocks((const void *)g.fn, kBatThreads, 0);   // cached
        const unsigned grid = (unsigned)(per_sm * sm_count());
        const unsigned per_cta = (unsigned)(kBatThreads / 32 / wpt);          // tiles a CTA works on at once
        const unsigned useful = (g.total_tiles + per_cta - 1) / per_cta;
        g.grid = grid < useful ? grid : (useful ? useful : 1);
        log_line("batch, brick layout %d: %d job(s), %u tiles, grid %u x %d threads", o - 1, g.njobs, g.total_tiles,
                 g.grid, kBatThreads);
    }
}

// Graph of one batched call: the counter reset, then one kernel node per
// non-empty group, the groups independent of one another so that the tail of
// one group's launch overlaps the work of the others.
static cudaError_t build_graph(BatchPlan *plan)
{
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e != cudaSuccess) return e;
    cudaGraphNode_t reset = nullptr;
    cudaMemsetParams mp = {};
    mp.dst = plan->counter;
    mp.value = 0;
    mp.elementSize = sizeof(unsigned);
    mp.width = kGroups;
    mp.height = 1;
    e = cudaGraphAddMemsetNode(&reset, graph, nullptr, 0, &mp);
    for (int g = 0; g < kGroups && e == cudaSuccess; ++g) {
        const Segment &sg = plan->seg[g];
        if (!sg.njobs) continue;
        const JobDev *djobs = plan->djobs + sg.first;
        int njobs = sg.njobs, log2_tw = plan->log2_tw;
        unsigned total = sg.total_tiles;
        unsigned *ctr = plan->counter + g;
        void *args[] = {&djobs, &njobs, &total, &ctr, &log2_tw};
        cudaKernelNodeParams kp = {};
        kp.func = (void *)sg.fn;
        kp.gridDim = dim3(sg.grid);
        kp.blockDim = dim3(kBatThreads);
        kp.sharedMemBytes = 0;
        kp.kernelParams = args;
        cudaGraphNode_t node = nullptr;
        e = cudaGraphAddKernelNode(&node, graph, &reset, 1, &kp);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&plan->exec, graph, 0);
    cudaGraphDestroy(graph);
    return e;
}

// Counter reset and one launch per non-empty group, in order on stream s.
static cudaError_t launch_segments(const Segment seg[kGroups], const JobDev *djobs, unsigned *counters,
                                   int log2_tw, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(counters, 0, kGroups * sizeof(unsigned), s);
    for (int o = 0; o < kGroups && e == cudaSuccess; ++o) {
        const Segment &g = seg[o];
        if (!g.njobs) continue;
        g.fn<<<g.grid, kBatThreads, 0, s>>>(djobs + g.first, g.njobs, g.total_tiles, counters + o, log2_tw);
        e = cudaGetLastError();
    }
    return e;
}

static vr_status validate_batch(const vr_job *jobs, int n, const vr_batch_opts *opts, int &tile_w, int &ctas,
                                int &wpt)
{
    if (!jobs || n < 1) return (set_error("jobs must be non-NULL with n >= 1"), VR_ERR_INVALID_ARG);
    if (n > 65536) return (set_error("n must be <= 65536"), VR_ERR_INVALID_ARG);
    tile_w = (opts && opts->tile_w) ? opts->tile_w : 8;
    const int tile_h = (opts && opts->tile_h) ? opts->tile_h : 32 / tile_w;
    if (log2_of(tile_w) < 0 || tile_w * tile_h != 32)
        return (set_error("tile_w * tile_h must be 32 with tile_w a power of two"), VR_ERR_INVALID_ARG);
    ctas = opts ? opts->ctas_per_sm : 0;
    if (ctas < 0 || ctas > 32) return (set_error("ctas_per_sm must be in [0, 32]"), VR_ERR_INVALID_ARG);
    wpt = (opts && opts->warps_per_tile) ? opts->warps_per_tile : 1;
    if (wpt != 1 && wpt != 2 && wpt != 4)
        return (set_error("warps_per_tile must be 0, 1, 2 or 4"), VR_ERR_INVALID_ARG);
    return VR_OK;
}

static void destroy_plan(BatchPlan *p)
{
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->djobs) cudaFree(p->djobs);
    if (p->counter) cudaFree(p->counter);
    delete p;
}

// Drops every cached plan that references `vol` (called before the volume is
// freed, with the device synchronised).
void purge_plans(const vr_volume *vol)
{
    std::lock_guard<std::mutex> g(g_plans_mu);
    for (auto it = g_plans.begin(); it != g_plans.end();) {
        const std::vector<const vr_volume *> &vs = it->second->vols;
        if (std::find(vs.begin(), vs.end(), vol) != vs.end()) {
            destroy_plan(it->second);
            it = g_plans.erase(it);
        } else {
            ++it;
        }
    }
}

}  // namespace vr

using namespace vr;

extern "C" vr_status vr_render_batched(const vr_job *jobs, int n, const vr_batch_opts *opts, void *cuda_stream)
{
    set_error("");
    int tile_w = 8, ctas = 0, wpt = 1;
    vr_status st = validate_batch(jobs, n, opts, tile_w, ctas, wpt);
    if (st != VR_OK) return st;
    for (int q = 0; q < n; ++q) {
        st = validate_job(&jobs[q], q);
        if (st != VR_OK) return st;
    }
    const int use_graph = opts ? opts->use_graph : 0;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0;
    cudaGetDevice(&dev);

    const std::vector<unsigned char> key = plan_key(dev, s, tile_w, ctas, wpt, jobs, n);

    std::lock_guard<std::mutex> g(g_plans_mu);
    BatchPlan *plan = nullptr;
    auto it = g_plans.find(key);
    if (it != g_plans.end()) plan = it->second;
    if (!plan) {
        std::vector<JobDev> hj((size_t)n);
        std::vector<int> group_of((size_t)n), order((size_t)n);
        std::vector<double> cost((size_t)n);
        Segment seg[kGroups];
        st = prepare_jobs(jobs, n, tile_w, wpt, true, s, hj.data(), group_of.data(), order.data(), cost.data(), seg,
                          "vr_render_batched");
        if (st != VR_OK) return st;
        size_grids(seg, ctas, wpt);
        plan = new BatchPlan();
        plan->key = key;
        plan->njobs = n;
        for (int q = 0; q < n; ++q)
            if (std::find(plan->vols.begin(), plan->vols.end(), jobs[q].vol) == plan->vols.end())
                plan->vols.push_back(jobs[q].vol);
        for (int g = 0; g < kGroups; ++g) plan->seg[g] = seg[g];
        plan->log2_tw = log2_of(tile_w);
        plan->log2_wpt = log2_of(wpt);
        plan->device = dev;
        cudaError_t e = dev_alloc(reinterpret_cast<void **>(&plan->djobs), sizeof(JobDev) * (size_t)n);
        if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void **>(&plan->counter), kGroups * sizeof(unsigned));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(plan->djobs, hj.data(), sizeof(JobDev) * (size_t)n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            destroy_plan(plan);
            return cuda_fail(e, "vr_render_batched: plan upload");
        }
        if (g_plans.size() >= kMaxPlans) {
            // bound the cache: the plans may still run on any stream, so the
            // device is synchronised before they are freed
            cudaDeviceSynchronize();
            for (auto &kv : g_plans) destroy_plan(kv.second);
            g_plans.clear();
        }
        g_plans[key] = plan;
    }
    cudaError_t e;
    if (use_graph) {
        if (!plan->exec) {
            e = build_graph(plan);
            if (e != cudaSuccess) {
                plan->exec = nullptr;
                return cuda_fail(e, "vr_render_batched: graph build");
            }
        }
        e = cudaGraphLaunch(plan->exec, s);
    } else {
        e = launch_segments(plan->seg, plan->djobs, plan->counter, plan->log2_tw, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "vr_render_batched launch");
    return VR_OK;
}

extern "C" vr_status vr_autotune_batched(const vr_job *jobs, int n, vr_batch_opts *best, void *cuda_stream)
{
    if (!best) return (set_error("best is NULL"), VR_ERR_INVALID_ARG);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int shapes[4][2] = {{8, 4}, {4, 8}, {16, 2}, {32, 1}};
    const int ctas_list[5] = {0, 1, 2, 3, 4};
    const int wpt_list[3] = {1, 2, 4};
    float best_ms = 1e30f;
    vr_batch_opts win = *best;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return (set_error("cudaEventCreate failed"), VR_ERR_CUDA);
    vr_status result = VR_OK;
    for (auto &sh : shapes) {
        for (int ct : ctas_list) {
          for (int wpt : wpt_list) {
            vr_batch_opts o = *best;
            o.tile_w = sh[0];
            o.tile_h = sh[1];
            o.ctas_per_sm = ct;
            o.warps_per_tile = wpt;
            o.use_graph = 0;
            vr_status st = vr_render_batched(jobs, n, &o, cuda_stream);      // warm-up (builds the plan)
            if (st != VR_OK) { result = st; goto done; }
            cudaEventRecord(e0, s);
            for (int rep = 0; rep < 3; ++rep) vr_render_batched(jobs, n, &o, cuda_stream);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) { result = cuda_fail(cudaGetLastError(), "autotune"); goto done; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) {
                best_ms = ms;
                win = o;
            }
          }
        }
    }
    win.use_graph = best->use_graph;
    *best = win;
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return result;
}

// ---------------------------------------------------------------------------
// Batched render without any allocation.
//
// vr_render_batched allocates a descriptor table and a work counter on the
// device the first time it sees a job list.  Callers that must not allocate
// device memory at call time -- services with a fixed memory budget,
// processes whose memory belongs to another allocator's pool, frame loops
// that cannot take the synchronisation an allocation may cause -- use
// vr_render_batched_noalloc instead.  Its scratch (the descriptors of up to
// kNoAllocMaxJobs jobs and the counter) is one static device array of about
// 64 KB that every GPU loading this library holds until the process exits.
// Every call reuses that array, so calls that overlap on the GPU race.
// ---------------------------------------------------------------------------
namespace vr {

constexpr int kNoAllocMaxJobs = VR_NOALLOC_MAX_JOBS;

struct NoAllocScratch {
    unsigned counter[kGroups];            // one work counter per brick-copy group
    unsigned pad[64 - kGroups];           // keeps the descriptor table 256-byte aligned
    JobDev jobs[kNoAllocMaxJobs];
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Device address of g_noalloc_scratch per device, looked up once per device
// (host code only sees a stand-in for the symbol, never its device address).
static NoAllocScratch *noalloc_scratch_ptr(vr_status &st)
{
    static std::mutex mu;
    static NoAllocScratch *ptrs[64] = {nullptr};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        st = cuda_fail(e, "cudaGetDevice");
        return nullptr;
    }
    if (dev < 0 || dev >= 64) {
        st = (set_error("vr_render_batched_noalloc: device index out of range"), VR_ERR_UNSUPPORTED);
        return nullptr;
    }
    std::lock_guard<std::mutex> g(mu);
    if (!ptrs[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            st = cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol, "cudaGetSymbolAddress(noalloc scratch)");
            return nullptr;
        }
        ptrs[dev] = static_cast<NoAllocScratch *>(p);
    }
    st = VR_OK;
    return ptrs[dev];
}

}  // namespace vr

extern "C" vr_status vr_render_batched_noalloc(const vr_job *jobs, int n, int tile_w, int tile_h, void *cuda_stream)
{
    set_error("");
    if (!jobs || n < 1) return (set_error("jobs must be non-NULL with n >= 1"), VR_ERR_INVALID_ARG);
    if (n > kNoAllocMaxJobs)
        return (set_error("vr_render_batched_noalloc: n = " + std::to_string(n) + " exceeds the maximum of " +
                          std::to_string(kNoAllocMaxJobs) + " jobs held by its static scratch"),
                VR_ERR_INVALID_ARG);
    if (tile_w == 0) tile_w = 8;
    if (tile_h == 0) tile_h = 32 / tile_w;
    const int log2_tw = log2_of(tile_w);
    if (log2_tw < 0 || tile_w * tile_h != 32)
        return (set_error("tile_w * tile_h must be 32 with tile_w a power of two"), VR_ERR_INVALID_ARG);
    for (int q = 0; q < n; ++q) {
        vr_status st = validate_job(&jobs[q], q);
        if (st != VR_OK) return st;
    }
    // descriptors, built in fixed host buffers (no host allocation either)
    static thread_local JobDev hj[kNoAllocMaxJobs];
    static thread_local int group_of[kNoAllocMaxJobs], order[kNoAllocMaxJobs];
    static thread_local double cost[kNoAllocMaxJobs];
    Segment seg[kGroups];
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // only brick copies that exist already are used (building one allocates)
    vr_status st = prepare_jobs(jobs, n, tile_w, 1, false, s, hj, group_of, order, cost, seg,
                                  "vr_render_batched_noalloc");
    if (st != VR_OK) return st;
    size_grids(seg, 0, 1);
    NoAllocScratch *scratch = noalloc_scratch_ptr(st);
    if (!scratch) return st;
    // The counters must start at zero; the descriptors overwrite the last call's.
    cudaError_t e = cudaMemcpyAsync(scratch->jobs, hj, sizeof(JobDev) * (size_t)n, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "vr_render_batched_noalloc: scratch upload");
    e = launch_segments(seg, scratch->jobs, scratch->counter, log2_tw, s);
    if (e != cudaSuccess) return cuda_fail(e, "vr_render_batched_noalloc launch");
    return VR_OK;
}
