// rt_batch.cu -- autotuning of the trace launch shape and batches of many
// scenes in one persistent, graph-captured launch (neither is in the paper;
// Sec. 4.3 re-traces the visibility of composed scenes, which is what a batch
// of scenes serves).
//
// Autotuner: for a full implicit ray set it times each candidate (traversal
// strategy: one thread per ray or one warp per 32 rays, binary or 4-wide
// tree; work order: tiles per direction sweep) on the same four blocks of
// tiles spread over the Morton range, and keeps the fastest if it beats the
// default strategy by more than 3 %.
//
// Batch: the work items (32 rays each) of all jobs form one virtual queue,
// job after job in decreasing estimated cost (rays x log2 n), consumed
// through one device counter by a persistent grid; each warp finds its job by
// binary search over the jobs' first item and runs that job's strategy.  The
// counter reset and the launch are captured into a CUDA graph at creation.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "rt_trace_core.cuh"

rt_status rt_trace_launch_job(const BvhDev &b, const RaySetDev &rs, const TraceJob &job, float *T_out,
                              int strat, rt_stream_t stream, unsigned long long *work);

namespace {

struct TuneKey {
    int dev, log2n, kind, K;
    bool operator<(const TuneKey &o) const {
        return std::tie(dev, log2n, kind, K) < std::tie(o.dev, o.log2n, o.kind, o.K);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune_cache;

constexpr int kTuneBlocks = 4;
constexpr float kTuneMargin = 0.97f;

// The strategy used without tuning, as the single-scene AUTO: for a
// direction set 4-wide packets sharing the direction, or one thread per ray
// on the 4-wide tree (far-first) for scenes of at most 2^19 Gaussians; one
// thread per ray on the 4-wide tree with lane refill for env-map and
// hemisphere rays (their directions differ within a tile); binary variants
// when there is no 4-wide tree.
int default_kernel(const rt_bvh *bvh, int32_t kind) {
    if (kind == RT_RAYS_DIRS) {
        if (bvh->n_wide == 0) return RT_KERNEL_PACKET;
        return bvh->n <= (int64_t(1) << 19) ? RT_KERNEL_RAY_WIDE : RT_KERNEL_WIDE;
    }
    return bvh->n_wide > 0 ? RT_KERNEL_RAY_REFILL : RT_KERNEL_RAY;
}

TraceJob full_job(const rt_bvh *bvh, int32_t K, int32_t order_block) {
    TraceJob job;
    memset(&job, 0, sizeof(job));
    job.mode = MODE_FULL;
    job.n_tiles = (bvh->n + 31) / 32;
    int64_t B = order_block > 0 ? order_block : 1;
    if (B > job.n_tiles) B = job.n_tiles;
    if (B < 1) B = 1;
    job.order_block = (int32_t)B;
    job.n_items = job.n_tiles * K;
    job.n_out = bvh->n * K;
    job.tile_base = 0;
    return job;
}

struct BatchJobDev {
    BvhDev b;
    RaySetDev rs;
    TraceJob job;
    float *T_out;
    int32_t strat;  // 0 per-ray, 1 packet, 2 4-wide packet, 3 4-wide packet with a shared direction,
                    // 4 per-ray 4-wide, 5 per-ray 4-wide with lane refill
    int64_t item_begin;  // item jobs: first item of the item queue
    int64_t slot_begin;  // refill jobs: first ray slot of the slot queue
};

// The lane-refill phase of the batch: the refill jobs' rays are the slots of
// one queue (job after job, item*32 + l within a job); idle lanes take slots
// as in trace_refill, each lane carrying its own job.
__device__ __forceinline__ void batch_refill(const BatchJobDev *__restrict__ jobs, int first, int n_jobs,
                                             int64_t total_slots, int *status, unsigned long long *work) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    bool has = false, exhausted = false;
    int jl = first;
    float3 o = make_float3(0.f, 0.f, 0.f), d = make_float3(0.f, 0.f, 1.f), inv = d, oi = o;
    int32_t src = -1;
    int64_t out_idx = 0;
    float T = 1.0f;
    uint32_t node = 0;
    int sp = 0;
    uint32_t stack[RT_WIDE_STACK];
    for (;;) {
        const unsigned idle = __ballot_sync(FULL, !has);
        const int n_idle = __popc(idle);
        if (!exhausted && (n_idle >= kRefillMin || n_idle == 32)) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(work, (unsigned long long)n_idle);
            base = __shfl_sync(FULL, base, 0);
            if (base + (unsigned long long)n_idle >= (unsigned long long)total_slots) exhausted = true;
            if (!has) {
                const int64_t slot = (int64_t)(base + (unsigned long long)__popc(idle & lt_mask));
                if (slot < total_slots) {
                    int lo = first, hi = n_jobs - 1;  // last refill job with slot_begin <= slot
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (jobs[mid].slot_begin <= slot) lo = mid;
                        else hi = mid - 1;
                    }
                    jl = lo;
                    const BatchJobDev &J = jobs[jl];
                    const int64_t local = slot - J.slot_begin;
                    int64_t tile;
                    int32_t k;
                    full_item(J.job, J.rs.K, local >> 5, tile, k);
                    const int64_t p = tile * 32 + (local & 31);
                    if (p < J.b.n) {
                        const float4 mu = __ldg(J.b.gauss + 4 * p);
                        const int64_t g = __float_as_int(__ldg(J.b.gauss + 4 * p + 1).w);
                        out_idx = g * J.rs.K + k;
                        implicit_ray(J.rs, out_idx, k, g, mu, o, d);
                        inv = safe_inv(d);
                        oi = make_float3(o.x * inv.x, o.y * inv.y, o.z * inv.z);
                        src = (int32_t)p;
                        T = 1.0f;
                        node = 0;
                        sp = 0;
                        has = true;
                    }
                }
            }
        }
        if (__ballot_sync(FULL, has) == 0) {
            if (exhausted) break;
            continue;
        }
        if (!has) continue;
        const BvhDev &b = jobs[jl].b;
        const bool far = far_first(jobs[jl].rs);
        const float4 *w = b.wide + 8 * (int64_t)node;
        const float4 lx = __ldg(w), hx = __ldg(w + 1), ly = __ldg(w + 2), hy = __ldg(w + 3), lz = __ldg(w + 4),
                     hz = __ldg(w + 5), rf = __ldg(w + 6);
        const uint32_t r[4] = {__float_as_uint(rf.x), __float_as_uint(rf.y), __float_as_uint(rf.z),
                               __float_as_uint(rf.w)};
        float tn[4];
        slab4_near(lx, hx, ly, hy, lz, hz, oi, inv, tn);
        const float inf = __int_as_float(0x7f800000);
        float ti[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            ti[c] = inf;
            if (!(tn[c] < inf)) continue;
            if (r[c] & RT_LEAF_BIT) {
                const int32_t p = (int32_t)(r[c] & ~RT_LEAF_BIT);
                if (p != src) gauss_hit(b, p, o, d, T);
            } else {
                ti[c] = tn[c];
            }
        }
        int next = -1;
        const bool overflow = !visit_order(ti[0], ti[1], ti[2], ti[3], r[0], r[1], r[2], r[3], far, stack, sp, next);
        if (overflow) rt_set_error(status, RT_ERR_STACK_OVERFLOW);
        bool done = overflow || T < b.t_min;
        if (!done) {
            if (next >= 0) node = (uint32_t)next;
            else if (sp > 0) node = stack[--sp];
            else done = true;
        }
        if (done) {
            jobs[jl].T_out[out_idx] = T < b.t_min ? 0.0f : T;
            has = false;
        }
    }
}

// Jobs [0, n_item_jobs) are consumed as 32-ray items (work[0]); jobs
// [n_item_jobs, n_jobs) as per-ray slots with lane refill (work[1]), after a
// warp finds the item queue empty.
#ifndef RT_BATCH_MIN_BLOCKS
#define RT_BATCH_MIN_BLOCKS 8
#endif
__global__ void __launch_bounds__(128, RT_BATCH_MIN_BLOCKS) k_trace_batch(const BatchJobDev *__restrict__ jobs, int n_item_jobs, int n_jobs,
                                                     int64_t total_items, int64_t total_slots, int *status,
                                                     unsigned long long *work) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    __shared__ int2 stk_all[4 * RT_WIDE_STACK];
    int2 *stk = stk_all + (threadIdx.x >> 5) * RT_WIDE_STACK;
    WorkCounts wc = {0, 0, 0};
    unsigned long long rays_done = 0;
    TraceAux aux;
    aux.counters = nullptr;
    aux.hit_ids = nullptr;
    aux.hit_count = nullptr;
    aux.cap = 0;
    aux.status = status;
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(work, 1ull);
        item = __shfl_sync(FULL, item, 0);
        if ((int64_t)item >= total_items) break;
        int lo = 0, hi = n_item_jobs - 1;  // last job with item_begin <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].item_begin <= (int64_t)item) lo = mid;
            else hi = mid - 1;
        }
        const BatchJobDev &J = jobs[lo];
        const int64_t local = (int64_t)item - J.item_begin;
        if (J.strat == 4) trace_item<4, false>(J.b, J.rs, J.job, J.T_out, aux, local, J.job.n_out, wc, rays_done, stk);
        else if (J.strat == 3) trace_item<3, false>(J.b, J.rs, J.job, J.T_out, aux, local, J.job.n_out, wc, rays_done, stk);
        else if (J.strat == 2) trace_item<2, false>(J.b, J.rs, J.job, J.T_out, aux, local, J.job.n_out, wc, rays_done, stk);
        else if (J.strat == 1) trace_item<1, false>(J.b, J.rs, J.job, J.T_out, aux, local, J.job.n_out, wc, rays_done, stk);
        else trace_item<0, false>(J.b, J.rs, J.job, J.T_out, aux, local, J.job.n_out, wc, rays_done, stk);
    }
    if (total_slots > 0) batch_refill(jobs, n_item_jobs, n_jobs, total_slots, status, work + 1);
}

int persistent_grid() {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_batch, 128, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return per_sm * rt_num_sms();
}

}  // namespace

extern "C" rt_status rt_trace_autotune(const rt_bvh *bvh, const rt_rayspec *rays, float *T_scratch,
                                       rt_trace_opts *opts, rt_stream_t stream) {
    if (!bvh || !rays || !opts || !T_scratch) return RT_ERR_INVALID_ARG;
    if (rays->kind == RT_RAYS_EXPLICIT || rays->ray_ids) return RT_ERR_UNSUPPORTED;
    RaySetDev rs;
    int64_t count = 0;
    RT_TRY(rt_rayset_dev(bvh, rays, &rs, &count));
    if (count == 0) return RT_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    int log2n = 0;
    while ((1ll << (log2n + 1)) <= bvh->n) ++log2n;
    const TuneKey key{dev, log2n, rays->kind, rs.K};
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            opts->kernel = it->second.first;
            opts->order_block = it->second.second;
            return RT_OK;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long *work = nullptr;
    RT_TRY(rt_alloc((void **)&work, 8 * kTuneBlocks, stream));
    const BvhDev b = bvh_dev(bvh);
    const int64_t ntiles = (bvh->n + 31) / 32;
    // about 4M rays per candidate: four contiguous blocks of tiles (all
    // directions of each tile) spread evenly over the Morton range, so the
    // sample sees several parts of the scene and each block keeps the
    // coherence of neighbouring tiles
    int64_t S = (1ll << 20) / (32ll * rs.K);
    if (S < 16) S = 16;
    int nb = kTuneBlocks;
    if (S * nb > ntiles) {
        nb = 1;
        S = ntiles;
    }
    const int blocks[] = {1, 16, 128, 1024};
    const int def_k = default_kernel(bvh, rays->kind);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f, def_ms = 1e30f;
    int best_k = def_k, best_b = 64, def_b = 64;
    rt_status res = RT_OK;
    for (int kernel = RT_KERNEL_RAY; kernel <= RT_KERNEL_RAY_REFILL && res == RT_OK; ++kernel) {
        const bool wide = kernel == RT_KERNEL_WIDE || kernel == RT_KERNEL_RAY_WIDE || kernel == RT_KERNEL_RAY_REFILL;
        // with a 4-wide tree the binary-tree strategies are not candidates (they
        // trail their 4-wide forms on every measured workload)
        if (wide != (bvh->n_wide > 0)) continue;
        // order_block only changes which rays share a warp for the packet strategies
        const int n_blocks = (kernel == RT_KERNEL_PACKET || kernel == RT_KERNEL_WIDE) ? 4 : 1;
        const int strat = kernel == RT_KERNEL_RAY_REFILL ? 5 : kernel == RT_KERNEL_RAY_WIDE ? 4 : kernel - 1;
        for (int bi = 0; bi < n_blocks && res == RT_OK; ++bi) {
            float ms = 1e30f;
            for (int rep = 0; rep < 2 && res == RT_OK; ++rep) {  // the first run warms caches
                cudaEventRecord(e0, st);
                for (int q = 0; q < nb && res == RT_OK; ++q) {
                    TraceJob job = full_job(bvh, rs.K, blocks[bi]);
                    job.n_tiles = S;
                    job.tile_base = nb == 1 ? 0 : (ntiles - S) * (2 * q + 1) / (2 * nb);
                    if (job.order_block > S) job.order_block = (int32_t)S;
                    job.n_items = S * rs.K;
                    res = rt_trace_launch_job(b, rs, job, T_scratch, strat, stream, work + q);
                }
                cudaEventRecord(e1, st);
                float t = 0.f;
                if (cudaEventSynchronize(e1) != cudaSuccess) res = RT_ERR_CUDA;
                cudaEventElapsedTime(&t, e0, e1);
                if (rep > 0 && t < ms) ms = t;
            }
            if (res != RT_OK) break;
            if (ms < best) {
                best = ms;
                best_k = kernel;
                best_b = blocks[bi];
            }
            if (kernel == def_k && ms < def_ms) {
                def_ms = ms;
                def_b = blocks[bi];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    rt_free(work, stream);
    if (res != RT_OK) return res;
    // another strategy replaces the default only when clearly faster: a
    // small margin on a sample is within run-to-run noise
    if (best_k != def_k && def_ms < 1e30f && best > kTuneMargin * def_ms) {
        best_k = def_k;
        best_b = def_b;
    }
    opts->kernel = best_k;
    opts->order_block = best_b;
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune_cache[key] = {best_k, best_b};
    return RT_OK;
}

struct rt_batch {
    int n_jobs;
    int64_t n_rays, n_items;
    std::vector<int32_t> kernel, order_block;  // per job, in the caller's order
    void *table;                                // BatchJobDev[n_jobs] + work counter
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

extern "C" rt_status rt_batch_create(const rt_batch_job *jobs, int32_t n_jobs, int32_t autotune,
                                     rt_stream_t stream, rt_batch **out) {
    if (!out || !jobs || n_jobs <= 0 || n_jobs > 4096) return RT_ERR_INVALID_ARG;
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<BatchJobDev> host(n_jobs);
    std::vector<double> cost(n_jobs);
    rt_batch *bt = new rt_batch();
    bt->n_jobs = n_jobs;
    bt->kernel.assign(n_jobs, 0);
    bt->order_block.assign(n_jobs, 0);
    bt->table = nullptr;
    bt->graph = nullptr;
    bt->exec = nullptr;
    for (int j = 0; j < n_jobs; ++j) {
        const rt_batch_job &J = jobs[j];
        int64_t count = 0;
        RaySetDev rs;
        rt_status r = (J.bvh && J.rays.kind != RT_RAYS_EXPLICIT && !J.rays.ray_ids)
                          ? rt_rayset_dev(J.bvh, &J.rays, &rs, &count)
                          : RT_ERR_INVALID_ARG;
        if (r == RT_OK && count > 0 && !J.T_out) r = RT_ERR_INVALID_ARG;
        if (r != RT_OK) {
            delete bt;
            return r;
        }
        rt_trace_opts o;
        memset(&o, 0, sizeof(o));
        o.kernel = default_kernel(J.bvh, J.rays.kind);
        o.order_block = 1;
        if (autotune && count > 0) {
            r = rt_trace_autotune(J.bvh, &J.rays, J.T_out, &o, stream);
            if (r != RT_OK) {
                delete bt;
                return r;
            }
        }
        bt->kernel[j] = o.kernel;
        bt->order_block[j] = o.order_block;
        BatchJobDev &H = host[j];
        memset(&H, 0, sizeof(H));
        H.b = bvh_dev(J.bvh);
        H.rs = rs;
        H.job = full_job(J.bvh, rs.K, o.order_block);
        H.T_out = J.T_out;
        H.strat = o.kernel == RT_KERNEL_RAY_REFILL ? (J.bvh->n_wide > 0 ? 5 : 0)
                  : o.kernel == RT_KERNEL_RAY_WIDE ? (J.bvh->n_wide > 0 ? 4 : 0)
                  : o.kernel == RT_KERNEL_WIDE ? (J.bvh->n_wide > 0 ? (J.rays.kind == RT_RAYS_DIRS ? 3 : 2) : 1)
                  : o.kernel == RT_KERNEL_PACKET ? 1 : 0;
        cost[j] = (double)count * log2((double)(J.bvh->n > 1 ? J.bvh->n : 2));
    }
    // item jobs first, then lane-refill jobs; largest estimated cost first in each
    std::vector<int> order(n_jobs);
    for (int j = 0; j < n_jobs; ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const bool ra = host[a].strat == 5, rb = host[b].strat == 5;
        return ra != rb ? rb : cost[a] > cost[b];
    });
    std::vector<BatchJobDev> queue(n_jobs);
    int64_t items = 0, slots = 0, rays = 0;
    int n_item_jobs = 0;
    for (int q = 0; q < n_jobs; ++q) {
        queue[q] = host[order[q]];
        if (queue[q].strat == 5) {
            queue[q].slot_begin = slots;
            slots += queue[q].job.n_items * 32;
        } else {
            queue[q].item_begin = items;
            items += queue[q].job.n_items;
            ++n_item_jobs;
        }
        rays += queue[q].job.n_out;
    }
    bt->n_items = items + slots / 32;
    bt->n_rays = rays;
    const size_t tbytes = ((sizeof(BatchJobDev) * n_jobs + 255) & ~(size_t)255);
    rt_status r = rt_alloc(&bt->table, tbytes + 256, stream);
    if (r != RT_OK) {
        delete bt;
        return r;
    }
    BatchJobDev *dtab = (BatchJobDev *)bt->table;
    unsigned long long *work = (unsigned long long *)((char *)bt->table + tbytes);
    if (cudaMemcpyAsync(dtab, queue.data(), sizeof(BatchJobDev) * n_jobs, cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        rt_free(bt->table, stream);
        delete bt;
        return RT_ERR_CUDA;
    }
    // capture: reset the queue counter, one persistent launch
    cudaStream_t cap;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
        rt_free(bt->table, stream);
        delete bt;
        return RT_ERR_CUDA;
    }
    const int grid = persistent_grid();
    int *status = rt_status_ptr();
    bool ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        cudaMemsetAsync(work, 0, 16, cap);
        k_trace_batch<<<grid, 128, 0, cap>>>(dtab, n_item_jobs, n_jobs, items, slots, status, work);
        ok = cudaStreamEndCapture(cap, &bt->graph) == cudaSuccess;
    }
    if (ok) ok = cudaGraphInstantiate(&bt->exec, bt->graph, 0) == cudaSuccess;
    cudaStreamDestroy(cap);
    if (!ok) {
        cudaGetLastError();
        if (bt->exec) cudaGraphExecDestroy(bt->exec);
        if (bt->graph) cudaGraphDestroy(bt->graph);
        rt_free(bt->table, stream);
        delete bt;
        return RT_ERR_CUDA;
    }
    *out = bt;
    return RT_OK;
}

extern "C" rt_status rt_batch_run(rt_batch *bt, rt_stream_t stream) {
    if (!bt) return RT_ERR_INVALID_ARG;
    return cudaGraphLaunch(bt->exec, (cudaStream_t)stream) == cudaSuccess ? RT_OK : RT_ERR_CUDA;
}

extern "C" rt_status rt_batch_info(const rt_batch *bt, int64_t *n_rays, int64_t *n_items, int32_t *kernel,
                                   int32_t *order_block) {
    if (!bt) return RT_ERR_INVALID_ARG;
    if (n_rays) *n_rays = bt->n_rays;
    if (n_items) *n_items = bt->n_items;
    for (int j = 0; j < bt->n_jobs; ++j) {
        if (kernel) kernel[j] = bt->kernel[j];
        if (order_block) order_block[j] = bt->order_block[j];
    }
    return RT_OK;
}

extern "C" rt_status rt_batch_destroy(rt_batch *bt, rt_stream_t stream) {
    if (!bt) return RT_ERR_INVALID_ARG;
    cudaStreamSynchronize((cudaStream_t)stream);
    if (bt->exec) cudaGraphExecDestroy(bt->exec);
    if (bt->graph) cudaGraphDestroy(bt->graph);
    rt_free(bt->table, stream);
    delete bt;
    return RT_OK;
}
