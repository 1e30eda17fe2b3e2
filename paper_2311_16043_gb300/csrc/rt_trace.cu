// rt_trace.cu -- visibility of a ray set (Eq. 13-15, Sec. 4.1-4.2).
//
// One persistent launch: each warp repeatedly takes a work item of 32 rays
// from a device counter.  For a full implicit set (every Gaussian x K
// directions) an item is 32 Gaussians adjacent in Morton order x one
// direction, so the warp's rays are nearly parallel and start close together.
// Items are ordered in sweeps: `order_block` tiles for direction 0, the same
// tiles for direction 1, ... .  The default, one tile per sweep, hands out a
// tile's K directions in turn: the rows T[g, 0..K) of a tile are written
// within a short window (whole sectors merge in L2) and the warps in flight
// start in the same region of the tree (sweeps of 64 to 62,500 tiles measured
// 0.6-2 % slower on the 2M-Gaussian object scene).  Explicit ray lists and id
// subsets are taken in chunks of 32 in the given order.
#include <string.h>

#include "rt_trace_core.cuh"

// Resident blocks per SM the trace kernels are compiled for (register cap).
#ifndef RT_TRACE_MIN_BLOCKS
#define RT_TRACE_MIN_BLOCKS 8
#endif

namespace {

template <int STRAT, bool COUNT>
__global__ void __launch_bounds__(128, RT_TRACE_MIN_BLOCKS) k_trace(BvhDev b, RaySetDev rs, TraceJob job, float *T_out,
                                               TraceAux aux, unsigned long long *work) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    __shared__ int2 stk_all[(STRAT == 2 || STRAT == 3) ? 4 * RT_WIDE_STACK : 1];
    int2 *stk = stk_all + ((STRAT == 2 || STRAT == 3) ? (threadIdx.x >> 5) * RT_WIDE_STACK : 0);
    WorkCounts wc = {0, 0, 0};
    unsigned long long rays_done = 0;
    if (STRAT == 5) {  // per-ray slots with lane refill (full implicit sets)
        trace_refill<COUNT>(b, rs, job, T_out, aux, work, wc, rays_done);
        flush_counts<COUNT>(aux, wc, rays_done);
        return;
    }
    if (STRAT == 6) {  // one warp per ray: an item is one ray
        __shared__ uint32_t wstk_all[STRAT == 6 ? 4 * kWarpStack : 1];
        uint32_t *wstk = wstk_all + (threadIdx.x >> 5) * kWarpStack;
        for (;;) {
            unsigned long long item = 0;
            if (lane == 0) item = atomicAdd(work, 1ull);
            item = __shfl_sync(FULL, item, 0);
            int64_t n_out = job.mode == MODE_FULL ? job.n_items * 32 : job.n_out;  // slots
            if (job.dyn_count) {
                const int64_t c = (int64_t)*job.dyn_count;
                n_out = c < n_out ? c : n_out;
            }
            if ((int64_t)item >= n_out) break;
            float3 o, d;
            int32_t src;
            int64_t out_idx;
            if (!ray_of(b, rs, job, (int64_t)item, o, d, src, out_idx, aux.status)) {
                if (lane == 0 && out_idx >= 0) T_out[out_idx] = __int_as_float(0x7fc00000);
                continue;
            }
            const float T = trace_warp_ray<COUNT>(b, o, d, src, wstk, wc, aux.status);
            if (lane == 0) {
                T_out[out_idx] = T;
                rays_done++;
            }
        }
        flush_counts<COUNT>(aux, wc, rays_done);
        return;
    }
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(work, 1ull);
        item = __shfl_sync(FULL, item, 0);
        if ((int64_t)item >= job.n_items) break;
        int64_t n_out = job.n_out;
        if (job.dyn_count) {
            const int64_t c = (int64_t)*job.dyn_count;
            n_out = c < n_out ? c : n_out;
            if ((int64_t)item * 32 >= n_out) break;
        }
        trace_item<STRAT, COUNT>(b, rs, job, T_out, aux, (int64_t)item, n_out, wc, rays_done, stk);
    }
    flush_counts<COUNT>(aux, wc, rays_done);
}

// Sort keys of an id list (per-ray traversal of long lists): rays of one
// direction index in the tree's (Morton) order of their Gaussians, so that
// neighbouring threads walk neighbouring parts of the tree.  DIRS: key =
// k * n + sorted position; hemisphere and env-map sets (directions differ
// per Gaussian or per sample): the sorted position alone.  Invalid ids sort
// last and are reported by the trace.
__global__ void k_list_keys(BvhDev b, RaySetDev rs, int64_t m, uint32_t *keys, int32_t *vals) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t rid = rs.ray_ids[i];
        uint32_t key = 0xffffffffu;
        if (rid >= 0 && rid < rs.n_rays) {
            const int64_t g = rid / rs.K;
            const uint32_t p = (uint32_t)b.rank[g];
            key = rs.kind == RT_RAYS_DIRS ? (uint32_t)(rid - g * rs.K) * (uint32_t)b.n + p : p;
        }
        keys[i] = key;
        vals[i] = (int32_t)i;
    }
}
// The list in sorted order and each entry's place in the caller's list.
__global__ void k_list_perm(const int64_t *ids, const int32_t *vals, int64_t m, int64_t *sorted_ids,
                            int64_t *out_index) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = vals[j];
        sorted_ids[j] = ids[i];
        out_index[j] = i;
    }
}

int persistent_blocks(const void *kernel, int threads) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return per_sm * rt_num_sms();
}

}  // namespace

// Launch the single-scene kernel on an explicit job (used by the autotuner).
rt_status rt_trace_launch_job(const BvhDev &b, const RaySetDev &rs, const TraceJob &job, float *T_out,
                              int strat, rt_stream_t stream, unsigned long long *work) {
    TraceAux aux;
    memset(&aux, 0, sizeof(aux));
    aux.status = rt_status_ptr();
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(work, 0, sizeof(unsigned long long), st) != cudaSuccess) return RT_ERR_CUDA;
    const int threads = 128;
    if (strat == 6 && b.wide) {
        int grid = persistent_blocks((const void *)k_trace<6, false>, threads);
        k_trace<6, false><<<grid, threads, 0, st>>>(b, rs, job, T_out, aux, work);
    } else if (strat == 5 && b.wide && job.mode == MODE_FULL) {
        int grid = persistent_blocks((const void *)k_trace<5, false>, threads);
        k_trace<5, false><<<grid, threads, 0, st>>>(b, rs, job, T_out, aux, work);
    } else if (strat >= 4 && b.wide) {
        int grid = persistent_blocks((const void *)k_trace<4, false>, threads);
        k_trace<4, false><<<grid, threads, 0, st>>>(b, rs, job, T_out, aux, work);
    } else if (strat >= 4) {
        int grid = persistent_blocks((const void *)k_trace<0, false>, threads);
        k_trace<0, false><<<grid, threads, 0, st>>>(b, rs, job, T_out, aux, work);
    } else if (strat >= 2 && b.wide) {
        if (job.mode == MODE_FULL && rs.kind == RT_RAYS_DIRS) {
            int grid = persistent_blocks((const void *)k_trace<3, false>, threads);
            k_trace<3, false><<<grid, threads, 0, st>>>(b, rs, job, T_out, aux, work);
        } else {
            int grid = persistent_blocks((const void *)k_trace<2, false>, threads);
            k_trace<2, false><<<grid, threads, 0, st>>>(b, rs, job, T_out, aux, work);
        }
    } else if (strat >= 1) {
        int grid = persistent_blocks((const void *)k_trace<1, false>, threads);
        k_trace<1, false><<<grid, threads, 0, st>>>(b, rs, job, T_out, aux, work);
    } else {
        int grid = persistent_blocks((const void *)k_trace<0, false>, threads);
        k_trace<0, false><<<grid, threads, 0, st>>>(b, rs, job, T_out, aux, work);
    }
    return rt_check_launch();
}

// Shared by rt_trace_visibility and the batched launch.
rt_status rt_trace_launch(const rt_bvh *bvh, const rt_rayspec *rays, float *T_out,
                          const rt_trace_opts *opts, rt_stream_t stream, unsigned long long *work) {
    RaySetDev rs;
    int64_t count = 0;
    RT_TRY(rt_rayset_dev(bvh, rays, &rs, &count));
    if (count > 0 && !T_out) return RT_ERR_INVALID_ARG;
    rt_trace_opts o;
    memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.kernel < 0 || o.kernel > 6 || o.order_block < 0 || o.block_threads < 0) return RT_ERR_INVALID_ARG;
    if ((o.hit_ids && (o.hit_cap <= 0 || !o.hit_count)) ) return RT_ERR_INVALID_ARG;
    if (count == 0) return RT_OK;

    TraceJob job;
    job.out_index = nullptr;
    job.dyn_count = nullptr;
    job.n_out = count;
    job.order_block = 1;
    job.n_tiles = 0;
    job.tile_base = 0;
    if (rays->kind == RT_RAYS_EXPLICIT) job.mode = MODE_EXPLICIT;
    else if (rays->ray_ids) job.mode = MODE_IDS;
    else job.mode = MODE_FULL;
    if (job.mode == MODE_FULL) {
        job.n_tiles = (bvh->n + 31) / 32;
        int64_t B = o.order_block > 0 ? o.order_block : 1;
        if (B > job.n_tiles) B = job.n_tiles;
        job.order_block = (int32_t)B;
        job.n_items = job.n_tiles * rs.K;
    } else {
        job.n_items = (count + 31) / 32;
    }
    int strat = o.kernel == RT_KERNEL_WARP_RAY ? 6 : o.kernel == RT_KERNEL_RAY_REFILL ? 5
              : o.kernel == RT_KERNEL_RAY_WIDE ? 4 : o.kernel == RT_KERNEL_WIDE ? 2
              : o.kernel == RT_KERNEL_PACKET ? 1 : 0;
    // one warp per ray needs the 4-wide tree and keeps no hit log
    if (strat == 6 && (bvh->n_wide == 0 || o.hit_ids)) strat = bvh->n_wide ? 4 : 0;
    // AUTO:
    // - a direction set: warp packets sharing the direction, except over at
    //   most 2^19 Gaussians, where the per-ray walk (farthest child first)
    //   is faster (object scenes: 100k 18 %, 300k 5 %, 500k 2.7 % with the
    //   nearest child first; from 1M on the packets win);
    // - env-map and hemisphere sets (directions differ across a tile): the
    //   per-ray walk with lane refill;
    // - explicit rays and id lists (scattered rays): one warp per ray up to
    //   2^22 rays, its lanes sharing one ray's nodes (2M object scene,
    //   scattered ids: 2^16 rays 3.7x and 2^20 rays 1.25x the per-ray
    //   walks), and one thread per ray over the 4-wide tree for longer lists
    //   (2^24 rays: 6 % faster than one warp per ray).
    if (o.kernel == RT_KERNEL_AUTO && job.mode == MODE_FULL)
        strat = rays->kind == RT_RAYS_DIRS ? (bvh->n <= (int64_t(1) << 19) ? 4 : 2) : 5;
    if (o.kernel == RT_KERNEL_AUTO && job.mode != MODE_FULL) strat = count <= (int64_t(1) << 22) ? 6 : 4;
    // lane refill needs the 4-wide tree and a full implicit set, and keeps no hit log
    if (strat == 5 && (bvh->n_wide == 0 || job.mode != MODE_FULL || o.hit_ids)) strat = 4;
    if (strat == 2 && bvh->n_wide == 0) strat = 1;
    if (strat == 4 && bvh->n_wide == 0) strat = 0;
    if (strat == 2 && job.mode == MODE_FULL && rays->kind == RT_RAYS_DIRS) strat = 3;  // shared direction

    TraceAux aux;
    aux.counters = (unsigned long long *)o.counters;
    aux.hit_ids = o.hit_ids;
    aux.hit_count = o.hit_count;
    aux.cap = o.hit_cap;
    aux.status = rt_status_ptr();
    BvhDev b = bvh_dev(bvh);
    cudaStream_t st = (cudaStream_t)stream;

    // AUTO on a long id list (per-ray traversal): trace it in the order of
    // (direction, the tree's order of the Gaussians), each T written back to
    // its place in the caller's list (2M object scene, 64M stratified
    // held-out rays: 141 against 111 M rays/s); each ray's traversal, and so
    // its T, is the same in any order
    void *sort_blk = nullptr;
    if (o.kernel == RT_KERNEL_AUTO && job.mode == MODE_IDS && strat == 4 && count < (int64_t(1) << 31) &&
        (uint64_t)rs.K * (uint64_t)bvh->n < (uint64_t(1) << 32)) {
        auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
        const size_t b4 = up(size_t(count) * 4), b8 = up(size_t(count) * 8);
        RT_TRY(rt_alloc(&sort_blk, 2 * b4 + 2 * b8, stream));
        uint32_t *keys = (uint32_t *)sort_blk;
        int32_t *vals = (int32_t *)((char *)sort_blk + b4);
        int64_t *sids = (int64_t *)((char *)sort_blk + 2 * b4), *oidx = (int64_t *)((char *)sort_blk + 2 * b4 + b8);
        const int g = rt_num_sms() * 8;
        k_list_keys<<<g, 256, 0, (cudaStream_t)stream>>>(bvh_dev(bvh), rs, count, keys, vals);
        rt_status r = rt_check_launch();
        if (r == RT_OK) r = rt_sort_pairs_u32(keys, vals, count, 32, stream);
        if (r == RT_OK) {
            k_list_perm<<<g, 256, 0, (cudaStream_t)stream>>>(rs.ray_ids, vals, count, sids, oidx);
            r = rt_check_launch();
        }
        if (r != RT_OK) {
            rt_free(sort_blk, stream);
            return r;
        }
        rs.ray_ids = sids;
        job.out_index = oidx;
    }
    bool own = false;
    if (!work) {
        if (rt_alloc((void **)&work, sizeof(unsigned long long), stream) != RT_OK) {
            if (sort_blk) rt_free(sort_blk, stream);
            return RT_ERR_OOM;
        }
        own = true;
    }
    rt_status res = RT_OK;
    if (cudaMemsetAsync(work, 0, sizeof(unsigned long long), st) != cudaSuccess) res = RT_ERR_CUDA;
    if (res == RT_OK) {
        const int threads = 128;
        const bool count = aux.counters != nullptr;
#define RT_LAUNCH(S, C)                                                                     \
    do {                                                                                    \
        int grid = persistent_blocks((const void *)k_trace<S, C>, threads);                 \
        k_trace<S, C><<<grid, threads, 0, st>>>(b, rs, job, T_out, aux, work);              \
    } while (0)
        if (strat == 6) { if (count) RT_LAUNCH(6, true); else RT_LAUNCH(6, false); }
        else if (strat == 5) { if (count) RT_LAUNCH(5, true); else RT_LAUNCH(5, false); }
        else if (strat == 4) { if (count) RT_LAUNCH(4, true); else RT_LAUNCH(4, false); }
        else if (strat == 3) { if (count) RT_LAUNCH(3, true); else RT_LAUNCH(3, false); }
        else if (strat == 2) { if (count) RT_LAUNCH(2, true); else RT_LAUNCH(2, false); }
        else if (strat == 1) { if (count) RT_LAUNCH(1, true); else RT_LAUNCH(1, false); }
        else { if (count) RT_LAUNCH(0, true); else RT_LAUNCH(0, false); }
#undef RT_LAUNCH
        res = rt_check_launch();
    }
    if (own) rt_free(work, stream);
    if (sort_blk) rt_free(sort_blk, stream);
    return res;
}

// Trace the rays listed in ray_ids[0 .. *count) (device count, at most
// max_count) of an implicit set and write T_out[out_index[i]].
rt_status rt_trace_launch_list(const rt_bvh *bvh, const rt_rayspec *rays, const int64_t *ray_ids,
                               const int64_t *out_index, const unsigned long long *count, int64_t max_count,
                               float *T_out, rt_stream_t stream, unsigned long long *work) {
    if (rays->kind == RT_RAYS_EXPLICIT || !ray_ids || !out_index || !count || !work) return RT_ERR_INVALID_ARG;
    RaySetDev rs;
    int64_t c = 0;
    rt_rayspec tmp = *rays;
    tmp.ray_ids = nullptr;
    RT_TRY(rt_rayset_dev(bvh, &tmp, &rs, &c));
    rs.ray_ids = ray_ids;
    if (max_count <= 0) return RT_OK;
    TraceJob job;
    job.mode = MODE_IDS;
    job.out_index = out_index;
    job.dyn_count = count;
    job.n_out = max_count;
    job.n_tiles = 0;
    job.tile_base = 0;
    job.order_block = 1;
    job.n_items = (max_count + 31) / 32;
    TraceAux aux;
    memset(&aux, 0, sizeof(aux));
    aux.status = rt_status_ptr();
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(work, 0, sizeof(unsigned long long), st) != cudaSuccess) return RT_ERR_CUDA;
    const int threads = 128;
    // the listed rays are few and scattered: one warp per ray over the 4-wide
    // tree (its lanes expand the ray's nodes in parallel), which cuts the
    // latency of the longest traversal
    if (bvh->n_wide > 0) {
        int grid = persistent_blocks((const void *)k_trace<6, false>, threads);
        k_trace<6, false><<<grid, threads, 0, st>>>(bvh_dev(bvh), rs, job, T_out, aux, work);
    } else {
        int grid = persistent_blocks((const void *)k_trace<0, false>, threads);
        k_trace<0, false><<<grid, threads, 0, st>>>(bvh_dev(bvh), rs, job, T_out, aux, work);
    }
    return rt_check_launch();
}

extern "C" rt_status rt_trace_visibility(const rt_bvh *bvh, const rt_rayspec *rays, float *T_out,
                                         const rt_trace_opts *opts, rt_stream_t stream) {
    if (!bvh || !rays) return RT_ERR_INVALID_ARG;
    return rt_trace_launch(bvh, rays, T_out, opts, stream, nullptr);
}

extern "C" rt_status rt_trace_visibility_dirs(const rt_bvh *bvh, const float *dirs, int32_t k,
                                              float *T_out, const rt_trace_opts *opts,
                                              rt_stream_t stream) {
    if (!bvh) return RT_ERR_INVALID_ARG;
    rt_rayspec rs;
    memset(&rs, 0, sizeof(rs));
    rs.kind = RT_RAYS_DIRS;
    rs.n_dirs = k;
    rs.dirs = dirs;
    return rt_trace_launch(bvh, &rs, T_out, opts, stream, nullptr);
}

// ---------------------------------------------------------------------------
// The precompute from host buffers: copies in, build, trace, copy out, all on
// one stream.
// ---------------------------------------------------------------------------
extern "C" rt_status rt_visibility_dirs_host(const float *mean, const float *scale, const float *quat,
                                             const float *opacity, int64_t n, const float *dirs, int32_t k,
                                             const rt_params *params, const rt_trace_opts *opts, float *T_host,
                                             rt_stream_t stream) {
    if (n < 0 || k < 0 || n >= (int64_t(1) << 31)) return RT_ERR_INVALID_ARG;
    const int64_t R = n * (int64_t)k;
    if (R == 0) return RT_OK;
    if (R >= (int64_t(1) << 40) || !mean || !scale || !quat || !opacity || !dirs || !T_host)
        return RT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t b3 = up(size_t(n) * 12), b4 = up(size_t(n) * 16), b1 = up(size_t(n) * 4), bd = up(size_t(k) * 12);
    void *blk = nullptr;
    rt_status s = rt_alloc(&blk, 2 * b3 + b4 + b1 + bd, stream);
    if (s != RT_OK) return s;
    char *base = (char *)blk;
    float *d_mean = (float *)base, *d_scale = (float *)(base + b3), *d_quat = (float *)(base + 2 * b3),
          *d_opac = (float *)(base + 2 * b3 + b4), *d_dirs = (float *)(base + 2 * b3 + b4 + b1);
    const struct { void *dst; const void *src; size_t bytes; } in[5] = {
        {d_mean, mean, size_t(n) * 12}, {d_scale, scale, size_t(n) * 12}, {d_quat, quat, size_t(n) * 16},
        {d_opac, opacity, size_t(n) * 4}, {d_dirs, dirs, size_t(k) * 12}};
    for (const auto &c : in) {
        if (cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            cudaGetLastError();
            rt_free(blk, stream);
            return RT_ERR_CUDA;
        }
    }
    rt_bvh *bvh = nullptr;
    s = rt_build_bvh(d_mean, d_scale, d_quat, d_opac, n, params, stream, &bvh);
    if (s != RT_OK) {
        rt_free(blk, stream);
        return s;
    }
    float *d_T = nullptr;
    s = rt_alloc((void **)&d_T, size_t(R) * 4, stream);
    if (s == RT_OK) {
        s = rt_trace_visibility_dirs(bvh, d_dirs, k, d_T, opts, stream);
        if (s == RT_OK && cudaMemcpyAsync(T_host, d_T, size_t(R) * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
            cudaGetLastError();
            s = RT_ERR_CUDA;
        }
        rt_free(d_T, stream);
    }
    rt_bvh_destroy(bvh, stream);
    rt_free(blk, stream);
    return s;
}

// ---------------------------------------------------------------------------
// Materialised rays of an implicit set (for inspection and the adjoint)
// ---------------------------------------------------------------------------
namespace {
__global__ void k_materialize(BvhDev b, RaySetDev rs, const int64_t *ids, int64_t m, float *ro,
                              float *rd, int32_t *rsrc, int *status) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t rid = ids[i];
        if (rid < 0 || rid >= rs.n_rays) {
            rt_set_error(status, RT_ERR_INVALID_ARG);
            continue;
        }
        int64_t g = rid / rs.K;
        int32_t k = (int32_t)(rid - g * rs.K);
        int32_t p = b.rank[g];
        float3 o, d;
        implicit_ray(rs, rid, k, g, __ldg(b.gauss + 4 * (int64_t)p), o, d);
        ro[3 * i] = o.x; ro[3 * i + 1] = o.y; ro[3 * i + 2] = o.z;
        rd[3 * i] = d.x; rd[3 * i + 1] = d.y; rd[3 * i + 2] = d.z;
        if (rsrc) rsrc[i] = (int32_t)g;
    }
}
}  // namespace

extern "C" rt_status rt_materialize_rays(const rt_bvh *bvh, const rt_rayspec *rays,
                                         const int64_t *ray_ids, int64_t m, float *ray_o,
                                         float *ray_d, int32_t *ray_src, rt_stream_t stream) {
    if (!bvh || !rays || m < 0) return RT_ERR_INVALID_ARG;
    if (rays->kind == RT_RAYS_EXPLICIT) return RT_ERR_INVALID_ARG;
    if (m == 0) return RT_OK;
    if (!ray_ids || !ray_o || !ray_d) return RT_ERR_INVALID_ARG;
    RaySetDev rs;
    int64_t c;
    rt_rayspec tmp = *rays;
    tmp.ray_ids = nullptr;
    RT_TRY(rt_rayset_dev(bvh, &tmp, &rs, &c));
    int grid = (int)((m + 255) / 256);
    if (grid > rt_num_sms() * 8) grid = rt_num_sms() * 8;
    k_materialize<<<grid, 256, 0, (cudaStream_t)stream>>>(bvh_dev(bvh), rs, ray_ids, m, ray_o, ray_d,
                                                          ray_src, rt_status_ptr());
    return rt_check_launch();
}
