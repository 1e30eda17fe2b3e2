// rt_api.cu -- status handling, parameters, allocation, environment maps and
// ray-set validation for the C ABI declared in include/rt3dg.h.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>

#include "rt_internal.cuh"

static __device__ int g_rt_status = 0;

int *rt_status_ptr() {
    static int *ptr = nullptr;
    static int dev_cached = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (!ptr || dev != dev_cached) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_rt_status) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        ptr = (int *)p;
        dev_cached = dev;
    }
    return ptr;
}

extern "C" void rt_params_default(rt_params *p) {
    if (!p) return;
    p->k_sigma = 3.0f;
    p->alpha_min = 1.0f / 255.0f;
    p->t_min = 1e-4f;
    p->origin_eps = 1e-4f;
    p->box_mode = 0;
    p->deterministic = 0;
}

extern "C" const char *rt_status_string(rt_status s) {
    switch (s) {
        case RT_OK: return "ok";
        case RT_ERR_INVALID_ARG: return "invalid argument";
        case RT_ERR_OOM: return "device allocation failed";
        case RT_ERR_CUDA: return "CUDA runtime error";
        case RT_ERR_STACK_OVERFLOW: return "traversal stack overflow";
        case RT_ERR_HITLOG_OVERFLOW: return "hit log capacity exceeded";
        case RT_ERR_TIMEOUT: return "bounded device wait timed out";
        case RT_ERR_NOT_TRAINED: return "surrogate not trained";
        case RT_ERR_UNSUPPORTED: return "unsupported option";
        case RT_ERR_RANGE: return "value outside the fixed-point range";
    }
    return "unknown status";
}

extern "C" rt_status rt_status_last(void) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_rt_status, sizeof(int)) != cudaSuccess) return RT_ERR_CUDA;
    return (rt_status)v;
}

extern "C" rt_status rt_status_clear(void) {
    int z = 0;
    if (cudaMemcpyToSymbol(g_rt_status, &z, sizeof(int)) != cudaSuccess) return RT_ERR_CUDA;
    return RT_OK;
}

rt_status rt_check_launch() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RT_OK : RT_ERR_CUDA;
}

namespace {
rt_allocator g_alloc = {nullptr, nullptr, nullptr};  // alloc == null: the library's pool

// The library's own stream-ordered pool per device.  Its release threshold is
// unbounded, so blocks freed in stream order stay mapped for the next call
// (the device's default pool would hand them back to the CUDA driver at every
// synchronisation and remap them on the next allocation); rt_memory_trim
// returns them.
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};

cudaMemPool_t pool_for_current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> g(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = ~uint64_t(0);
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool[dev] = pool;
    }
    return g_pool[dev];
}
}  // namespace

extern "C" rt_status rt_memory_trim(int64_t keep_bytes) {
    if (keep_bytes < 0) return RT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(g_pool_mu);
    for (int d = 0; d < kMaxDevices; ++d)
        if (g_pool[d] && cudaMemPoolTrimTo(g_pool[d], (size_t)keep_bytes) != cudaSuccess) {
            cudaGetLastError();
            return RT_ERR_CUDA;
        }
    return RT_OK;
}

extern "C" rt_status rt_set_allocator(const rt_allocator *a) {
    if (a && (!a->alloc || !a->free)) return RT_ERR_INVALID_ARG;
    if (a) g_alloc = *a;
    else g_alloc = rt_allocator{nullptr, nullptr, nullptr};
    return RT_OK;
}

rt_status rt_alloc(void **p, size_t bytes, rt_stream_t s) {
    *p = nullptr;
    if (bytes == 0) bytes = 256;
    if (g_alloc.alloc) {
        *p = g_alloc.alloc(bytes, s, g_alloc.ctx);
        if (!*p || ((uintptr_t)*p & 255u)) {  // the layouts need 256-byte alignment
            if (*p) g_alloc.free(*p, s, g_alloc.ctx);
            *p = nullptr;
            return RT_ERR_OOM;
        }
        return RT_OK;
    }
    cudaMemPool_t pool = pool_for_current_device();
    cudaError_t e = pool ? cudaMallocFromPoolAsync(p, bytes, pool, (cudaStream_t)s)
                         : cudaMallocAsync(p, bytes, (cudaStream_t)s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return RT_ERR_OOM;
    }
    return RT_OK;
}

void rt_free(void *p, rt_stream_t s) {
    if (!p) return;
    if (g_alloc.free) g_alloc.free(p, s, g_alloc.ctx);
    else cudaFreeAsync(p, (cudaStream_t)s);
}

int rt_num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

// ---------------------------------------------------------------------------
// Environment map: float64 CDF built on the host in index order.
// ---------------------------------------------------------------------------
extern "C" rt_status rt_envmap_create(const double *radiance, const double *solid_angle,
                                      const float *corners, int32_t h, int32_t w,
                                      rt_stream_t stream, rt_envmap **out) {
    if (!out || !radiance || !solid_angle || !corners || h <= 0 || w <= 0 || h > 4096 || w > 4096)
        return RT_ERR_INVALID_ARG;
    *out = nullptr;
    const int64_t np = (int64_t)h * w;
    double *cdf = (double *)malloc(sizeof(double) * np);
    if (!cdf) return RT_ERR_OOM;
    double run = 0.0;
    for (int64_t p = 0; p < np; ++p) {
        double wgt = radiance[p] * solid_angle[p];
        if (!(wgt >= 0.0) || !isfinite(wgt)) {
            free(cdf);
            return RT_ERR_INVALID_ARG;
        }
        run += wgt;
        cdf[p] = run;
    }
    if (!(run > 0.0)) {
        free(cdf);
        return RT_ERR_INVALID_ARG;
    }
    for (int64_t p = 0; p < np; ++p) cdf[p] = cdf[p] / run;
    rt_envmap *env = new rt_envmap();
    env->h = h;
    env->w = w;
    size_t cdf_bytes = (sizeof(double) * np + 255) & ~(size_t)255;
    size_t cor_bytes = sizeof(float) * (size_t)(h + 1) * (w + 1) * 3;
    rt_status st = rt_alloc(&env->block, cdf_bytes + cor_bytes, stream);
    if (st != RT_OK) {
        free(cdf);
        delete env;
        return st;
    }
    env->cdf = (double *)env->block;
    env->corners = (float *)((char *)env->block + cdf_bytes);
    cudaError_t e1 = cudaMemcpyAsync(env->cdf, cdf, sizeof(double) * np, cudaMemcpyHostToDevice,
                                     (cudaStream_t)stream);
    cudaError_t e2 = cudaMemcpyAsync(env->corners, corners, cor_bytes, cudaMemcpyHostToDevice,
                                     (cudaStream_t)stream);
    // the host staging buffer must outlive the copies
    cudaError_t e3 = cudaStreamSynchronize((cudaStream_t)stream);
    free(cdf);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        rt_free(env->block, stream);
        delete env;
        return RT_ERR_CUDA;
    }
    *out = env;
    return RT_OK;
}

extern "C" rt_status rt_envmap_destroy(rt_envmap *env, rt_stream_t stream) {
    if (!env) return RT_ERR_INVALID_ARG;
    rt_free(env->block, stream);
    delete env;
    return RT_OK;
}

// ---------------------------------------------------------------------------
// Ray sets
// ---------------------------------------------------------------------------
rt_status rt_rayset_dev(const rt_bvh *bvh, const rt_rayspec *rays, RaySetDev *out, int64_t *count) {
    if (!bvh) return RT_ERR_INVALID_ARG;
    return rt_rayset_dev_n(bvh->n, bvh->params.origin_eps, rays, out, count);
}

rt_status rt_rayset_dev_n(int64_t n, float origin_eps, const rt_rayspec *rays, RaySetDev *out, int64_t *count) {
    if (!rays || !out || n < 0) return RT_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    out->kind = rays->kind;
    out->eps = origin_eps;
    out->seed = rays->seed;
    int64_t cnt = -1;
    switch (rays->kind) {
        case RT_RAYS_EXPLICIT:
            if (rays->n_rays < 0) return RT_ERR_INVALID_ARG;
            if (rays->n_rays > 0 && (!rays->ray_o || !rays->ray_d)) return RT_ERR_INVALID_ARG;
            if (rays->ray_ids) return RT_ERR_UNSUPPORTED;
            out->n_rays = rays->n_rays;
            out->ray_o = rays->ray_o;
            out->ray_d = rays->ray_d;
            out->ray_src = rays->ray_src;
            cnt = rays->n_rays;
            break;
        case RT_RAYS_DIRS:
            if (rays->n_dirs <= 0 || !rays->dirs) return RT_ERR_INVALID_ARG;
            out->K = rays->n_dirs;
            out->dirs = rays->dirs;
            cnt = n * rays->n_dirs;
            break;
        case RT_RAYS_HEMI:
            if (rays->n_dirs <= 0 || !rays->dirs || (n > 0 && !rays->normals)) return RT_ERR_INVALID_ARG;
            out->K = rays->n_dirs;
            out->dirs = rays->dirs;
            out->normals = rays->normals;
            cnt = n * rays->n_dirs;
            break;
        case RT_RAYS_ENV:
            if (rays->n_dirs <= 0 || !rays->env) return RT_ERR_INVALID_ARG;
            out->K = rays->n_dirs;
            out->env_cdf = rays->env->cdf;
            out->env_corners = rays->env->corners;
            out->env_h = rays->env->h;
            out->env_w = rays->env->w;
            cnt = n * rays->n_dirs;
            break;
        default:
            return RT_ERR_INVALID_ARG;
    }
    out->n_rays = cnt;
    if (rays->kind != RT_RAYS_EXPLICIT && rays->ray_ids) {
        if (rays->n_ids < 0) return RT_ERR_INVALID_ARG;
        out->ray_ids = rays->ray_ids;
        cnt = rays->n_ids;
    }
    if (count) *count = cnt;
    return RT_OK;
}

extern "C" int64_t rt_rayspec_count(const rt_bvh *bvh, const rt_rayspec *rays) {
    RaySetDev d;
    int64_t c = -1;
    if (rt_rayset_dev(bvh, rays, &d, &c) != RT_OK) return -1;
    return c;
}
