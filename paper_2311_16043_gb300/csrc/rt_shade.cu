// rt_shade.cu -- consumers of the visibility: the per-Gaussian PBR colour of
// Eq. 10 (Sec. 3.3) and ambient occlusion.
//
// Sec. 3.3 computes a PBR colour per Gaussian by summing the rendering
// equation over N_s hemisphere directions about the Gaussian's normal, with
// the incident light of Eq. 8 (visibility x a global environment map plus
// per-Gaussian SH indirect light) and the simplified Disney BRDF of Eq. 9;
// Sec. 4.2 precomputes the visibility of those directions.  Two forms:
//   - from a visibility table V[n, K] (the paper's order: precompute once,
//     shade every iteration): one thread per Gaussian, HBM/ALU bound;
//   - fused: one warp per 32 Morton-adjacent Gaussians traces all K rays of
//     each and shades in the epilogue, so V is never written.
// Ambient occlusion is the fused form with the mean of T as the epilogue.
// The shading arithmetic is one function, so both forms give the same bits
// for the same T.
#include <string.h>

#include "rt_trace_core.cuh"

namespace {

constexpr int kMaxEnvTexels = 2048;  // RGB map staged in shared memory (24 KB)
constexpr float kPi = 3.14159265358979f;
constexpr float kF0 = 0.04f;
constexpr float kRoughMin = 0.04f;
// Default traversal of hemisphere sets in the fused kernels: one thread per
// ray over the 4-wide tree (measured faster than the warp packet on the 2M
// object scene, where the lanes' k-th directions differ with the normals).
constexpr int kHemiStrat = 4;

struct ShadeDev {
    const float *albedo, *rough, *sh, *env;
    const float *normals, *hemi;
    int32_t env_h, env_w, K;
    float3 cam;
};

__device__ __forceinline__ float dot3f(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Bilinear lookup between pixel centres of the equirectangular map (row i:
// polar angles [i pi/h, (i+1) pi/h]; azimuth wraps, polar angle clamps).
__device__ __forceinline__ void env_lookup(const float *env, int h, int w, float3 d, float L[3]) {
    const float z = fminf(fmaxf(d.z, -1.0f), 1.0f);
    const float th = acosf(z);
    float ph = atan2f(d.y, d.x);
    if (ph < 0.0f) ph += 2.0f * kPi;
    const float v = th / kPi * (float)h - 0.5f, u = ph / (2.0f * kPi) * (float)w - 0.5f;
    const float fv = floorf(v), fu = floorf(u);
    const float bv = v - fv, bu = u - fu;
    int i0 = (int)fv, j0 = (int)fu;
    int i1 = i0 + 1, j1 = j0 + 1;
    i0 = min(max(i0, 0), h - 1);
    i1 = min(max(i1, 0), h - 1);
    j0 = ((j0 % w) + w) % w;
    j1 = ((j1 % w) + w) % w;
    const float *e00 = env + 3 * (i0 * w + j0), *e01 = env + 3 * (i0 * w + j1);
    const float *e10 = env + 3 * (i1 * w + j0), *e11 = env + 3 * (i1 * w + j1);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float a = e00[c] * (1.0f - bu) + e01[c] * bu;
        const float b = e10[c] * (1.0f - bu) + e11[c] * bu;
        L[c] = a * (1.0f - bv) + b * bv;
    }
}

// Specular term of Eq. 9: D F G / (4 (n.wi)(n.wo)) with GGX D (alpha = r^2),
// Schlick F (F0 = 0.04) and Smith-Schlick G (k = (r+1)^2/8), written with
// G1(x)/x = 1/(x(1-k)+k) so it stays finite at grazing angles.  The GGX
// denominator 1 + (n.h)^2 (alpha^2 - 1) is evaluated as |n x h|^2 +
// (n.h)^2 alpha^2, which has no cancellation near the mirror direction.
__device__ __forceinline__ float spec_term(float3 n, float3 wi, float3 wo, float r, float nl, float nv) {
    const float3 hv = make_float3(wi.x + wo.x, wi.y + wo.y, wi.z + wo.z);
    const float hl2 = dot3f(hv, hv);
    if (!(hl2 > 0.0f)) return 0.0f;
    const float inv = rsqrtf(hl2);
    const float3 h = make_float3(hv.x * inv, hv.y * inv, hv.z * inv);
    const float nh = dot3f(n, h), vh = fmaxf(dot3f(wo, h), 0.0f);
    const float3 cr = make_float3(n.y * h.z - n.z * h.y, n.z * h.x - n.x * h.z, n.x * h.y - n.y * h.x);
    const float al = r * r, a2 = al * al;
    const float q = dot3f(cr, cr) + nh * nh * a2;
    const float D = a2 / (kPi * q * q);
    const float m = 1.0f - vh, m2 = m * m;
    const float F = kF0 + (1.0f - kF0) * (m2 * m2 * m);
    const float k = (r + 1.0f) * (r + 1.0f) * 0.125f;
    const float gl = 1.0f / (nl * (1.0f - k) + k), gv = 1.0f / (nv * (1.0f - k) + k);
    return 0.25f * D * F * gl * gv;
}

// Per-Gaussian constants of the shading sum.
struct ShadeLane {
    float3 n, wo, alb;
    float r;
    const float *sh;  // 27 coefficients or null
};

__device__ __forceinline__ ShadeLane shade_lane(const ShadeDev &S, const HemiFrame &f, int64_t g, float4 mu) {
    ShadeLane L;
    L.n = f.n;
    float3 wo = make_float3(S.cam.x - mu.x, S.cam.y - mu.y, S.cam.z - mu.z);
    const float il = rsqrtf(dot3f(wo, wo));
    L.wo = make_float3(wo.x * il, wo.y * il, wo.z * il);
    L.alb = make_float3(__ldg(S.albedo + 3 * g), __ldg(S.albedo + 3 * g + 1), __ldg(S.albedo + 3 * g + 2));
    L.r = fminf(fmaxf(__ldg(S.rough + g), kRoughMin), 1.0f);
    L.sh = S.sh ? S.sh + 27 * g : nullptr;
    return L;
}

// One term of Eq. 10: acc += (b/pi + f_s) (V L_direct + max(0, SH)) max(n.wi, 0).
__device__ __forceinline__ void shade_add(const ShadeDev &S, const float *env, const ShadeLane &L, float3 wi,
                                          float V, float acc[3]) {
    const float nl = fmaxf(dot3f(L.n, wi), 0.0f), nv = fmaxf(dot3f(L.n, L.wo), 0.0f);
    const float fs = spec_term(L.n, wi, L.wo, L.r, nl, nv);
    float Ld[3];
    env_lookup(env, S.env_h, S.env_w, wi, Ld);
    float Li[3] = {0.0f, 0.0f, 0.0f};
    if (L.sh) {
        const float c0 = 0.282094791773878f, c1 = 0.488602511902920f, c2a = 1.092548430592079f,
                    c2b = 0.315391565252520f, c2c = 0.546274215296040f;
        const float x = wi.x, y = wi.y, z = wi.z;
        const float Y[9] = {c0, -c1 * y, c1 * z, -c1 * x, c2a * x * y, -c2a * y * z,
                            c2b * (2.0f * z * z - x * x - y * y), -c2a * x * z, c2c * (x * x - y * y)};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float s = 0.0f;
#pragma unroll
            for (int j = 0; j < 9; ++j) s += __ldg(L.sh + 3 * j + c) * Y[j];
            Li[c] = fmaxf(s, 0.0f);
        }
    }
    const float alb[3] = {L.alb.x, L.alb.y, L.alb.z};
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[c] += (alb[c] * (1.0f / kPi) + fs) * (V * Ld[c] + Li[c]) * nl;
}

__device__ __forceinline__ void load_env(const ShadeDev &S, float *env_s) {
    const int nf = 3 * S.env_h * S.env_w;
    for (int i = threadIdx.x; i < nf; i += blockDim.x) env_s[i] = __ldg(S.env + i);
    __syncthreads();
}

// Shading from a visibility table: one thread per Gaussian (original order).
__global__ void __launch_bounds__(128) k_pbr_shade_v(BvhDev b, ShadeDev S, const float *__restrict__ V,
                                                     float *__restrict__ rgb) {
    extern __shared__ float env_s[];
    load_env(S, env_s);
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < b.n;
         g += (int64_t)gridDim.x * blockDim.x) {
        const float4 mu = __ldg(b.gauss + 4 * (int64_t)b.rank[g]);
        const HemiFrame f = hemi_frame(S.normals + 3 * g);
        const ShadeLane L = shade_lane(S, f, g, mu);
        float acc[3] = {0.0f, 0.0f, 0.0f};
        const float *Vg = V + g * S.K;
        for (int k = 0; k < S.K; ++k) shade_add(S, env_s, L, hemi_rotate(f, S.hemi + 3 * k), __ldg(Vg + k), acc);
        const float w = 2.0f * kPi / (float)S.K;
        rgb[3 * g] = acc[0] * w;
        rgb[3 * g + 1] = acc[1] * w;
        rgb[3 * g + 2] = acc[2] * w;
    }
}

// Fused trace + reduction over all K rays of each Gaussian.  An item is a
// tile of 32 Morton-adjacent Gaussians; the warp traces ray k of all 32
// lanes together (STRAT 2/3: warp packet over the 4-wide tree, 3 when the
// direction is shared; 4: one thread per ray) for k = 0..K-1.
// MODE 0: PBR colour (Eq. 10); MODE 1: ambient occlusion (mean of T).
template <int STRAT, int MODE>
__global__ void __launch_bounds__(128, 8) k_trace_reduce(BvhDev b, RaySetDev rs, ShadeDev S, float *__restrict__ out,
                                                         int *status, unsigned long long *work) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    __shared__ int2 stk_all[(STRAT == 2 || STRAT == 3) ? 4 * RT_WIDE_STACK : 1];
    int2 *stk = stk_all + ((STRAT == 2 || STRAT == 3) ? (threadIdx.x >> 5) * RT_WIDE_STACK : 0);
    extern __shared__ float env_s[];
    if (MODE == 0) load_env(S, env_s);
    const int64_t n_tiles = (b.n + 31) / 32;
    WorkCounts wc = {0, 0, 0};
    LaneLog lg;
    lg.ids = nullptr;
    lg.cap = 0;
    lg.count = 0;
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(work, 1ull);
        item = __shfl_sync(FULL, item, 0);
        if ((int64_t)item >= n_tiles) break;
        const int64_t p = (int64_t)item * 32 + lane;
        const bool valid = p < b.n;
        float4 mu = make_float4(0.f, 0.f, 0.f, 0.f);
        int64_t g = 0;
        if (valid) {
            mu = __ldg(b.gauss + 4 * p);
            g = __float_as_int(__ldg(b.gauss + 4 * p + 1).w);
        }
        float acc[3] = {0.0f, 0.0f, 0.0f};
        for (int32_t k = 0; k < rs.K; ++k) {
            float3 o = make_float3(0.f, 0.f, 0.f), d = make_float3(0.f, 0.f, 1.f);
            if (valid) implicit_ray(rs, g * rs.K + k, k, g, mu, o, d);
            const int32_t src = valid ? (int32_t)p : -1;
            float T;
            if (STRAT == 4) T = valid ? trace_ray_wide<false>(b, o, d, src, lg, wc, status, far_first(rs)) : 1.0f;
            else T = trace_wide<false, STRAT == 3>(b, o, d, src, valid, lg, wc, status, stk);
            if (!valid) continue;
            if (MODE == 0) {
                // the per-Gaussian constants are rebuilt after each traversal
                // (a few dozen instructions and L1 hits) so that they hold no
                // registers across it
                const float4 m2 = __ldg(b.gauss + 4 * p);
                shade_add(S, env_s, shade_lane(S, hemi_frame(S.normals + 3 * g), g, m2), d, T, acc);
            } else {
                acc[0] += T;
            }
        }
        if (!valid) continue;
        if (MODE == 0) {
            const float w = 2.0f * kPi / (float)rs.K;
            out[3 * g] = acc[0] * w;
            out[3 * g + 1] = acc[1] * w;
            out[3 * g + 2] = acc[2] * w;
        } else {
            out[g] = acc[0] / (float)rs.K;
        }
    }
}

int grid_for(const void *kernel, int threads, size_t smem) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return per_sm * rt_num_sms();
}

rt_status shade_dev(const rt_bvh *bvh, const rt_rayspec *rays, const rt_pbr_inputs *in, RaySetDev *rs,
                    ShadeDev *S) {
    if (!bvh || !rays || !in || rays->kind != RT_RAYS_HEMI || rays->ray_ids) return RT_ERR_INVALID_ARG;
    int64_t count = 0;
    RT_TRY(rt_rayset_dev(bvh, rays, rs, &count));
    if (in->env_h <= 0 || in->env_w <= 0 || (int64_t)in->env_h * in->env_w > kMaxEnvTexels || !in->env)
        return RT_ERR_INVALID_ARG;
    if (bvh->n > 0 && (!in->albedo || !in->roughness)) return RT_ERR_INVALID_ARG;
    memset(S, 0, sizeof(*S));
    S->albedo = in->albedo;
    S->rough = in->roughness;
    S->sh = in->sh;
    S->env = in->env;
    S->env_h = in->env_h;
    S->env_w = in->env_w;
    S->normals = rays->normals;
    S->hemi = rays->dirs;
    S->K = rays->n_dirs;
    S->cam = make_float3(in->cam[0], in->cam[1], in->cam[2]);
    return RT_OK;
}

// strat: 2 warp packet (per-lane directions), 3 warp packet with a shared
// direction (DIRS), 4 one thread per ray; all over the 4-wide tree.
template <int MODE>
rt_status launch_reduce(const rt_bvh *bvh, const RaySetDev &rs, const ShadeDev &S, float *out, size_t smem,
                        int strat, cudaStream_t st) {
    unsigned long long *work = nullptr;
    RT_TRY(rt_alloc((void **)&work, sizeof(unsigned long long), st));
    rt_status res = RT_OK;
    if (cudaMemsetAsync(work, 0, sizeof(unsigned long long), st) != cudaSuccess) res = RT_ERR_CUDA;
    const BvhDev b = bvh_dev(bvh);
    if (res == RT_OK) {
#define RT_REDUCE(ST)                                                                     \
    do {                                                                                  \
        const int grid = grid_for((const void *)k_trace_reduce<ST, MODE>, 128, smem);     \
        k_trace_reduce<ST, MODE><<<grid, 128, smem, st>>>(b, rs, S, out, rt_status_ptr(), work); \
        res = rt_check_launch();                                                          \
    } while (0)
        // a tree of fewer than 2 Gaussians has no 4-wide form: strategy 4
        // handles it without touching one
        if (b.wide == nullptr && b.n >= 2) res = RT_ERR_UNSUPPORTED;
        else if (b.wide == nullptr) RT_REDUCE(4);
        else if (strat == 3) RT_REDUCE(3);
        else if (strat == 2) RT_REDUCE(2);
        else RT_REDUCE(4);
#undef RT_REDUCE
    }
    rt_free(work, st);
    return res;
}

}  // namespace

extern "C" rt_status rt_pbr_shade(const rt_bvh *bvh, const rt_rayspec *rays, const float *V,
                                  const rt_pbr_inputs *in, float *rgb, rt_stream_t stream) {
    RaySetDev rs;
    ShadeDev S;
    RT_TRY(shade_dev(bvh, rays, in, &rs, &S));
    if (in->kernel != RT_KERNEL_AUTO && in->kernel != RT_KERNEL_WIDE && in->kernel != RT_KERNEL_RAY_WIDE)
        return RT_ERR_INVALID_ARG;
    if (bvh->n == 0) return RT_OK;
    if (!rgb) return RT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t smem = sizeof(float) * 3 * (size_t)S.env_h * S.env_w;
    if (V) {
        const int grid = grid_for((const void *)k_pbr_shade_v, 128, smem);
        k_pbr_shade_v<<<grid, 128, smem, st>>>(bvh_dev(bvh), S, V, rgb);
        return rt_check_launch();
    }
    const int strat = in->kernel == RT_KERNEL_WIDE ? 2 : in->kernel == RT_KERNEL_RAY_WIDE ? 4 : kHemiStrat;
    return launch_reduce<0>(bvh, rs, S, rgb, smem, strat, st);
}

extern "C" rt_status rt_trace_ao(const rt_bvh *bvh, const rt_rayspec *rays, const rt_trace_opts *opts, float *ao,
                                 rt_stream_t stream) {
    const int kernel = opts ? opts->kernel : RT_KERNEL_AUTO;
    if (kernel != RT_KERNEL_AUTO && kernel != RT_KERNEL_WIDE && kernel != RT_KERNEL_RAY_WIDE) return RT_ERR_INVALID_ARG;
    if (!bvh || !rays || rays->ray_ids || (rays->kind != RT_RAYS_DIRS && rays->kind != RT_RAYS_HEMI))
        return RT_ERR_INVALID_ARG;
    RaySetDev rs;
    int64_t count = 0;
    RT_TRY(rt_rayset_dev(bvh, rays, &rs, &count));
    if (bvh->n == 0) return RT_OK;
    if (!ao) return RT_ERR_INVALID_ARG;
    ShadeDev S;
    memset(&S, 0, sizeof(S));
    int strat = rays->kind == RT_RAYS_DIRS ? 3 : kHemiStrat;
    if (kernel == RT_KERNEL_WIDE) strat = rays->kind == RT_RAYS_DIRS ? 3 : 2;
    if (kernel == RT_KERNEL_RAY_WIDE) strat = 4;
    return launch_reduce<1>(bvh, rs, S, ao, 0, strat, (cudaStream_t)stream);
}
