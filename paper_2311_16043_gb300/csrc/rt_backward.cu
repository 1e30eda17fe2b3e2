// rt_backward.cu -- adjoint of the visibility trace.
//
// For a ray with final transmittance T = prod_j (1 - alpha_j) and upstream
// gradient g = dL/dT, each accepted Gaussian j receives
//   dL/dalpha_j = -g T / (1 - alpha_j),
//   alpha = o exp(-m^2/2):  dalpha/do = exp(-m^2/2),  dalpha/dm^2 = -alpha/2.
// m^2 is stationary in t at the peak t*, so with the peak point held fixed and
// e = x(t*) - mu, u = S^-1 R^T e, w = S^-1 u:
//   dm^2/dmu = -2 R w,  dm^2/dorigin = +2 R w,  dm^2/ds_k = -2 u_k^2 / s_k,
//   dm^2/dR_ck = 2 e_c w_k, then through R(q/|q|) to the raw quaternion.
// Rays cast from a Gaussian (DIRS / ENV sets) start at mu_src + eps d, so
// their origin gradient is added to the source Gaussian's mean.
// Hits are replayed from the forward's hit log when it is complete for the
// ray, otherwise found again by traversal (same code path as the forward, so
// the same accepted set).  Rays the forward snapped to T = 0 have zero
// gradient.
// Accumulation: float32 atomics into the caller's arrays, or (params
// deterministic = 1) integer atomics on 64-bit fixed point with 2^-32
// resolution, one accumulator per parameter component, added to the caller's
// arrays afterwards: integer addition is associative, so the result does not
// depend on the order in which rays finish.
#include "rt_trace_core.cuh"

namespace {

struct GradOut {
    float *d_mean, *d_scale, *d_quat, *d_opacity, *d_ray_o;
    const float *mean, *scale, *quat, *opacity;
    long long *fx;  // deterministic mode: [n][kFxPer] fixed-point accumulators
    int *status;
};

// Fixed-point layout per Gaussian: mean 0-2, scale 3-5, quat 6-9, opacity 10.
constexpr int kFxPer = 11;
constexpr float kFxScale = 4294967296.0f;  // 2^32

// v * 2^32 rounded to the nearest integer, added with an integer atomic; a
// value or a sum outside the signed 64-bit range records RT_ERR_RANGE.
__device__ __forceinline__ void fx_add(long long *p, float v, int *status) {
    const float s = v * kFxScale;  // exact: a power of two
    if (!(fabsf(s) < 9.2e18f)) {   // also NaN
        rt_set_error(status, RT_ERR_RANGE);
        return;
    }
    const long long q = __float2ll_rn(s);
    const unsigned long long old = atomicAdd((unsigned long long *)p, (unsigned long long)q);
    const long long o = (long long)old, sum = (long long)(old + (unsigned long long)q);
    if (((o ^ sum) & (q ^ sum)) < 0) rt_set_error(status, RT_ERR_RANGE);
}

template <bool DET>
__device__ __forceinline__ void grad_add(const GradOut &G, float *dst, int64_t i, int slot, float v) {
    if (DET) fx_add(G.fx + i * kFxPer + slot, v, G.status);
    else atomicAdd(dst, v);
}

// Peak point for the gradient: e = x(t*) - mu and alpha with IEEE division
// and exponential.  dm^2/dmu = -2 Sigma^-1 e is first order in e, so t* must
// be accurate here (the forward's accept decision tolerates a fast
// reciprocal because m^2 itself is stationary in t).
__device__ __forceinline__ void peak_accurate(const BvhDev &b, int32_t p, float3 o, float3 d, float &alpha,
                                              float3 &e) {
    const float4 g0 = __ldg(b.gauss + 4 * p);
    const float4 g1 = __ldg(b.gauss + 4 * p + 1);
    const float4 g2 = __ldg(b.gauss + 4 * p + 2);
    const float4 g3 = __ldg(b.gauss + 4 * p + 3);
    float hx, lx, hy, ly, hz, lz;
    two_diff(o.x, g0.x, hx, lx);
    two_diff(o.y, g0.y, hy, ly);
    two_diff(o.z, g0.z, hz, lz);
    const float3 w0 = make_float3(g1.x, g1.y, g1.z);
    const float3 w1 = make_float3(g2.x, g2.y, g2.z);
    const float3 w2 = make_float3(g3.x, g3.y, g3.z);
    const float3 dh = make_float3(hx, hy, hz);
    const float3 ud = make_float3(dot3(w0, d), dot3(w1, d), dot3(w2, d));
    const float3 uo = make_float3(dot3(w0, dh), dot3(w1, dh), dot3(w2, dh));
    const float t = -dot3(uo, ud) / dot3(ud, ud);
    e = make_float3(fmaf(t, d.x, hx) + lx, fmaf(t, d.y, hy) + ly, fmaf(t, d.z, hz) + lz);
    const float3 u = make_float3(dot3(w0, e), dot3(w1, e), dot3(w2, e));
    alpha = g0.w * expf(-0.5f * dot3(u, u));
}

// Gradient contribution of one accepted hit (Gaussian with original index i).
template <bool DET>
__device__ __forceinline__ void hit_grad(const GradOut &G, int32_t i, float gT, float T, float alpha,
                                         float3 e, float3 &d_origin) {
    const float qw0 = G.quat[4 * i], qx0 = G.quat[4 * i + 1], qy0 = G.quat[4 * i + 2], qz0 = G.quat[4 * i + 3];
    const float qn = sqrtf(qw0 * qw0 + qx0 * qx0 + qy0 * qy0 + qz0 * qz0);
    const float w = qw0 / qn, x = qx0 / qn, y = qy0 / qn, z = qz0 / qn;
    float R[3][3];
    R[0][0] = 1.f - 2.f * (y * y + z * z); R[0][1] = 2.f * (x * y - w * z); R[0][2] = 2.f * (x * z + w * y);
    R[1][0] = 2.f * (x * y + w * z); R[1][1] = 1.f - 2.f * (x * x + z * z); R[1][2] = 2.f * (y * z - w * x);
    R[2][0] = 2.f * (x * z - w * y); R[2][1] = 2.f * (y * z + w * x); R[2][2] = 1.f - 2.f * (x * x + y * y);
    const float s[3] = {G.scale[3 * i], G.scale[3 * i + 1], G.scale[3 * i + 2]};
    const float ec[3] = {e.x, e.y, e.z};
    float u[3], wv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        u[k] = (R[0][k] * ec[0] + R[1][k] * ec[1] + R[2][k] * ec[2]) / s[k];
        wv[k] = u[k] / s[k];
    }
    float sie[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) sie[c] = R[c][0] * wv[0] + R[c][1] * wv[1] + R[c][2] * wv[2];
    const float gA = gT * (-T / (1.0f - alpha));  // dL/dalpha
    const float ex = alpha / G.opacity[i];        // exp(-m^2/2)
    const float gM = gA * (-0.5f * alpha);        // dL/dm^2
    grad_add<DET>(G, G.d_opacity + i, i, 10, gA * ex);
#pragma unroll
    for (int c = 0; c < 3; ++c) grad_add<DET>(G, G.d_mean + 3 * i + c, i, c, -2.0f * gM * sie[c]);
#pragma unroll
    for (int k = 0; k < 3; ++k) grad_add<DET>(G, G.d_scale + 3 * i + k, i, 3 + k, -2.0f * gM * u[k] * u[k] / s[k]);
    float Gm[9];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 3; ++k) Gm[3 * c + k] = 2.0f * gM * ec[c] * wv[k];
    const float gw = 2.f * (-z * Gm[1] + y * Gm[2] + z * Gm[3] - x * Gm[5] - y * Gm[6] + x * Gm[7]);
    const float gx = 2.f * (y * Gm[1] + z * Gm[2] + y * Gm[3] - 2.f * x * Gm[4] - w * Gm[5] + z * Gm[6] + w * Gm[7] - 2.f * x * Gm[8]);
    const float gy = 2.f * (-2.f * y * Gm[0] + x * Gm[1] + w * Gm[2] + x * Gm[3] + z * Gm[5] - w * Gm[6] + z * Gm[7] - 2.f * y * Gm[8]);
    const float gz = 2.f * (-2.f * z * Gm[0] - w * Gm[1] + x * Gm[2] + w * Gm[3] - 2.f * z * Gm[4] + y * Gm[5] + x * Gm[6] + y * Gm[7]);
    const float dot = w * gw + x * gx + y * gy + z * gz;
    grad_add<DET>(G, G.d_quat + 4 * i + 0, i, 6, (gw - w * dot) / qn);
    grad_add<DET>(G, G.d_quat + 4 * i + 1, i, 7, (gx - x * dot) / qn);
    grad_add<DET>(G, G.d_quat + 4 * i + 2, i, 8, (gy - y * dot) / qn);
    grad_add<DET>(G, G.d_quat + 4 * i + 3, i, 9, (gz - z * dot) / qn);
    d_origin.x += 2.0f * gM * sie[0];
    d_origin.y += 2.0f * gM * sie[1];
    d_origin.z += 2.0f * gM * sie[2];
}

template <bool DET>
__global__ void __launch_bounds__(128) k_backward(BvhDev b, RaySetDev rs, int64_t R, const float *T,
                                                  const float *dL_dT, const int32_t *hit_ids,
                                                  const int32_t *hit_count, int32_t cap, GradOut G,
                                                  int *status) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R;
         r += (int64_t)gridDim.x * blockDim.x) {
        float3 o, d;
        int32_t src = -1;      // sorted position of the excluded Gaussian
        int32_t src_orig = -1; // its original index (implicit sets)
        if (rs.kind == RT_RAYS_EXPLICIT) {
            o = make_float3(rs.ray_o[3 * r], rs.ray_o[3 * r + 1], rs.ray_o[3 * r + 2]);
            d = make_float3(rs.ray_d[3 * r], rs.ray_d[3 * r + 1], rs.ray_d[3 * r + 2]);
            if (rs.ray_src) {
                const int32_t s = rs.ray_src[r];
                src = (s >= 0 && s < b.n) ? b.rank[s] : -1;
            }
        } else {
            const int64_t rid = rs.ray_ids ? rs.ray_ids[r] : r;
            if (rid < 0 || rid >= rs.n_rays) {
                rt_set_error(status, RT_ERR_INVALID_ARG);
                continue;
            }
            const int64_t g = rid / rs.K;
            const int32_t k = (int32_t)(rid - g * rs.K);
            src = b.rank[g];
            src_orig = (int32_t)g;
            implicit_ray(rs, rid, k, g, __ldg(b.gauss + 4 * (int64_t)src), o, d);
        }
        float3 d_origin = make_float3(0.f, 0.f, 0.f);
        const float Tr = T[r];
        const float gT = dL_dT[r];
        const bool live = gT != 0.0f && !(b.t_min > 0.0f && Tr == 0.0f);
        if (live) {
            const int32_t cnt = hit_count ? hit_count[r] : -1;
            if (hit_ids && cnt >= 0 && cnt <= cap) {
                for (int32_t h = 0; h < cnt; ++h) {  // the forward accepted these: no re-check
                    const int32_t i = hit_ids[r * (int64_t)cap + h];
                    const int32_t p = b.rank[i];
                    float alpha;
                    float3 e;
                    peak_accurate(b, p, o, d, alpha, e);
                    hit_grad<DET>(G, i, gT, Tr, alpha, e, d_origin);
                }
            } else if (b.n == 1) {
                float alpha;
                float3 e;
                if (src != 0 && gauss_eval(b, 0, o, d, alpha, e)) {
                    peak_accurate(b, 0, o, d, alpha, e);
                    hit_grad<DET>(G, __float_as_int(__ldg(b.gauss + 1).w), gT, Tr, alpha, e, d_origin);
                }
            } else if (b.n > 1) {
                const float3 inv = safe_inv(d);
                const float3 oi = make_float3(o.x * inv.x, o.y * inv.y, o.z * inv.z);
                uint32_t stack[RT_STACK];
                int sp = 0;
                uint32_t node = 0;
                for (;;) {
                    const float4 n0 = __ldg(b.nodes + 4 * node);
                    const float4 n1 = __ldg(b.nodes + 4 * node + 1);
                    const float4 n2 = __ldg(b.nodes + 4 * node + 2);
                    const float4 n3 = __ldg(b.nodes + 4 * node + 3);
                    bool hl = slab(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, oi, inv);
                    bool hr = slab(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, oi, inv);
                    const uint32_t ch[2] = {__float_as_uint(n3.x), __float_as_uint(n3.y)};
                    bool hit2[2] = {hl, hr};
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        if (hit2[c] && (ch[c] & RT_LEAF_BIT)) {
                            hit2[c] = false;
                            const int32_t p = (int32_t)(ch[c] & ~RT_LEAF_BIT);
                            float alpha;
                            float3 e;
                            if (p != src && gauss_eval(b, p, o, d, alpha, e)) {  // the forward's decision
                                peak_accurate(b, p, o, d, alpha, e);
                                hit_grad<DET>(G, __float_as_int(__ldg(b.gauss + 4 * p + 1).w), gT, Tr, alpha,
                                              e, d_origin);
                            }
                        }
                    }
                    if (hit2[0] && hit2[1]) {
                        if (sp >= RT_STACK) {
                            rt_set_error(status, RT_ERR_STACK_OVERFLOW);
                            break;
                        }
                        stack[sp++] = ch[1];
                        node = ch[0];
                    } else if (hit2[0]) {
                        node = ch[0];
                    } else if (hit2[1]) {
                        node = ch[1];
                    } else {
                        if (sp == 0) break;
                        node = stack[--sp];
                    }
                }
            }
        }
        if (G.d_ray_o) {
            G.d_ray_o[3 * r] = d_origin.x;
            G.d_ray_o[3 * r + 1] = d_origin.y;
            G.d_ray_o[3 * r + 2] = d_origin.z;
        }
        if (src_orig >= 0 && live) {
            grad_add<DET>(G, G.d_mean + 3 * src_orig, src_orig, 0, d_origin.x);
            grad_add<DET>(G, G.d_mean + 3 * src_orig + 1, src_orig, 1, d_origin.y);
            grad_add<DET>(G, G.d_mean + 3 * src_orig + 2, src_orig, 2, d_origin.z);
        }
    }
}

// Deterministic mode: adds the fixed-point sums (times 2^-32) to the caller's
// arrays.
__global__ void k_fx_finalize(const long long *__restrict__ fx, int64_t n, float *d_mean, float *d_scale,
                              float *d_quat, float *d_opacity) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n * kFxPer;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = j / kFxPer;
        const int c = (int)(j - i * kFxPer);
        const float v = (float)((double)fx[j] * (1.0 / 4294967296.0));
        if (c < 3) d_mean[3 * i + c] += v;
        else if (c < 6) d_scale[3 * i + c - 3] += v;
        else if (c < 10) d_quat[4 * i + c - 6] += v;
        else d_opacity[i] += v;
    }
}

}  // namespace

extern "C" rt_status rt_trace_visibility_backward(const rt_bvh *bvh, const rt_rayspec *rays,
                                                  const float *mean, const float *scale,
                                                  const float *quat, const float *opacity,
                                                  const float *T, const float *dL_dT,
                                                  const int32_t *hit_ids, const int32_t *hit_count,
                                                  int32_t hit_cap, float *d_mean, float *d_scale,
                                                  float *d_quat, float *d_opacity, float *d_ray_o,
                                                  rt_stream_t stream) {
    if (!bvh || !rays) return RT_ERR_INVALID_ARG;
    RaySetDev rs;
    int64_t R = 0;
    RT_TRY(rt_rayset_dev(bvh, rays, &rs, &R));
    if (R == 0 || bvh->n == 0) return RT_OK;
    if (!mean || !scale || !quat || !opacity || !T || !dL_dT || !d_mean || !d_scale || !d_quat || !d_opacity)
        return RT_ERR_INVALID_ARG;
    if (hit_ids && (!hit_count || hit_cap <= 0)) return RT_ERR_INVALID_ARG;
    GradOut G;
    G.d_mean = d_mean;
    G.d_scale = d_scale;
    G.d_quat = d_quat;
    G.d_opacity = d_opacity;
    G.d_ray_o = d_ray_o;
    G.mean = mean;
    G.scale = scale;
    G.quat = quat;
    G.opacity = opacity;
    G.fx = nullptr;
    G.status = rt_status_ptr();
    int64_t grid = (R + 127) / 128;
    const int64_t cap_grid = (int64_t)rt_num_sms() * 16;
    if (grid > cap_grid) grid = cap_grid;
    cudaStream_t st = (cudaStream_t)stream;
    if (!bvh->params.deterministic) {
        k_backward<false><<<(int)grid, 128, 0, st>>>(bvh_dev(bvh), rs, R, T, dL_dT, hit_ids, hit_count, hit_cap, G,
                                                     G.status);
        return rt_check_launch();
    }
    const size_t fx_bytes = (size_t)bvh->n * kFxPer * sizeof(long long);
    RT_TRY(rt_alloc((void **)&G.fx, fx_bytes, stream));
    rt_status s = cudaMemsetAsync(G.fx, 0, fx_bytes, st) == cudaSuccess ? RT_OK : RT_ERR_CUDA;
    if (s == RT_OK) {
        k_backward<true><<<(int)grid, 128, 0, st>>>(bvh_dev(bvh), rs, R, T, dL_dT, hit_ids, hit_count, hit_cap, G,
                                                    G.status);
        int64_t fgrid = (bvh->n * kFxPer + 255) / 256;
        if (fgrid > (int64_t)rt_num_sms() * 8) fgrid = (int64_t)rt_num_sms() * 8;
        k_fx_finalize<<<(int)fgrid, 256, 0, st>>>(G.fx, bvh->n, d_mean, d_scale, d_quat, d_opacity);
        s = rt_check_launch();
    } else {
        cudaGetLastError();
    }
    rt_free(G.fx, stream);
    return s;
}
