// rt_internal.cuh -- layouts and device helpers shared by the library's
// translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rt3dg.h"

// ---------------------------------------------------------------------------
// Device-resident layouts (all in Morton-sorted order)
//
// Gaussian record, 64 B = 4 x float4, one per sorted position p:
//   g[4p+0] = (mu.x, mu.y, mu.z, opacity)
//   g[4p+1] = (W00, W01, W02, original index as int bits)
//   g[4p+2] = (W10, W11, W12, 0)
//   g[4p+3] = (W20, W21, W22, 0)
// with W = S^-1 R^T (row k = local axis k divided by s_k), so the
// Mahalanobis distance of x is |W (x - mu)|^2 (Eq. 1).
//
// Internal node record, 64 B = 4 x float4, node i = 0..n-2 (root = 0):
//   nd[4i+0] = (L.lo.x, L.hi.x, L.lo.y, L.hi.y)
//   nd[4i+1] = (L.lo.z, L.hi.z, R.lo.x, R.hi.x)
//   nd[4i+2] = (R.lo.y, R.hi.y, R.lo.z, R.hi.z)
//   nd[4i+3] = (left ref, right ref, 0, 0) as int bits; bit 31 = leaf,
//              low bits = sorted position of the leaf's Gaussian.
// ---------------------------------------------------------------------------

#define RT_LEAF_BIT 0x80000000u
#define RT_EMPTY 0x7fffffffu  // empty child slot of a wide node (its box is NaN)
#define RT_STACK 64  // >= tree depth: keys are 64-bit and unique
#define RT_WIDE_STACK 256  // >= 3 pushes x 64 levels of the 4-wide tree

// 4-wide node record, 128 B = 8 x float4, node j (root = 0):
//   w[8j+0..5] = lo.x[4], hi.x[4], lo.y[4], hi.y[4], lo.z[4], hi.z[4]
//   w[8j+6]    = child refs (int bits): bit 31 = leaf (sorted position),
//                RT_EMPTY = no child, else a wide node index
//   w[8j+7]    = unused
// Empty children and empty leaf boxes are NaN boxes, which no ray hits.

struct rt_bvh {
    int64_t n;
    rt_params params;
    float lo[3], hi[3];      // scene bounds of the means (host copy)
    int64_t bytes;           // device bytes owned
    void *block;             // single device allocation holding everything below
    float4 *gauss;           // [4n]
    float4 *nodes;           // [4(n-1)]
    int32_t *perm;           // [n] sorted position -> original index
    int32_t *rank;           // [n] original index -> sorted position
    uint64_t *keys;          // [n] sorted keys
    int32_t *parent;         // [2n-1]
    float *bounds;           // [6] device copy of lo, hi
    float4 *wide;            // [8 * (n-1)] 4-wide nodes (collapsed binary tree)
    int64_t n_wide;          // number of 4-wide nodes (host copy)
    // refit links, made by the first rt_bvh_refit: 4*w + slot of each leaf
    // (sorted position) and of each wide node in its wide parent (root: -1),
    // and per-wide-node arrival counters
    void *links;
    int32_t *leaf_slot;      // [n]
    int32_t *wide_parent;    // [n_wide]
    uint32_t *wide_arrivals; // [n_wide]
};

struct rt_envmap {
    int32_t h, w;
    void *block;
    double *cdf;      // [h*w] normalised cumulative weights
    float *corners;   // [(h+1)*(w+1)*3]
};

// The sticky status word lives in rt_api.cu; kernels receive its address
// (rt_status_ptr) as an argument and record the first error with a CAS.
__device__ __forceinline__ void rt_set_error(int *status, int code) {
    if (status) atomicCAS(status, 0, code);
}
int *rt_status_ptr();

// host helpers (rt_api.cu)
rt_status rt_check_launch();
rt_status rt_alloc(void **p, size_t bytes, rt_stream_t s);
void rt_free(void *p, rt_stream_t s);
// Stable LSD radix sort (8-bit digits) of n <= 2^31 (key, value) pairs in
// place by the low `bits` bits of the keys; scratch from rt_alloc, released
// in stream order (rt_build.cu).
rt_status rt_sort_pairs_u32(uint32_t *keys, int32_t *vals, int64_t n, int bits, rt_stream_t stream);
int rt_num_sms();

#define RT_TRY(x)                              \
    do {                                       \
        rt_status _st = (x);                   \
        if (_st != RT_OK) return _st;          \
    } while (0)

// ---------------------------------------------------------------------------
// Device math helpers
// ---------------------------------------------------------------------------

// Exact difference a - b = hi + lo (Knuth's TwoSum with b negated).
__device__ __forceinline__ void two_diff(float a, float b, float &hi, float &lo) {
    float s = __fsub_rn(a, b);
    float bb = __fsub_rn(s, a);
    lo = __fsub_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fadd_rn(b, bb));
    hi = s;
}

__device__ __forceinline__ float dot3(float3 a, float3 b) {
    return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z));
}

// Philox4x64-10 (Salmon et al., SC'11).
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint64_t lo0 = 0xD2E7470EE14C6C93ull * c[0];
        uint64_t hi0 = __umul64hi(0xD2E7470EE14C6C93ull, c[0]);
        uint64_t lo1 = 0xCA5A826395121157ull * c[2];
        uint64_t hi1 = __umul64hi(0xCA5A826395121157ull, c[2]);
        uint64_t n0 = hi1 ^ c[1] ^ k0;
        uint64_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B97F4A7C15ull;
        k1 += 0xBB67AE8584CAA73Bull;
    }
}

// ---------------------------------------------------------------------------
// Ray sets on the device
// ---------------------------------------------------------------------------
struct RaySetDev {
    int32_t kind;
    int32_t K;            // directions / samples per Gaussian
    int64_t n_rays;
    const float *ray_o, *ray_d;
    const int32_t *ray_src;
    const float *dirs;
    const double *env_cdf;
    const float *env_corners;
    int32_t env_h, env_w;
    uint64_t seed;
    const int64_t *ray_ids;
    float eps;
    const float *normals;  // HEMI: [n*3], original order
};

// Direction of env sample with ray id r (see rt3dg.h): pixel by binary
// search of the float64 CDF (first entry > u0), then the normalised bilinear
// blend of the pixel's corners with separately rounded float32 operations.
__device__ __forceinline__ float3 env_direction(const RaySetDev &rs, int64_t r) {
    uint64_t c[4] = {(uint64_t)r, 0ull, 0ull, 0ull};
    philox4x64_10(c, rs.seed, 0ull);
    double u0 = (double)(c[0] >> 11) * (1.0 / 9007199254740992.0);
    int np = rs.env_h * rs.env_w;
    int lo = 0, hi = np - 1;  // invariant: answer in [lo, hi]
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (rs.env_cdf[mid] > u0) hi = mid;
        else lo = mid + 1;
    }
    int pi = lo / rs.env_w, pj = lo % rs.env_w;
    float a = __fmul_rn((float)(c[1] >> 40), 1.0f / 16777216.0f);
    float b = __fmul_rn((float)(c[2] >> 40), 1.0f / 16777216.0f);
    int W1 = rs.env_w + 1;
    const float *c00 = rs.env_corners + 3 * (pi * W1 + pj);
    const float *c01 = c00 + 3;
    const float *c10 = rs.env_corners + 3 * ((pi + 1) * W1 + pj);
    const float *c11 = c10 + 3;
    float v[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float top = __fadd_rn(c00[k], __fmul_rn(a, __fsub_rn(c01[k], c00[k])));
        float bot = __fadd_rn(c10[k], __fmul_rn(a, __fsub_rn(c11[k], c10[k])));
        v[k] = __fadd_rn(top, __fmul_rn(b, __fsub_rn(bot, top)));
    }
    float ss = __fadd_rn(__fadd_rn(__fmul_rn(v[0], v[0]), __fmul_rn(v[1], v[1])), __fmul_rn(v[2], v[2]));
    float len = __fsqrt_rn(ss);
    return make_float3(__fdiv_rn(v[0], len), __fdiv_rn(v[1], len), __fdiv_rn(v[2], len));
}

// Frame (t1, t2, n) of a Gaussian's hemisphere set (Sec. 3.3): the normal
// normalised in float32, then the branchless orthonormal basis of Duff et
// al. 2017; every operation separately rounded (the oracle repeats them).
struct HemiFrame {
    float3 t1, t2, n;
};

__device__ __forceinline__ HemiFrame hemi_frame(const float *nrm) {
    const float x = __ldg(nrm), y = __ldg(nrm + 1), z = __ldg(nrm + 2);
    const float s = __fadd_rn(__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)), __fmul_rn(z, z));
    const float l = __fsqrt_rn(s);
    HemiFrame f;
    f.n = make_float3(__fdiv_rn(x, l), __fdiv_rn(y, l), __fdiv_rn(z, l));
    const float sg = copysignf(1.0f, f.n.z);
    const float a = __fdiv_rn(-1.0f, __fadd_rn(sg, f.n.z));
    const float b = __fmul_rn(__fmul_rn(f.n.x, f.n.y), a);
    f.t1 = make_float3(__fadd_rn(1.0f, __fmul_rn(__fmul_rn(__fmul_rn(sg, f.n.x), f.n.x), a)), __fmul_rn(sg, b),
                       -__fmul_rn(sg, f.n.x));
    f.t2 = make_float3(b, __fadd_rn(sg, __fmul_rn(__fmul_rn(f.n.y, f.n.y), a)), -f.n.y);
    return f;
}

// Local direction h (z along the normal) in the frame: (h.x t1 + h.y t2) + h.z n.
__device__ __forceinline__ float3 hemi_rotate(const HemiFrame &f, const float *h) {
    const float hx = __ldg(h), hy = __ldg(h + 1), hz = __ldg(h + 2);
    return make_float3(__fadd_rn(__fadd_rn(__fmul_rn(hx, f.t1.x), __fmul_rn(hy, f.t2.x)), __fmul_rn(hz, f.n.x)),
                       __fadd_rn(__fadd_rn(__fmul_rn(hx, f.t1.y), __fmul_rn(hy, f.t2.y)), __fmul_rn(hz, f.n.y)),
                       __fadd_rn(__fadd_rn(__fmul_rn(hx, f.t1.z), __fmul_rn(hy, f.t2.z)), __fmul_rn(hz, f.n.z)));
}

// Ray r = g*K + k of an implicit set (DIRS / ENV / HEMI) cast from Gaussian g
// (original index) whose mean is mu: direction and origin fl(mu + fl(eps d)).
__device__ __forceinline__ void implicit_ray(const RaySetDev &rs, int64_t r, int32_t k, int64_t g, float4 mu,
                                             float3 &o, float3 &d) {
    if (rs.kind == RT_RAYS_DIRS) {
        d = make_float3(rs.dirs[3 * k], rs.dirs[3 * k + 1], rs.dirs[3 * k + 2]);
    } else if (rs.kind == RT_RAYS_HEMI) {
        d = hemi_rotate(hemi_frame(rs.normals + 3 * g), rs.dirs + 3 * k);
    } else {
        d = env_direction(rs, r);
    }
    o.x = __fadd_rn(mu.x, __fmul_rn(rs.eps, d.x));
    o.y = __fadd_rn(mu.y, __fmul_rn(rs.eps, d.y));
    o.z = __fadd_rn(mu.z, __fmul_rn(rs.eps, d.z));
}

// Host: convert a public ray set into the device view (validates it).
rt_status rt_rayset_dev(const rt_bvh *bvh, const rt_rayspec *rays, RaySetDev *out, int64_t *count);
// The same for a set over n Gaussians (a composed scene's rows) with origin
// offset origin_eps.
rt_status rt_rayset_dev_n(int64_t n, float origin_eps, const rt_rayspec *rays, RaySetDev *out, int64_t *count);

// Host: enqueue one trace of a ray set (rt_trace.cu).  `work` is an optional
// caller-provided device counter (8 bytes); NULL allocates one per call.
rt_status rt_trace_launch(const rt_bvh *bvh, const rt_rayspec *rays, float *T_out,
                          const rt_trace_opts *opts, rt_stream_t stream, unsigned long long *work);

// Host: trace the rays listed in ray_ids[0 .. *count) of an implicit set
// (count is a device value, at most max_count) writing T_out[out_index[i]].
// `work` is a device counter (8 bytes) owned by the caller.
rt_status rt_trace_launch_list(const rt_bvh *bvh, const rt_rayspec *rays, const int64_t *ray_ids,
                               const int64_t *out_index, const unsigned long long *count, int64_t max_count,
                               float *T_out, rt_stream_t stream, unsigned long long *work);
