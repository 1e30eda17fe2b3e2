// rt_trace_core.cuh -- ray/Gaussian and ray/box tests and the two traversal
// strategies, shared by the forward trace, the adjoint and the batched launch.
#pragma once

#include "rt_internal.cuh"

struct BvhDev {
    const float4 *gauss;
    const float4 *nodes;
    const float4 *wide;  // null if the 4-wide tree is unavailable
    const int32_t *rank;
    int64_t n;
    float k2;         // k_sigma^2
    float alpha_min;
    float t_min;
};

inline BvhDev bvh_dev(const rt_bvh *b) {
    BvhDev d;
    d.gauss = b->gauss;
    d.nodes = b->nodes;
    d.wide = b->n_wide > 0 ? b->wide : nullptr;
    d.rank = b->rank;
    d.n = b->n;
    d.k2 = b->params.k_sigma * b->params.k_sigma;
    d.alpha_min = b->params.alpha_min;
    d.t_min = b->params.t_min;
    return d;
}

struct TraceAux {
    unsigned long long *counters;  // [4] or null
    int32_t *hit_ids;              // [R*cap] or null
    int32_t *hit_count;            // [R] or null
    int32_t cap;
    int *status;
};

struct LaneLog {
    int32_t *ids;  // this ray's slots (null = no log)
    int32_t cap;
    int32_t count;
};

// Reciprocal direction with exact zeros replaced by a tiny signed value, so
// (lo - o) * inv never forms 0 * inf.
__device__ __forceinline__ float3 safe_inv(float3 d) {
    const float tiny = 1e-30f;
    float x = fabsf(d.x) < tiny ? copysignf(tiny, d.x) : d.x;
    float y = fabsf(d.y) < tiny ? copysignf(tiny, d.y) : d.y;
    float z = fabsf(d.z) < tiny ? copysignf(tiny, d.z) : d.z;
    return make_float3(1.0f / x, 1.0f / y, 1.0f / z);
}

// Ray vs axis-aligned box over t in [0, inf), t = lo * inv - o * inv (one
// FMA per plane, oi = o * inv precomputed).  The rounding of oi is absorbed
// by the boxes' absolute margin (1e-6 of the scene extent) and the far
// distance gets a 1e-6 relative allowance, so rounding never rejects a box
// that an accepted peak lies in.
__device__ __forceinline__ bool slab(float lox, float hix, float loy, float hiy, float loz, float hiz,
                                     float3 oi, float3 inv) {
    float tx0 = fmaf(lox, inv.x, -oi.x), tx1 = fmaf(hix, inv.x, -oi.x);
    float ty0 = fmaf(loy, inv.y, -oi.y), ty1 = fmaf(hiy, inv.y, -oi.y);
    float tz0 = fmaf(loz, inv.z, -oi.z), tz1 = fmaf(hiz, inv.z, -oi.z);
    float tnear = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.0f));
    float tfar = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fmaxf(tz0, tz1));
    return tnear <= fmaf(fabsf(tfar), 1e-6f, tfar);
}

// slab for two children at once (children a, b of a 4-wide node, lo/hi as
// (a, b) pairs), packed FMAs as in slab_sorted2; same results as two slab
// calls.
__device__ __forceinline__ void slab2(float2 lx, float2 hx, float2 ly, float2 hy, float2 lz, float2 hz, float2 ix,
                                      float2 iy, float2 iz, float2 ox, float2 oy, float2 oz, bool &ha, bool &hb) {
    const float2 tx0 = __ffma2_rn(lx, ix, ox), tx1 = __ffma2_rn(hx, ix, ox);
    const float2 ty0 = __ffma2_rn(ly, iy, oy), ty1 = __ffma2_rn(hy, iy, oy);
    const float2 tz0 = __ffma2_rn(lz, iz, oz), tz1 = __ffma2_rn(hz, iz, oz);
    const float na = fmaxf(fmaxf(fminf(tx0.x, tx1.x), fminf(ty0.x, ty1.x)), fmaxf(fminf(tz0.x, tz1.x), 0.0f));
    const float fa = fminf(fminf(fmaxf(tx0.x, tx1.x), fmaxf(ty0.x, ty1.x)), fmaxf(tz0.x, tz1.x));
    const float nb = fmaxf(fmaxf(fminf(tx0.y, tx1.y), fminf(ty0.y, ty1.y)), fmaxf(fminf(tz0.y, tz1.y), 0.0f));
    const float fb = fminf(fminf(fmaxf(tx0.y, tx1.y), fmaxf(ty0.y, ty1.y)), fmaxf(tz0.y, tz1.y));
    ha = na <= fmaf(fabsf(fa), 1e-6f, fa);
    hb = nb <= fmaf(fabsf(fb), 1e-6f, fb);
}

// The four children of a 4-wide node (rows lo.x, hi.x, lo.y, hi.y, lo.z,
// hi.z as float4) against a ray: two slab2 calls.
__device__ __forceinline__ void slab4(float4 lx, float4 hx, float4 ly, float4 hy, float4 lz, float4 hz, float3 oi,
                                      float3 inv, bool (&h)[4]) {
    const float2 ix = make_float2(inv.x, inv.x), iy = make_float2(inv.y, inv.y), iz = make_float2(inv.z, inv.z);
    const float2 ox = make_float2(-oi.x, -oi.x), oy = make_float2(-oi.y, -oi.y), oz = make_float2(-oi.z, -oi.z);
    slab2(make_float2(lx.x, lx.y), make_float2(hx.x, hx.y), make_float2(ly.x, ly.y), make_float2(hy.x, hy.y),
          make_float2(lz.x, lz.y), make_float2(hz.x, hz.y), ix, iy, iz, ox, oy, oz, h[0], h[1]);
    slab2(make_float2(lx.z, lx.w), make_float2(hx.z, hx.w), make_float2(ly.z, ly.w), make_float2(hy.z, hy.w),
          make_float2(lz.z, lz.w), make_float2(hz.z, hz.w), ix, iy, iz, ox, oy, oz, h[2], h[3]);
}

// The four children of a 4-wide node against a ray: each box's entry
// distance along the ray (the near distance of slab2's test), +inf where
// the ray misses the box.
__device__ __forceinline__ void slab4_near(float4 lx, float4 hx, float4 ly, float4 hy, float4 lz, float4 hz,
                                           float3 oi, float3 inv, float (&tn)[4]) {
    const float2 ix = make_float2(inv.x, inv.x), iy = make_float2(inv.y, inv.y), iz = make_float2(inv.z, inv.z);
    const float2 ox = make_float2(-oi.x, -oi.x), oy = make_float2(-oi.y, -oi.y), oz = make_float2(-oi.z, -oi.z);
    const float inf = __int_as_float(0x7f800000);
#pragma unroll
    for (int pr = 0; pr < 2; ++pr) {
        const float2 l_x = pr ? make_float2(lx.z, lx.w) : make_float2(lx.x, lx.y);
        const float2 h_x = pr ? make_float2(hx.z, hx.w) : make_float2(hx.x, hx.y);
        const float2 l_y = pr ? make_float2(ly.z, ly.w) : make_float2(ly.x, ly.y);
        const float2 h_y = pr ? make_float2(hy.z, hy.w) : make_float2(hy.x, hy.y);
        const float2 l_z = pr ? make_float2(lz.z, lz.w) : make_float2(lz.x, lz.y);
        const float2 h_z = pr ? make_float2(hz.z, hz.w) : make_float2(hz.x, hz.y);
        const float2 tx0 = __ffma2_rn(l_x, ix, ox), tx1 = __ffma2_rn(h_x, ix, ox);
        const float2 ty0 = __ffma2_rn(l_y, iy, oy), ty1 = __ffma2_rn(h_y, iy, oy);
        const float2 tz0 = __ffma2_rn(l_z, iz, oz), tz1 = __ffma2_rn(h_z, iz, oz);
        const float na = fmaxf(fmaxf(fminf(tx0.x, tx1.x), fminf(ty0.x, ty1.x)), fmaxf(fminf(tz0.x, tz1.x), 0.0f));
        const float fa = fminf(fminf(fmaxf(tx0.x, tx1.x), fmaxf(ty0.x, ty1.x)), fmaxf(tz0.x, tz1.x));
        const float nb = fmaxf(fmaxf(fminf(tx0.y, tx1.y), fminf(ty0.y, ty1.y)), fmaxf(fminf(tz0.y, tz1.y), 0.0f));
        const float fb = fminf(fminf(fmaxf(tx0.y, tx1.y), fmaxf(ty0.y, ty1.y)), fmaxf(tz0.y, tz1.y));
        tn[2 * pr] = na <= fmaf(fabsf(fa), 1e-6f, fa) ? na : inf;
        tn[2 * pr + 1] = nb <= fmaf(fabsf(fb), 1e-6f, fb) ? nb : inf;
    }
}

__device__ __forceinline__ void cswap_near(float &ta, uint32_t &qa, float &tb, uint32_t &qb) {
    const bool sw = tb < ta;
    const float t = sw ? tb : ta;
    const uint32_t q = sw ? qb : qa;
    tb = sw ? ta : tb;
    qb = sw ? qa : qb;
    ta = t;
    qa = q;
}

// The per-ray walk's next node among a visited node's internal children hit
// (entry distances t, +inf for the others): the nearest (far: the farthest)
// becomes `next` (-1: none) and the rest are pushed so that the stack pops
// them in the same order.  The order decides only how soon the walk stops
// once T < T_min: the accepted set and the factors are the same.
// Returns false (nothing pushed) if the stack would overflow.
__device__ __forceinline__ bool visit_order(float t0, float t1, float t2, float t3, uint32_t r0, uint32_t r1,
                                            uint32_t r2, uint32_t r3, bool far, uint32_t *stack, int &sp,
                                            int &next) {
    const float inf = __int_as_float(0x7f800000);
    if (far) {
        t0 = t0 < inf ? -t0 : inf;
        t1 = t1 < inf ? -t1 : inf;
        t2 = t2 < inf ? -t2 : inf;
        t3 = t3 < inf ? -t3 : inf;
    }
    cswap_near(t0, r0, t1, r1);
    cswap_near(t2, r2, t3, r3);
    cswap_near(t0, r0, t2, r2);
    cswap_near(t1, r1, t3, r3);
    cswap_near(t1, r1, t2, r2);
    next = t0 < inf ? (int)r0 : -1;
    const int n = (t1 < inf) + (t2 < inf) + (t3 < inf);
    if (sp + n > RT_WIDE_STACK) return false;
    if (t3 < inf) stack[sp++] = r3;
    if (t2 < inf) stack[sp++] = r2;
    if (t1 < inf) stack[sp++] = r1;
    return true;
}

// The per-ray walks' order for a ray set.  A direction set covers the whole
// sphere about each Gaussian: about half its rays go into the body the
// Gaussian lies on, and their occluders are that body's far side, while the
// near boxes hold the Gaussian's own neighbours, which such a ray enters and
// leaves mostly without a hit; so direction rays visit the farthest child
// first.  Hemisphere and env-map rays leave the surface: the occluders that
// put them in shadow come first along the ray, so they visit the nearest
// child first.
__device__ __forceinline__ bool far_first(const RaySetDev &rs) { return rs.kind == RT_RAYS_DIRS; }

// The slab test of two children at once with the planes already ordered
// along the ray (near plane first on every axis: slab() without the per-axis
// min/max): the plane distances of both along an axis come from one packed
// FMA (fma.rn.f32x2 rounds each half as fmaf), so each packed instruction
// does the work of two issued ones.  i* = (inv, inv), o* = (-oi, -oi).
__device__ __forceinline__ void slab_sorted2(float2 nx, float2 fx, float2 ny, float2 fy, float2 nz, float2 fz,
                                             float2 ix, float2 iy, float2 iz, float2 ox, float2 oy, float2 oz,
                                             bool &ha, bool &hb) {
    const float2 tnx = __ffma2_rn(nx, ix, ox), tfx = __ffma2_rn(fx, ix, ox);
    const float2 tny = __ffma2_rn(ny, iy, oy), tfy = __ffma2_rn(fy, iy, oy);
    const float2 tnz = __ffma2_rn(nz, iz, oz), tfz = __ffma2_rn(fz, iz, oz);
    const float na = fmaxf(fmaxf(tnx.x, tny.x), fmaxf(tnz.x, 0.0f));
    const float fa = fminf(fminf(tfx.x, tfy.x), tfz.x);
    const float nb = fmaxf(fmaxf(tnx.y, tny.y), fmaxf(tnz.y, 0.0f));
    const float fb = fminf(fminf(tfx.y, tfy.y), tfz.y);
    ha = na <= fmaf(fabsf(fa), 1e-6f, fa);
    hb = nb <= fmaf(fabsf(fb), 1e-6f, fb);
}

// Peak response of the Gaussian at sorted position p along the ray
// (Eq. 13-14 with Sigma^-1).  In the whitened frame u = W (x - mu) the squared
// Mahalanobis distance along the ray is |u_o + t u_d|^2, minimised at
// t* = -(u_o . u_d)/(u_d . u_d).
// Accuracy: o - mu is split exactly into hi + lo; the point e = x(t*) - mu is
// rebuilt in world space as fma(t*, d, hi) + lo (it is small, so this has no
// cancellation), and m^2 = |W e|^2.  m^2 is stationary at t*, so t* needs only
// a fast reciprocal (its relative error ~1e-7 enters m^2 squared; its sign is
// exact); alpha = o exp(-m^2/2) uses the fast exponential (relative error
// ~4e-7).  Returns true if the Gaussian is accepted (t* > 0, m^2 <= K^2,
// alpha >= alpha_min), with alpha and e.  The forward and the adjoint both use
// this routine, so they make the same decisions.
// two_diff of two components at once; fma(b, -1, a) rounds a - b once, as
// a subtraction does, so the halves equal two two_diff calls.
__device__ __forceinline__ void two_diff2(float2 a, float2 b, float2 &hi, float2 &lo) {
    const float2 m1 = make_float2(-1.0f, -1.0f);
    const float2 s = __ffma2_rn(b, m1, a);   // a - b
    const float2 bb = __ffma2_rn(a, m1, s);  // s - a
    const float2 t = __ffma2_rn(bb, m1, s);  // s - bb
    const float2 u = __ffma2_rn(t, m1, a);   // a - (s - bb)
    const float2 v = __fadd2_rn(b, bb);      // b + bb
    lo = __ffma2_rn(v, m1, u);               // u - v
    hi = s;
}

__device__ __forceinline__ bool gauss_eval(const BvhDev &b, int32_t p, float3 o, float3 d, float &alpha,
                                           float3 &e) {
    const float4 g0 = __ldg(b.gauss + 4 * p);
    const float4 g1 = __ldg(b.gauss + 4 * p + 1);
    const float4 g2 = __ldg(b.gauss + 4 * p + 2);
    const float4 g3 = __ldg(b.gauss + 4 * p + 3);
    float2 hxy, lxy;
    two_diff2(make_float2(o.x, o.y), make_float2(g0.x, g0.y), hxy, lxy);
    const float hx = hxy.x, hy = hxy.y;
    float hz, lz;
    two_diff(o.z, g0.z, hz, lz);
    const float3 w0 = make_float3(g1.x, g1.y, g1.z);
    const float3 w1 = make_float3(g2.x, g2.y, g2.z);
    const float3 w2 = make_float3(g3.x, g3.y, g3.z);
    const float3 dh = make_float3(hx, hy, hz);
    const float3 ud = make_float3(dot3(w0, d), dot3(w1, d), dot3(w2, d));
    const float3 uo = make_float3(dot3(w0, dh), dot3(w1, dh), dot3(w2, dh));
    const float t = __fdividef(-dot3(uo, ud), dot3(ud, ud));
    if (!(t > 0.0f)) return false;
    const float2 exy = __fadd2_rn(__ffma2_rn(make_float2(t, t), make_float2(d.x, d.y), hxy), lxy);
    e = make_float3(exy.x, exy.y, fmaf(t, d.z, hz) + lz);
    const float3 u = make_float3(dot3(w0, e), dot3(w1, e), dot3(w2, e));
    const float m2 = dot3(u, u);
    if (!(m2 <= b.k2)) return false;
    alpha = g0.w * __expf(-0.5f * m2);
    return alpha >= b.alpha_min;
}

// gauss_eval and, when accepted, the transmittance update of Eq. 15.
__device__ __forceinline__ bool gauss_hit(const BvhDev &b, int32_t p, float3 o, float3 d, float &T) {
    float alpha;
    float3 e;
    if (!gauss_eval(b, p, o, d, alpha, e)) return false;
    T *= (1.0f - alpha);
    return true;
}

__device__ __forceinline__ void log_hit(LaneLog &lg, const BvhDev &b, int32_t p) {
    if (lg.ids) {
        if (lg.count < lg.cap) lg.ids[lg.count] = __float_as_int(__ldg(b.gauss + 4 * p + 1).w);
        lg.count++;
    }
}

struct WorkCounts {
    unsigned long long box, gauss, hits;
};

// Strategy 1: each thread traverses alone with a private stack.
template <bool COUNT>
__device__ __forceinline__ float trace_ray(const BvhDev &b, float3 o, float3 d, int32_t src,
                                           LaneLog &lg, WorkCounts &wc, int *status) {
    float T = 1.0f;
    if (b.n <= 0) return T;
    if (b.n == 1) {
        if (COUNT) wc.gauss++;
        if (src != 0 && gauss_hit(b, 0, o, d, T)) {
            if (COUNT) wc.hits++;
            log_hit(lg, b, 0);
        }
        return T < b.t_min ? 0.0f : T;
    }
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
        if (COUNT) wc.box += 2;
        const uint32_t cl = __float_as_uint(n3.x), cr = __float_as_uint(n3.y);
        if (hl && (cl & RT_LEAF_BIT)) {
            int32_t p = (int32_t)(cl & ~RT_LEAF_BIT);
            hl = false;
            if (p != src) {
                if (COUNT) wc.gauss++;
                if (gauss_hit(b, p, o, d, T)) {
                    if (COUNT) wc.hits++;
                    log_hit(lg, b, p);
                }
            }
        }
        if (hr && (cr & RT_LEAF_BIT)) {
            int32_t p = (int32_t)(cr & ~RT_LEAF_BIT);
            hr = false;
            if (p != src) {
                if (COUNT) wc.gauss++;
                if (gauss_hit(b, p, o, d, T)) {
                    if (COUNT) wc.hits++;
                    log_hit(lg, b, p);
                }
            }
        }
        if (T < b.t_min) break;
        if (hl && hr) {
            if (sp >= RT_STACK) {
                rt_set_error(status, RT_ERR_STACK_OVERFLOW);
                break;
            }
            stack[sp++] = cr;
            node = cl;
        } else if (hl) {
            node = cl;
        } else if (hr) {
            node = cr;
        } else {
            if (sp == 0) break;
            node = stack[--sp];
        }
    }
    return T < b.t_min ? 0.0f : T;
}

// Strategy 2: the warp's 32 rays traverse together.  A node is visited if
// any lane's ray hit its box; each lane tests the children only if its own
// ray hit the node (the lane mask travels with the node on the stack), so the
// per-ray work counts equal strategy 1's.  The stack is warp-uniform and
// lives in registers: entry e sits in lane e % 32, column e / 32.
template <bool COUNT>
__device__ __forceinline__ float trace_packet(const BvhDev &b, float3 o, float3 d, int32_t src,
                                              bool valid, LaneLog &lg, WorkCounts &wc,
                                              int *status) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    float T = 1.0f;
    if (b.n <= 0) return T;
    if (b.n == 1) {
        if (valid) {
            if (COUNT) wc.gauss++;
            if (src != 0 && gauss_hit(b, 0, o, d, T)) {
                if (COUNT) wc.hits++;
                log_hit(lg, b, 0);
            }
        }
        return T < b.t_min ? 0.0f : T;
    }
    const float3 inv = safe_inv(d);
    const float3 oi = make_float3(o.x * inv.x, o.y * inv.y, o.z * inv.z);
    uint32_t alive = __ballot_sync(FULL, valid);
    uint32_t s_node0 = 0, s_node1 = 0, s_mask0 = 0, s_mask1 = 0;
    int sp = 0;
    uint32_t node = 0, mask = alive;
    while (mask) {
        const bool mine = (mask >> lane) & 1u;
        const float4 n0 = __ldg(b.nodes + 4 * node);
        const float4 n1 = __ldg(b.nodes + 4 * node + 1);
        const float4 n2 = __ldg(b.nodes + 4 * node + 2);
        const float4 n3 = __ldg(b.nodes + 4 * node + 3);
        bool hl = false, hr = false;
        if (mine) {
            hl = slab(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, oi, inv);
            hr = slab(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, oi, inv);
            if (COUNT) wc.box += 2;
        }
        const uint32_t cl = __float_as_uint(n3.x), cr = __float_as_uint(n3.y);
        if (cl & RT_LEAF_BIT) {
            int32_t p = (int32_t)(cl & ~RT_LEAF_BIT);
            if (hl && p != src) {
                if (COUNT) wc.gauss++;
                if (gauss_hit(b, p, o, d, T)) {
                    if (COUNT) wc.hits++;
                    log_hit(lg, b, p);
                }
            }
            hl = false;
        }
        if (cr & RT_LEAF_BIT) {
            int32_t p = (int32_t)(cr & ~RT_LEAF_BIT);
            if (hr && p != src) {
                if (COUNT) wc.gauss++;
                if (gauss_hit(b, p, o, d, T)) {
                    if (COUNT) wc.hits++;
                    log_hit(lg, b, p);
                }
            }
            hr = false;
        }
        alive = __ballot_sync(FULL, valid && !(T < b.t_min));
        const uint32_t ml = __ballot_sync(FULL, hl) & alive;
        const uint32_t mr = __ballot_sync(FULL, hr) & alive;
        if (ml && mr) {
            if (sp >= 2 * 32) {
                rt_set_error(status, RT_ERR_STACK_OVERFLOW);
                break;
            }
            if (lane == (sp & 31)) {
                if (sp < 32) {
                    s_node0 = cr;
                    s_mask0 = mr;
                } else {
                    s_node1 = cr;
                    s_mask1 = mr;
                }
            }
            ++sp;
            node = cl;
            mask = ml;
        } else if (ml) {
            node = cl;
            mask = ml;
        } else if (mr) {
            node = cr;
            mask = mr;
        } else {
            mask = 0;
            while (sp > 0) {
                --sp;
                const int srcl = sp & 31;
                const bool lo = sp < 32;
                node = __shfl_sync(FULL, lo ? s_node0 : s_node1, srcl);
                mask = __shfl_sync(FULL, lo ? s_mask0 : s_mask1, srcl) & alive;
                if (mask) break;
            }
        }
    }
    return T < b.t_min ? 0.0f : T;
}

// Strategy 3: warp packet over the 4-wide tree.  As strategy 2, but a visit
// tests four child boxes per lane (one float4 of each coordinate), evaluates
// the leaf children each lane hit, and pushes all but one of the internal
// children some lane still needs onto a warp stack in shared memory.
// UNIFORM: every lane has the same direction (a direction set): each box is
// then tested against its near and far planes, chosen once per packet from
// the direction's signs, without per-box min/max.
template <bool COUNT, bool UNIFORM>
__device__ __forceinline__ float trace_wide(const BvhDev &b, float3 o, float3 d, int32_t src, bool valid,
                                            LaneLog &lg, WorkCounts &wc, int *status, int2 *stk) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    float T = 1.0f;
    if (b.n <= 0) return T;
    if (b.n == 1) {
        if (valid) {
            if (COUNT) wc.gauss++;
            if (src != 0 && gauss_hit(b, 0, o, d, T)) {
                if (COUNT) wc.hits++;
                log_hit(lg, b, 0);
            }
        }
        return T < b.t_min ? 0.0f : T;
    }
    const float3 inv = safe_inv(d);
    const float3 oi = make_float3(o.x * inv.x, o.y * inv.y, o.z * inv.z);
    const int sx = inv.x < 0.0f, sy = inv.y < 0.0f, sz = inv.z < 0.0f;
    const float2 ix2 = make_float2(inv.x, inv.x), iy2 = make_float2(inv.y, inv.y), iz2 = make_float2(inv.z, inv.z);
    const float2 ox2 = make_float2(-oi.x, -oi.x), oy2 = make_float2(-oi.y, -oi.y), oz2 = make_float2(-oi.z, -oi.z);
    uint32_t alive = __ballot_sync(FULL, valid);
    int sp = 0;
    uint32_t node = 0, mask = alive;
    while (mask) {
        const bool mine = (mask >> lane) & 1u;
        const float4 *w = b.wide + 8 * (int64_t)node;
        const float4 rf = __ldg(w + 6);
        const uint32_t r0 = __float_as_uint(rf.x), r1 = __float_as_uint(rf.y), r2 = __float_as_uint(rf.z),
                       r3 = __float_as_uint(rf.w);
        bool h0 = false, h1 = false, h2 = false, h3 = false;
        if (UNIFORM) {
            // near/far planes by the shared direction's signs (sx = 1 if d.x < 0)
            const float4 nx = __ldg(w + sx), fx = __ldg(w + 1 - sx), ny = __ldg(w + 2 + sy),
                         fy = __ldg(w + 3 - sy), nz = __ldg(w + 4 + sz), fz = __ldg(w + 5 - sz);
            if (mine) {
                slab_sorted2(make_float2(nx.x, nx.y), make_float2(fx.x, fx.y), make_float2(ny.x, ny.y),
                             make_float2(fy.x, fy.y), make_float2(nz.x, nz.y), make_float2(fz.x, fz.y), ix2, iy2, iz2,
                             ox2, oy2, oz2, h0, h1);
                slab_sorted2(make_float2(nx.z, nx.w), make_float2(fx.z, fx.w), make_float2(ny.z, ny.w),
                             make_float2(fy.z, fy.w), make_float2(nz.z, nz.w), make_float2(fz.z, fz.w), ix2, iy2, iz2,
                             ox2, oy2, oz2, h2, h3);
            }
        } else {
            const float4 lx = __ldg(w), hx = __ldg(w + 1), ly = __ldg(w + 2), hy = __ldg(w + 3),
                         lz = __ldg(w + 4), hz = __ldg(w + 5);
            if (mine) {
                bool h[4];
                slab4(lx, hx, ly, hy, lz, hz, oi, inv, h);
                h0 = h[0];
                h1 = h[1];
                h2 = h[2];
                h3 = h[3];
            }
        }
        if (COUNT && mine) wc.box += (r0 != RT_EMPTY) + (r1 != RT_EMPTY) + (r2 != RT_EMPTY) + (r3 != RT_EMPTY);
        // leaf children this lane hit, one Gaussian test each
        uint32_t leaves = ((h0 && (r0 & RT_LEAF_BIT)) ? 1u : 0u) | ((h1 && (r1 & RT_LEAF_BIT)) ? 2u : 0u) |
                          ((h2 && (r2 & RT_LEAF_BIT)) ? 4u : 0u) | ((h3 && (r3 & RT_LEAF_BIT)) ? 8u : 0u);
        while (leaves) {
            const int c = __ffs(leaves) - 1;
            leaves &= leaves - 1u;
            const uint32_t r = c == 0 ? r0 : c == 1 ? r1 : c == 2 ? r2 : r3;
            const int32_t p = (int32_t)(r & ~RT_LEAF_BIT);
            if (p != src) {
                if (COUNT) wc.gauss++;
                if (gauss_hit(b, p, o, d, T)) {
                    if (COUNT) wc.hits++;
                    log_hit(lg, b, p);
                }
            }
        }
        alive = __ballot_sync(FULL, valid && !(T < b.t_min));
        const uint32_t m0 = (r0 & RT_LEAF_BIT) ? 0u : __ballot_sync(FULL, h0) & alive;
        const uint32_t m1 = (r1 & RT_LEAF_BIT) ? 0u : __ballot_sync(FULL, h1) & alive;
        const uint32_t m2 = (r2 & RT_LEAF_BIT) ? 0u : __ballot_sync(FULL, h2) & alive;
        const uint32_t m3 = (r3 & RT_LEAF_BIT) ? 0u : __ballot_sync(FULL, h3) & alive;
        // the first needed child is visited next; the others are pushed in
        // slot order (popped last-first).  Lane c (< 4) holds child c, so
        // the pushes are one compaction, with no indexed local array.
        const uint32_t ml = lane == 0 ? m0 : lane == 1 ? m1 : lane == 2 ? m2 : m3;
        const uint32_t rl = lane == 0 ? r0 : lane == 1 ? r1 : lane == 2 ? r2 : r3;
        const uint32_t need = __ballot_sync(FULL, lane < 4 && ml != 0u);
        const int first = __ffs(need) - 1;
        const uint32_t nn = first == 0 ? r0 : first == 1 ? r1 : first == 2 ? r2 : r3;
        const uint32_t nm = first == 0 ? m0 : first == 1 ? m1 : first == 2 ? m2 : first == 3 ? m3 : 0u;
        const uint32_t pushm = need & (need - 1u);  // all but the first
        const int npush = __popc(pushm);
        if (sp + npush > RT_WIDE_STACK) {
            rt_set_error(status, RT_ERR_STACK_OVERFLOW);
            break;
        }
        if ((pushm >> lane) & 1u) stk[sp + __popc(pushm & ((1u << lane) - 1u))] = make_int2((int)rl, (int)ml);
        sp += npush;
        __syncwarp();
        if (nm) {
            node = nn;
            mask = nm;
        } else {
            mask = 0;
            while (sp > 0) {
                const int2 e = stk[--sp];
                node = (uint32_t)e.x;
                mask = (uint32_t)e.y & alive;
                if (mask) break;
            }
            __syncwarp();
        }
    }
    return T < b.t_min ? 0.0f : T;
}

// Strategy 4: one thread per ray over the 4-wide tree with a private stack,
// for rays without a shared direction (env-map samples, explicit rays).
// Multiplies the running transmittance T by this tree's accepted factors and
// stops once T < t_min (no snap: a ray may go on through other trees).
// Children in visit_order (far: farthest first).
template <bool COUNT>
__device__ __forceinline__ void trace_ray_wide_run(const BvhDev &b, float3 o, float3 d, int32_t src, float &T,
                                                   LaneLog &lg, WorkCounts &wc, int *status, bool far) {
    if (b.n <= 0) return;
    if (b.n == 1) {
        if (COUNT) wc.gauss++;
        if (src != 0 && gauss_hit(b, 0, o, d, T)) {
            if (COUNT) wc.hits++;
            log_hit(lg, b, 0);
        }
        return;
    }
    const float3 inv = safe_inv(d);
    const float3 oi = make_float3(o.x * inv.x, o.y * inv.y, o.z * inv.z);
    uint32_t stack[RT_WIDE_STACK];
    int sp = 0;
    uint32_t node = 0;
    for (;;) {
        const float4 *w = b.wide + 8 * (int64_t)node;
        const float4 lx = __ldg(w), hx = __ldg(w + 1), ly = __ldg(w + 2), hy = __ldg(w + 3), lz = __ldg(w + 4),
                     hz = __ldg(w + 5), rf = __ldg(w + 6);
        const uint32_t r[4] = {__float_as_uint(rf.x), __float_as_uint(rf.y), __float_as_uint(rf.z),
                               __float_as_uint(rf.w)};
        float tn[4];
        slab4_near(lx, hx, ly, hy, lz, hz, oi, inv, tn);
        if (COUNT) wc.box += (r[0] != RT_EMPTY) + (r[1] != RT_EMPTY) + (r[2] != RT_EMPTY) + (r[3] != RT_EMPTY);
        const float inf = __int_as_float(0x7f800000);
        float ti[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            ti[c] = inf;
            if (!(tn[c] < inf)) continue;
            if (r[c] & RT_LEAF_BIT) {
                const int32_t p = (int32_t)(r[c] & ~RT_LEAF_BIT);
                if (p != src) {
                    if (COUNT) wc.gauss++;
                    if (gauss_hit(b, p, o, d, T)) {
                        if (COUNT) wc.hits++;
                        log_hit(lg, b, p);
                    }
                }
            } else {
                ti[c] = tn[c];
            }
        }
        int next = -1;
        const bool overflow = !visit_order(ti[0], ti[1], ti[2], ti[3], r[0], r[1], r[2], r[3], far, stack, sp, next);
        if (overflow) {
            rt_set_error(status, RT_ERR_STACK_OVERFLOW);
            break;
        }
        if (T < b.t_min) break;
        if (next >= 0) {
            node = (uint32_t)next;
        } else {
            if (sp == 0) break;
            node = stack[--sp];
        }
    }
}

template <bool COUNT>
__device__ __forceinline__ float trace_ray_wide(const BvhDev &b, float3 o, float3 d, int32_t src, LaneLog &lg,
                                                WorkCounts &wc, int *status, bool far) {
    float T = 1.0f;
    trace_ray_wide_run<COUNT>(b, o, d, src, T, lg, wc, status, far);
    return T < b.t_min ? 0.0f : T;
}

// ---------------------------------------------------------------------------
// Work items of a trace job
// ---------------------------------------------------------------------------
enum { MODE_EXPLICIT = 0, MODE_FULL = 1, MODE_IDS = 2 };

struct TraceJob {
    int mode;
    const int64_t *out_index;                // MODE_IDS: output position of entry r (null = r)
    const unsigned long long *dyn_count;     // MODE_IDS: device-side entry count (null = n_out)
    int64_t n_items;
    int64_t n_tiles;      // MODE_FULL
    int32_t order_block;  // MODE_FULL: tiles per sweep
    int64_t n_out;        // outputs (rays)
    int64_t tile_base;    // MODE_FULL: first tile (a sample starts elsewhere than 0)
};

// Decode a MODE_FULL item into (tile, direction).
__device__ __forceinline__ void full_item(const TraceJob &job, int32_t K, int64_t item, int64_t &tile,
                                          int32_t &k) {
    const int64_t B = job.order_block;
    const int64_t grp = item / (B * K);
    const int64_t rem = item - grp * B * K;
    int64_t in_grp = job.n_tiles - grp * B;
    if (in_grp > B) in_grp = B;
    k = (int32_t)(rem / in_grp);
    tile = job.tile_base + grp * B + rem % in_grp;
}


// Ray r of a job in slot order: MODE_FULL slot r (item r/32, lane r%32;
// false past a ragged last tile, out_idx = -1), MODE_EXPLICIT / MODE_IDS
// entry r (an invalid id records RT_ERR_INVALID_ARG and returns false with
// out_idx set).
__device__ __forceinline__ bool ray_of(const BvhDev &b, const RaySetDev &rs, const TraceJob &job, int64_t r,
                                       float3 &o, float3 &d, int32_t &src, int64_t &out_idx, int *status) {
    src = -1;
    out_idx = -1;
    o = make_float3(0.f, 0.f, 0.f);
    d = make_float3(0.f, 0.f, 1.f);
    if (job.mode == MODE_FULL) {
        int64_t tile;
        int32_t k;
        full_item(job, rs.K, r >> 5, tile, k);
        const int64_t p = tile * 32 + (r & 31);
        if (p >= b.n) return false;
        const float4 mu = __ldg(b.gauss + 4 * p);
        const int64_t g = __float_as_int(__ldg(b.gauss + 4 * p + 1).w);
        out_idx = g * rs.K + k;
        implicit_ray(rs, out_idx, k, g, mu, o, d);
        src = (int32_t)p;
        return true;
    }
    out_idx = job.out_index ? job.out_index[r] : r;
    if (job.mode == MODE_EXPLICIT) {
        o = make_float3(rs.ray_o[3 * r], rs.ray_o[3 * r + 1], rs.ray_o[3 * r + 2]);
        d = make_float3(rs.ray_d[3 * r], rs.ray_d[3 * r + 1], rs.ray_d[3 * r + 2]);
        if (rs.ray_src) {
            const int32_t sg = rs.ray_src[r];
            src = (sg >= 0 && sg < b.n) ? b.rank[sg] : -1;
        }
        return true;
    }
    const int64_t rid = rs.ray_ids[r];
    if (rid < 0 || rid >= rs.n_rays) {
        rt_set_error(status, RT_ERR_INVALID_ARG);
        return false;
    }
    const int64_t g = rid / rs.K;
    const int32_t k = (int32_t)(rid - g * rs.K);
    const int32_t p = b.rank[g];
    implicit_ray(rs, rid, k, g, __ldg(b.gauss + 4 * (int64_t)p), o, d);
    src = p;
    return true;
}

// One work item (32 rays) of a trace job: build each lane's ray, traverse,
// write T (and the hit log).  Shared by the single-scene and batched kernels.
// STRAT: 0 per-ray binary, 1 packet binary, 2 packet 4-wide, 3 packet 4-wide
// for a direction set (all lanes share the direction), 4 per-ray 4-wide
// (stk: this warp's RT_WIDE_STACK shared-memory entries, strategies 2-3).
template <int STRAT, bool COUNT>
__device__ __forceinline__ void trace_item(const BvhDev &b, const RaySetDev &rs, const TraceJob &job,
                                           float *T_out, const TraceAux &aux, int64_t item, int64_t n_out,
                                           WorkCounts &wc, unsigned long long &rays_done, int2 *stk) {
    const int lane = threadIdx.x & 31;
    bool valid = false;
    float3 o = make_float3(0.f, 0.f, 0.f), d = make_float3(0.f, 0.f, 1.f);
    int32_t src = -1;
    int64_t out_idx = 0;
    if (job.mode == MODE_FULL) {
        int64_t tile;
        int32_t k;
        full_item(job, rs.K, item, tile, k);
        const int64_t p = tile * 32 + lane;
        if (p < b.n) {
            valid = true;
            const float4 mu = __ldg(b.gauss + 4 * p);
            const int32_t g = __float_as_int(__ldg(b.gauss + 4 * p + 1).w);
            out_idx = (int64_t)g * rs.K + k;
            implicit_ray(rs, out_idx, k, g, mu, o, d);
            src = (int32_t)p;
        }
    } else {
        const int64_t r = item * 32 + lane;
        if (r < n_out) {
            valid = true;
            out_idx = job.out_index ? job.out_index[r] : r;
            if (job.mode == MODE_EXPLICIT) {
                o = make_float3(rs.ray_o[3 * r], rs.ray_o[3 * r + 1], rs.ray_o[3 * r + 2]);
                d = make_float3(rs.ray_d[3 * r], rs.ray_d[3 * r + 1], rs.ray_d[3 * r + 2]);
                if (rs.ray_src) {
                    const int32_t s = rs.ray_src[r];
                    src = (s >= 0 && s < b.n) ? b.rank[s] : -1;
                }
            } else {
                const int64_t rid = rs.ray_ids[r];
                if (rid < 0 || rid >= rs.n_rays) {
                    rt_set_error(aux.status, RT_ERR_INVALID_ARG);
                    valid = false;
                    T_out[out_idx] = __int_as_float(0x7fc00000);
                } else {
                    const int64_t g = rid / rs.K;
                    const int32_t k = (int32_t)(rid - g * rs.K);
                    const int32_t p = b.rank[g];
                    const float4 mu = __ldg(b.gauss + 4 * (int64_t)p);
                    implicit_ray(rs, rid, k, g, mu, o, d);
                    src = p;
                }
            }
        }
    }
    LaneLog lg;
    lg.ids = (aux.hit_ids && valid) ? aux.hit_ids + out_idx * aux.cap : nullptr;
    lg.cap = aux.cap;
    lg.count = 0;
    float T;
    if (STRAT == 4) {
        T = valid ? trace_ray_wide<COUNT>(b, o, d, src, lg, wc, aux.status, far_first(rs)) : 1.0f;
    } else if (STRAT == 3) {
        T = trace_wide<COUNT, true>(b, o, d, src, valid, lg, wc, aux.status, stk);
    } else if (STRAT == 2) {
        T = trace_wide<COUNT, false>(b, o, d, src, valid, lg, wc, aux.status, stk);
    } else if (STRAT == 1) {
        T = trace_packet<COUNT>(b, o, d, src, valid, lg, wc, aux.status);
    } else {
        T = valid ? trace_ray<COUNT>(b, o, d, src, lg, wc, aux.status) : 1.0f;
    }
    if (valid) {
        T_out[out_idx] = T;
        if (aux.hit_count) aux.hit_count[out_idx] = lg.count;
        rays_done++;
    }
}

template <bool COUNT>
__device__ __forceinline__ void flush_counts(const TraceAux &aux, const WorkCounts &wc, unsigned long long rays_done) {
    if (COUNT && aux.counters) {
        const int lane = threadIdx.x & 31;
        unsigned long long v[4] = {wc.box, wc.gauss, wc.hits, rays_done};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            unsigned long long x = v[c];
            for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
            if (lane == 0 && x) atomicAdd(aux.counters + c, x);
        }
    }
}


// Strategy 5: one thread per ray over the 4-wide tree, with lanes refilled as
// their rays finish (persistent threads with dynamic ray fetch, Aila & Laine
// 2009).  Rays are the slots item*32 + l of a full implicit set (in the job's
// item order); whenever at least kRefillMin lanes of the warp are idle, lane
// 0 takes that many slots with one atomic and the idle lanes start them, so a
// warp no longer waits for its longest ray.  Each step of a lane is one node
// visit of trace_ray_wide's loop, and a ray's visits and factors come in the
// same order as there: the same T.  Slots past a ragged last tile are
// skipped.  `work` counts slots.
#ifndef RT_REFILL_MIN
#define RT_REFILL_MIN 8
#endif
constexpr int kRefillMin = RT_REFILL_MIN;

template <bool COUNT>
__device__ __forceinline__ void trace_refill(const BvhDev &b, const RaySetDev &rs, const TraceJob &job, float *T_out,
                                             const TraceAux &aux, unsigned long long *work, WorkCounts &wc,
                                             unsigned long long &rays_done) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const unsigned long long total = (unsigned long long)job.n_items * 32ull;
    bool has = false, exhausted = false;
    float3 o = make_float3(0.f, 0.f, 0.f), d = make_float3(0.f, 0.f, 1.f), inv = d, oi = o;
    int32_t src = -1;
    int64_t out_idx = 0;
    float T = 1.0f;
    uint32_t node = 0;
    int sp = 0;
    uint32_t stack[RT_WIDE_STACK];
    const bool far = far_first(rs);
    for (;;) {
        const unsigned idle = __ballot_sync(FULL, !has);
        const int n_idle = __popc(idle);
        if (!exhausted && (n_idle >= kRefillMin || n_idle == 32)) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(work, (unsigned long long)n_idle);
            base = __shfl_sync(FULL, base, 0);
            if (base + (unsigned long long)n_idle >= total) exhausted = true;
            if (!has) {
                const unsigned long long slot = base + (unsigned long long)__popc(idle & lt_mask);
                if (slot < total) {
                    int64_t tile;
                    int32_t k;
                    full_item(job, rs.K, (int64_t)(slot >> 5), tile, k);
                    const int64_t p = tile * 32 + (int64_t)(slot & 31ull);
                    if (p < b.n) {
                        const float4 mu = __ldg(b.gauss + 4 * p);
                        const int64_t g = __float_as_int(__ldg(b.gauss + 4 * p + 1).w);
                        out_idx = g * rs.K + k;
                        implicit_ray(rs, out_idx, k, g, mu, o, d);
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
        // one visit of trace_ray_wide's loop
        const float4 *w = b.wide + 8 * (int64_t)node;
        const float4 lx = __ldg(w), hx = __ldg(w + 1), ly = __ldg(w + 2), hy = __ldg(w + 3), lz = __ldg(w + 4),
                     hz = __ldg(w + 5), rf = __ldg(w + 6);
        const uint32_t r[4] = {__float_as_uint(rf.x), __float_as_uint(rf.y), __float_as_uint(rf.z),
                               __float_as_uint(rf.w)};
        float tn[4];
        slab4_near(lx, hx, ly, hy, lz, hz, oi, inv, tn);
        if (COUNT) wc.box += (r[0] != RT_EMPTY) + (r[1] != RT_EMPTY) + (r[2] != RT_EMPTY) + (r[3] != RT_EMPTY);
        const float inf = __int_as_float(0x7f800000);
        float ti[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            ti[c] = inf;
            if (!(tn[c] < inf)) continue;
            if (r[c] & RT_LEAF_BIT) {
                const int32_t p = (int32_t)(r[c] & ~RT_LEAF_BIT);
                if (p != src) {
                    if (COUNT) wc.gauss++;
                    if (gauss_hit(b, p, o, d, T) && COUNT) wc.hits++;
                }
            } else {
                ti[c] = tn[c];
            }
        }
        int next = -1;
        const bool overflow = !visit_order(ti[0], ti[1], ti[2], ti[3], r[0], r[1], r[2], r[3], far, stack, sp, next);
        if (overflow) rt_set_error(aux.status, RT_ERR_STACK_OVERFLOW);
        bool done = overflow || T < b.t_min;
        if (!done) {
            if (next >= 0) node = (uint32_t)next;
            else if (sp > 0) node = stack[--sp];
            else done = true;
        }
        if (done) {
            T_out[out_idx] = T < b.t_min ? 0.0f : T;
            rays_done++;
            has = false;
        }
    }
}

// Strategy 6: one warp per ray over the 4-wide tree, for few or latency-bound
// rays (fallback lists, small sets).  The lanes take up to 32 entries off the
// top of a shared stack, visit those nodes in parallel, multiply the factors
// of their leaf hits into lane-local partial products and push the hit
// internal children (warp prefix sum); T is the product of the partials,
// formed by a warp butterfly after every step for the early exit.  A step
// takes k = min(32, size, (cap - size)/3) entries, so the stack never exceeds
// cap (RT_ERR_STACK_OVERFLOW if no entry can be taken).  Same accepted set as
// the per-ray traversals; the product is formed in another order.
constexpr int kWarpStack = 2048;

__device__ __forceinline__ float warp_product(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v *= __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

template <bool COUNT>
__device__ __forceinline__ float trace_warp_ray(const BvhDev &b, float3 o, float3 d, int32_t src, uint32_t *wstk,
                                                WorkCounts &wc, int *status) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    float Tl = 1.0f;
    if (b.n <= 0) return 1.0f;
    if (b.n == 1) {
        if (lane == 0 && src != 0) {
            if (COUNT) wc.gauss++;
            if (gauss_hit(b, 0, o, d, Tl) && COUNT) wc.hits++;
        }
        const float T = __shfl_sync(FULL, Tl, 0);
        return T < b.t_min ? 0.0f : T;
    }
    const float3 inv = safe_inv(d);
    const float3 oi = make_float3(o.x * inv.x, o.y * inv.y, o.z * inv.z);
    if (lane == 0) wstk[0] = 0u;
    int size = 1;
    __syncwarp();
    for (;;) {
        int k = min(32, min(size, (kWarpStack - size) / 3));
        if (k <= 0) {
            if (size > 0) rt_set_error(status, RT_ERR_STACK_OVERFLOW);
            break;
        }
        const bool active = lane < k;
        const uint32_t node = active ? wstk[size - 1 - lane] : 0u;
        size -= k;
        __syncwarp();
        // internal children to push: a mask over c (a register array indexed by
        // a running count would live in local memory)
        uint32_t r[4] = {0u, 0u, 0u, 0u}, pm = 0u;
        if (active) {
            const float4 *w = b.wide + 8 * (int64_t)node;
            const float4 lx = __ldg(w), hx = __ldg(w + 1), ly = __ldg(w + 2), hy = __ldg(w + 3),
                         lz = __ldg(w + 4), hz = __ldg(w + 5), rf = __ldg(w + 6);
            r[0] = __float_as_uint(rf.x);
            r[1] = __float_as_uint(rf.y);
            r[2] = __float_as_uint(rf.z);
            r[3] = __float_as_uint(rf.w);
            bool h[4];
            slab4(lx, hx, ly, hy, lz, hz, oi, inv, h);
            if (COUNT) wc.box += (r[0] != RT_EMPTY) + (r[1] != RT_EMPTY) + (r[2] != RT_EMPTY) + (r[3] != RT_EMPTY);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (!h[c]) continue;
                if (r[c] & RT_LEAF_BIT) {
                    const int32_t p = (int32_t)(r[c] & ~RT_LEAF_BIT);
                    if (p != src) {
                        if (COUNT) wc.gauss++;
                        if (gauss_hit(b, p, o, d, Tl) && COUNT) wc.hits++;
                    }
                } else {
                    pm |= 1u << c;
                }
            }
        }
        // warp prefix sum of the pushes, then write them above the stack top
        const int n_push = __popc(pm);
        int pre = n_push;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(FULL, pre, off);
            if (lane >= off) pre += v;
        }
        const int total = __shfl_sync(FULL, pre, 31);
        int at = size + pre - n_push;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if ((pm >> c) & 1u) wstk[at++] = r[c];
        size += total;
        __syncwarp();
        if (warp_product(Tl) < b.t_min || size == 0) break;
    }
    const float T = warp_product(Tl);
    return T < b.t_min ? 0.0f : T;
}
