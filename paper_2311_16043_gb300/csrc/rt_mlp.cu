// rt_mlp.cu -- learned visibility surrogate on the 5th-generation tensor
// cores (not in the paper; the paper precomputes visibility by tracing).
//
// Network: frequency encoding of (origin, direction) -> 80 inputs ->
// 4 x 128 ReLU -> 1 sigmoid.  bf16 weights and activations, f32 accumulation
// in TMEM.  One CTA per SM; sample row r of a 128-sample tile is TMEM lane r
// of the accumulator.
//
// Inference (k_mlp_infer): the four weight images stay in shared memory; per
// tile the encoding is written to shared memory, each layer is one chain of
// tcgen05.mma (M=128, N=128, K=80/128) into TMEM, and the epilogue (bias,
// ReLU, bf16) writes the next layer's operand back to shared memory; the last
// epilogue does the 128->1 layer and the sigmoid on the CUDA cores.  Rays
// whose prediction is within `band` of 0.5 are appended (warp-aggregated
// atomics) to a fallback list that the tracer then resolves.
//
// Training (k_mlp_train, 512 threads: four warpgroups split the columns of
// every epilogue of one 128-sample tile): per tile, forward (activations kept
// in shared memory, weight images streamed by bulk async copies into two
// buffers), then backward with the same operands read K-major or MN-major:
//   dW_l += dz_l^T x_{l-1}   (M = units, N = inputs, K = samples; TMEM-resident
//                             across the CTA's tiles for l = 2..4)
//   dX_{l-1} = dz_l W_l      (M = samples, N = inputs, K = units)
// The bias gradients (sums of dz over samples) come out of the tensor cores
// through a column of ones in the input tile.  Each CTA writes one partial
// gradient; k_mlp_reduce_adam sums the partials in a fixed order
// (deterministic), applies Adam to the f32 master weights and re-packs the
// bf16 weight images.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <atomic>
#include <mutex>

#include "rt_tc.cuh"
#include "rt_trace_core.cuh"

namespace {

constexpr int H = 128;
constexpr int IN = 80;       // 78 features and two pad columns
constexpr int IN_FEAT = 78;  // the bf16 images hold zero weights in the pad columns
constexpr int OFF_W1 = 0, OFF_B1 = 10240, OFF_W2 = 10368, OFF_B2 = 26752, OFF_W3 = 26880, OFF_B3 = 43264,
              OFF_W4 = 43392, OFF_B4 = 59776, OFF_W5 = 59904, OFF_B5 = 60032, NPARAM = 60033;
constexpr int IMG_W1 = 0, IMG_W2 = 20480, IMG_W3 = 53248, IMG_W4 = 86016, IMG_BYTES = 118784;
constexpr long long WAIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz: default bound of every wait
constexpr unsigned FULL = 0xffffffffu;

__host__ __device__ __forceinline__ uint32_t img_off(int r, int c, int kdim) {
    return (uint32_t)((r >> 3) * (kdim / 8 * 128) + (c >> 3) * 128 + (r & 7) * 16 + (c & 7) * 2);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}
__device__ __forceinline__ float bf16_round(float a) { return __bfloat162float(__float2bfloat16_rn(a)); }
// bf16 pair of max(a, 0), max(b, 0) (a in the low half): one conversion with
// the ReLU folded in; rounding commutes with max(., 0), so the bits equal
// pack_bf16(fmaxf(a, 0), fmaxf(b, 0)) for finite inputs.
__device__ __forceinline__ uint32_t pack_bf16_relu(float a, float b) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
    return d;
}
__device__ __forceinline__ float bf16_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t u) { return __uint_as_float(u & 0xffff0000u); }

// Frequency encoding of one ray into 80 floats (rounded to bf16 at store).
// The sin/cos arguments pi 2^k x reach 32 pi x, so x must be far more
// accurate than one float rounding for the features to round to the same
// bf16 values as an exact evaluation.  With float32 error-free transforms:
// p - lo and hi - lo are split exactly into pairs, the quotient is a pair
// q + ql (remainder-corrected, relative error ~1e-13), x = 2 (q + ql) - 1 is
// kept as a pair xh + xl, and 2^k x is reduced modulo 2 exactly
// (t_h - 2 rint(t_h / 2) is exact) before sincospif.  No float64 is used
// (float64 throughput is very low on this part).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void normalise_pair(float p, float lo, float eh, float el, float &xh, float &xl) {
    if (eh == 0.0f) {
        xh = 0.0f;
        xl = 0.0f;
        return;
    }
    float dh, dl;
    two_diff(p, lo, dh, dl);                 // dh + dl = p - lo exactly
    const float q = __fdiv_rn(dh, eh);
    float r = fmaf(-q, eh, dh);              // exact remainder
    r = __fadd_rn(r, dl);
    r = fmaf(-q, el, r);
    const float ql = __fdiv_rn(r, eh);       // (p - lo)/(hi - lo) = q + ql
    float s, e;
    two_sum(2.0f * q, -1.0f, s, e);
    const float lo2 = __fadd_rn(e, 2.0f * ql);
    xh = __fadd_rn(s, lo2);                  // renormalise the pair
    xl = __fsub_rn(lo2, __fsub_rn(xh, s));
}

__device__ __forceinline__ void sincospi_k(float xh, float xl, int k, float &s, float &c) {
    const float th = ldexpf(xh, k), tl = ldexpf(xl, k);   // exact
    const float n = 2.0f * rintf(0.5f * th);
    const float r = __fadd_rn(__fsub_rn(th, n), tl);      // th - n exact
    sincospif(r, &s, &c);
}

__device__ __forceinline__ void encode(float3 p, float3 d, const float *lo, const float *eh, const float *el,
                                       float (&f)[IN]) {
    float xh[6], xl[6];
    normalise_pair(p.x, lo[0], eh[0], el[0], xh[0], xl[0]);
    normalise_pair(p.y, lo[1], eh[1], el[1], xh[1], xl[1]);
    normalise_pair(p.z, lo[2], eh[2], el[2], xh[2], xl[2]);
    xh[3] = d.x;
    xh[4] = d.y;
    xh[5] = d.z;
    xl[3] = xl[4] = xl[5] = 0.0f;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        f[13 * c] = xh[c];
#pragma unroll
        for (int k = 0; k < 6; k += 2) {
            // even k from the exactly reduced argument; odd k by one
            // double-angle step from it, sin 2a = 2 sin a cos a and
            // cos 2a = (cos a - sin a)(cos a + sin a): ~2 float32 ulp,
            // far below the bf16 spacing the features are rounded to
            float sv, cv;
            sincospi_k(xh[c], xl[c], k, sv, cv);
            f[13 * c + 1 + 2 * k] = sv;
            f[13 * c + 2 + 2 * k] = cv;
            f[13 * c + 3 + 2 * k] = 2.0f * (sv * cv);
            f[13 * c + 4 + 2 * k] = (cv - sv) * (cv + sv);
        }
    }
    f[78] = 0.0f;
    f[79] = 0.0f;
}

__device__ __forceinline__ void store_row_x0(uint8_t *x0, int r, const float (&f)[IN]) {
#pragma unroll
    for (int q = 0; q < IN / 8; ++q) {
        uint4 v;
        v.x = pack_bf16(f[8 * q + 0], f[8 * q + 1]);
        v.y = pack_bf16(f[8 * q + 2], f[8 * q + 3]);
        v.z = pack_bf16(f[8 * q + 4], f[8 * q + 5]);
        v.w = pack_bf16(f[8 * q + 6], f[8 * q + 7]);
        *reinterpret_cast<uint4 *>(x0 + img_off(r, 8 * q, IN)) = v;
    }
}

// 32 values of row r, columns c0..c0+31, to a K-major bf16 image (kdim 128).
__device__ __forceinline__ void store_chunk(uint8_t *img, int r, int c0, const float (&v)[32]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint4 u;
        u.x = pack_bf16(v[8 * q + 0], v[8 * q + 1]);
        u.y = pack_bf16(v[8 * q + 2], v[8 * q + 3]);
        u.z = pack_bf16(v[8 * q + 4], v[8 * q + 5]);
        u.w = pack_bf16(v[8 * q + 6], v[8 * q + 7]);
        *reinterpret_cast<uint4 *>(img + img_off(r, c0 + 8 * q, H)) = u;
    }
}

// As store_chunk with the ReLU applied in the conversion.
__device__ __forceinline__ void store_chunk_relu(uint8_t *img, int r, int c0, const float (&v)[32]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint4 u;
        u.x = pack_bf16_relu(v[8 * q + 0], v[8 * q + 1]);
        u.y = pack_bf16_relu(v[8 * q + 2], v[8 * q + 3]);
        u.z = pack_bf16_relu(v[8 * q + 4], v[8 * q + 5]);
        u.w = pack_bf16_relu(v[8 * q + 6], v[8 * q + 7]);
        *reinterpret_cast<uint4 *>(img + img_off(r, c0 + 8 * q, H)) = u;
    }
}

// Row r, columns c0..c0+31, of a K-major bf16 image (kdim 128) as 16 bf16
// pairs (column c0 + 2k in the low half of u[k]), and back.
__device__ __forceinline__ void load_chunk_raw(const uint8_t *img, int r, int c0, uint32_t (&u)[16]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint4 x = *reinterpret_cast<const uint4 *>(img + img_off(r, c0 + 8 * q, H));
        u[4 * q] = x.x;
        u[4 * q + 1] = x.y;
        u[4 * q + 2] = x.z;
        u[4 * q + 3] = x.w;
    }
}
__device__ __forceinline__ void store_chunk_raw(uint8_t *img, int r, int c0, const uint32_t (&u)[16]) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4 *>(img + img_off(r, c0 + 8 * q, H)) =
            make_uint4(u[4 * q], u[4 * q + 1], u[4 * q + 2], u[4 * q + 3]);
}
// Per half of a bf16 pair: all ones where the value is > 0, else zero (NaN: zero).
__device__ __forceinline__ uint32_t bf16x2_pos_mask(uint32_t u) {
    __nv_bfloat162 h;
    memcpy(&h, &u, sizeof(u));
    return __hgt2_mask(h, __float2bfloat162_rn(0.0f));
}

// Warp transpose-reduction: afterwards lane l holds sum over the warp's
// lanes of v[l] (31 shuffles for 32 columns).  Destroys v.
template <int S>
__device__ __forceinline__ void tr_step(float (&v)[32], int lane) {
    const bool upper = (lane & S) != 0;
#pragma unroll
    for (int i = 0; i < S; ++i) {
        float keep = upper ? v[i + S] : v[i];
        float send = upper ? v[i] : v[i + S];
        v[i] = keep + __shfl_xor_sync(FULL, send, S);
    }
}
__device__ __forceinline__ float transpose_reduce32(float (&v)[32], int lane) {
    tr_step<16>(v, lane);
    tr_step<8>(v, lane);
    tr_step<4>(v, lane);
    tr_step<2>(v, lane);
    tr_step<1>(v, lane);
    return v[0];
}

// Chain of MMAs D (+)= A * B^T over K in steps of 16.
__device__ __forceinline__ void issue_mma(uint32_t tmem_d, uint32_t a, uint32_t a_lbo, uint32_t a_sbo,
                                          uint32_t a_kstep, uint32_t b, uint32_t b_lbo, uint32_t b_sbo,
                                          uint32_t b_kstep, uint32_t idesc, int K, bool acc_first) {
    // a descriptor's start-address field is bits 0-13 (address / 16); shared
    // addresses stay below 2^18 bytes, so stepping the address adds to the
    // descriptor without a carry out of that field
    const uint64_t da = tc_smem_desc(a, a_lbo, a_sbo), db = tc_smem_desc(b, b_lbo, b_sbo);
    for (int kk = 0; kk < K / 16; ++kk)
        tc_mma(tmem_d, da + (uint64_t)((kk * a_kstep) >> 4), db + (uint64_t)((kk * b_kstep) >> 4), idesc,
               (kk > 0 || acc_first) ? 1u : 0u);
}

// Sample sources
struct SampleSrc {
    int mode;  // 0 explicit pos/dir(/y); 1 implicit set (rays); 2 implicit, Philox-drawn training ids
    const float *pos, *dir, *y;
    BvhDev b;
    RaySetDev rs;
    const float *T_target;
    uint64_t seed;
    int64_t step;
    int64_t R;  // rays in the implicit set
    // training (mode 2): per-CTA buffer of one tile's drawn samples
    // ([gridDim][7][128] floats); pf_use: this launch's first tile is there
    // (drawn by the previous step's launch); pf_make: draw the next step's
    // first tile into it
    float *pf;
    int pf_use, pf_make;
};

__device__ __forceinline__ bool get_sample(const SampleSrc &S, int64_t i, int64_t m, float3 &p, float3 &d,
                                           float &y, int64_t &rid) {
    if (i >= m) return false;
    if (S.mode == 0) {
        p = make_float3(S.pos[3 * i], S.pos[3 * i + 1], S.pos[3 * i + 2]);
        d = make_float3(S.dir[3 * i], S.dir[3 * i + 1], S.dir[3 * i + 2]);
        y = S.y ? S.y[i] : 0.0f;
        rid = i;
        return true;
    }
    if (S.mode == 1) {
        rid = S.rs.ray_ids ? S.rs.ray_ids[i] : i;
    } else {
        // uniform id in [0, R): the high 64 bits of x * R for a uniform
        // 64-bit x (bias below R / 2^64)
        uint64_t c[4] = {(uint64_t)i, (uint64_t)S.step, 0ull, 0ull};
        philox4x64_10(c, S.seed, 1ull);
        rid = (int64_t)__umul64hi(c[0], (uint64_t)S.R);
    }
    if (rid < 0 || rid >= S.R) return false;  // reported by the caller's status check
    int64_t g;
    int32_t k;
    if (rid <= 0xffffffffll) {  // 32-bit division when the id fits
        const uint32_t r32 = (uint32_t)rid, g32 = r32 / (uint32_t)S.rs.K;
        g = g32;
        k = (int32_t)(r32 - g32 * (uint32_t)S.rs.K);
    } else {
        g = rid / S.rs.K;
        k = (int32_t)(rid - g * S.rs.K);
    }
    const int32_t ps = S.b.rank[g];
    implicit_ray(S.rs, rid, k, g, __ldg(S.b.gauss + 4 * (int64_t)ps), p, d);
    y = S.T_target ? S.T_target[rid] : 0.0f;
    return true;
}

// The training kernel draws a sample in three steps spread over one tile
// (see k_mlp_train): sample_index gives the ids without any load; the
// Gaussian's sorted position, the target and then the mean arrive by
// asynchronous copies; the ray is formed last.
// The id of sample i without any load: ray id, Gaussian (caller order) and
// direction index; ok = false beyond the minibatch or for an invalid id.
struct SampleIdx {
    int64_t rid, g;
    int32_t k;
    bool ok;
};

__device__ __forceinline__ SampleIdx sample_index(const SampleSrc &S, int64_t i, int64_t m, int64_t step) {
    SampleIdx o;
    o.rid = i;
    o.g = 0;
    o.k = 0;
    o.ok = false;
    if (i >= m) return o;
    if (S.mode == 0) {
        o.ok = true;
        return o;
    }
    uint64_t c[4] = {(uint64_t)i, (uint64_t)step, 0ull, 0ull};
    philox4x64_10(c, S.seed, 1ull);
    const int64_t rid = (int64_t)__umul64hi(c[0], (uint64_t)S.R);
    if (rid < 0 || rid >= S.R) return o;
    if (rid <= 0xffffffffll) {
        const uint32_t r32 = (uint32_t)rid, g32 = r32 / (uint32_t)S.rs.K;
        o.g = g32;
        o.k = (int32_t)(r32 - g32 * (uint32_t)S.rs.K);
    } else {
        o.g = rid / S.rs.K;
        o.k = (int32_t)(rid - o.g * S.rs.K);
    }
    o.rid = rid;
    o.ok = true;
    return o;
}

// 4-byte asynchronous copy global -> shared (Ampere-style cp.async), and its
// group commit / wait.
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

struct MlpDev {
    const float *params;  // f32 master
    const uint8_t *img;   // bf16 images
    float lo[3];          // origin normalisation x = 2 (p - lo)/(hi - lo) - 1 with
    float eh[3], el[3];   // hi - lo = eh + el exactly
    float pos_w;          // weight w of the lit term of the loss
    long long wait_cycles;  // bound of the first wait on each MMA commit
};

// ---------------------------------------------------------------------------
// Inference
// ---------------------------------------------------------------------------
// INF_WG warpgroups per CTA work on separate tiles (own activation buffer,
// TMEM columns and mbarrier, named barrier 1 + g) and share the weight
// images, so one group's MMAs run while the others encode or run epilogues.
constexpr int INF_WG = 3;
constexpr int INF_SMEM_ACT = IMG_BYTES;                          // INF_WG x 32768
constexpr int INF_SMEM_B = INF_SMEM_ACT + INF_WG * 32768;        // b1..b4, w5: 5*128 floats
constexpr int INF_SMEM_BAR = INF_SMEM_B + 5 * 128 * 4;           // 2 x INF_WG mbarriers + tmem slot
constexpr int INF_SMEM_TOTAL = INF_SMEM_BAR + 64;
static_assert(2 * INF_WG * 8 + 4 <= 64, "barrier area of the inference kernel");

__device__ __forceinline__ void wg_sync(int g) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(128) : "memory");
}

// True iff v holds in all 128 threads of warpgroup g (a barrier of the group
// with an AND reduction), so that the group takes every exit together.
__device__ __forceinline__ bool wg_all(int g, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"(v ? 1u : 0u), "r"(1 + g)
        : "memory");
    return r != 0;
}

// Layer l's bias into this thread's accumulator row (128 columns), so the
// MMA accumulates onto it and the epilogue adds nothing.
__device__ __forceinline__ void tmem_store_bias(uint32_t lane_addr, const float *b) {
#pragma unroll 1
    for (int cc = 0; cc < 4; ++cc) {
        float v[32];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float4 x = reinterpret_cast<const float4 *>(b + 32 * cc)[q];
            v[4 * q] = x.x;
            v[4 * q + 1] = x.y;
            v[4 * q + 2] = x.z;
            v[4 * q + 3] = x.w;
        }
        tmem_st32(lane_addr + 32 * cc, v);
    }
}

// out[i] is the network output p (decode == 0) or the visibility estimate
// p / (p + w (1 - p)) = 1 / (1 + w e^-z) (decode != 0).
__global__ void __launch_bounds__(128 * INF_WG, 1) k_mlp_infer(MlpDev net, SampleSrc S, int64_t m, float *out,
                                                               int decode, float band, int64_t *fb_rid,
                                                               int64_t *fb_pos, unsigned long long *fb_count,
                                                               int *status) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *wimg = smem;
    float *bias = reinterpret_cast<float *>(smem + INF_SMEM_B);  // [4][128], then w5[128]
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + INF_SMEM_BAR);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + INF_SMEM_BAR + 16 * INF_WG);
    const int t = threadIdx.x, g = t >> 7, tl = t & 127, wq = tl >> 5, lane = t & 31;
    uint8_t *act = smem + INF_SMEM_ACT + g * 32768;
    uint64_t *bar = bars + g;

    for (int i = t; i < IMG_BYTES / 16; i += 128 * INF_WG)
        reinterpret_cast<uint4 *>(wimg)[i] = __ldg(reinterpret_cast<const uint4 *>(net.img) + i);
    for (int i = t; i < 128; i += 128 * INF_WG) {
        bias[i] = net.params[OFF_B1 + i];
        bias[128 + i] = net.params[OFF_B2 + i];
        bias[256 + i] = net.params[OFF_B3 + i];
        bias[384 + i] = net.params[OFF_B4 + i];
        bias[512 + i] = net.params[OFF_W5 + i];
    }
    const float b5 = net.params[OFF_B5];
    if (t == 0)
        for (int k = 0; k < 2 * INF_WG; ++k) mbar_init(bars + k, 1);  // MMA commits, then drains
    if (t < 32) tmem_alloc(tslot, 512);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot + (uint32_t)(g * 128);  // this group's 128 columns
    const uint32_t lane_addr = tmem + ((uint32_t)(wq * 32) << 16);
    const uint32_t a_addr = smem_u32(act);
    const uint32_t w_addr = smem_u32(wimg);
    const uint32_t idesc = tc_idesc_bf16(128, 128, false, false);
    uint32_t phase = 0;
    bool ok = true;
    const int64_t ntiles = (m + 127) / 128;

    for (int64_t tile = (int64_t)blockIdx.x * INF_WG + g; tile < ntiles && ok; tile += (int64_t)gridDim.x * INF_WG) {
        const int64_t i = tile * 128 + tl;
        float3 p = make_float3(0.f, 0.f, 0.f), d = make_float3(0.f, 0.f, 1.f);
        float y;
        int64_t rid = -1;
        const bool valid = get_sample(S, i, m, p, d, y, rid);
        {
            float f[IN];
            if (valid) encode(p, d, net.lo, net.eh, net.el, f);
            else
#pragma unroll
                for (int k = 0; k < IN; ++k) f[k] = 0.0f;
            store_row_x0(act, tl, f);
        }
        tmem_store_bias(lane_addr, bias);
        float2 z5p = make_float2(0.0f, 0.0f);  // even / odd units of the output layer
        for (int l = 0; l < 4; ++l) {
            tmem_st_wait();
            fence_async_smem();
            tc_fence_before();
            wg_sync(g);
            if (tl == 0) {
                tc_fence_after();
                const int K = l == 0 ? IN : H;
                const uint32_t sbo = (uint32_t)(K / 8 * 128);
                const uint32_t wb = w_addr + (l == 0 ? IMG_W1 : l == 1 ? IMG_W2 : l == 2 ? IMG_W3 : IMG_W4);
                issue_mma(tmem, a_addr, 128, sbo, 256, wb, 128, sbo, 256, idesc, K, true);  // onto the bias
                tc_commit(bar);
            }
            // a wait that gives up marks this thread; the thread still runs
            // the tile's remaining steps (garbage values, no early exit), so
            // the group stays in step until it votes at the end of the tile
            if (!mbar_wait(bar, phase, net.wait_cycles)) ok = false;
            phase ^= 1u;
            tc_fence_after();
#pragma unroll 1
            for (int cc = 0; cc < 4; ++cc) {
                float v[32];
                tmem_ld32(lane_addr + 32 * cc, v);
                if (l < 3) {
                    store_chunk_relu(act, tl, 32 * cc, v);
                } else {
                    // z5 += w5_k bf16(relu(h_k)), two units per packed FMA
                    const float2 *w5 = reinterpret_cast<const float2 *>(bias + 512 + 32 * cc);
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const uint32_t hq = pack_bf16_relu(v[2 * q], v[2 * q + 1]);
                        z5p = __ffma2_rn(make_float2(bf16_lo(hq), bf16_hi(hq)), w5[q], z5p);
                    }
                }
            }
            if (l < 3) tmem_store_bias(lane_addr, bias + 128 * (l + 1));
        }
        if (valid) {
            const float z5 = b5 + (z5p.x + z5p.y);
            const float ez = __expf(-z5);
            const float pr = 1.0f / (1.0f + ez);
            out[i] = decode ? 1.0f / (1.0f + net.pos_w * ez) : pr;
            const bool fb = band > 0.0f && fabsf(pr - 0.5f) < band;
            const uint32_t mask = __ballot_sync(__activemask(), fb);
            if (fb) {
                const int leader = __ffs(mask) - 1;
                unsigned long long base = 0;
                if (lane == leader) base = atomicAdd(fb_count, (unsigned long long)__popc(mask));
                base = __shfl_sync(mask, base, leader);
                const unsigned long long slot = base + __popc(mask & ((1u << lane) - 1u));
                fb_rid[slot] = rid;
                fb_pos[slot] = i;
            }
        }
        tc_fence_before();
        // the end-of-tile barrier doubles as the vote: the group leaves
        // together after a give-up anywhere in it, once its MMAs are done
        if (!wg_all(g, ok)) {
            ok = false;
            if (tl == 0) {
                tc_commit(bars + INF_WG + g);  // completes when all MMAs issued so far have
                rt_set_error(status, RT_ERR_TIMEOUT);
            }
            mbar_wait(bars + INF_WG + g, 0, WAIT_CYCLES);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (t < 32) tmem_dealloc(*tslot, 512);
}

// ---------------------------------------------------------------------------
// Training: forward + backward of a minibatch, per-CTA partial gradients
// ---------------------------------------------------------------------------
// 512 threads = 4 warpgroups on one 128-sample tile at a time: thread t owns
// sample row r = t % 128 (TMEM lane r) and warpgroup q = t / 128 owns
// columns [32q, 32q + 32) of every 128-wide epilogue, so each epilogue is a
// quarter of a row per thread and 16 warps hide each other's latencies.
// Weight images stream through two shared-memory buffers by bulk async
// copies (cp.async.bulk, completion on an mbarrier) issued as soon as the
// MMA that last read the buffer has finished, so each copy overlaps the next
// MMA and epilogue.  Per tile the buffers hold, in use order,
//   forward  L1: B0 = W1   L2: B1 = W2   L3: B0 = W3   L4: B1 = W4
//   backward dX3: B1 = W4  dX2: B0 = W3  dX1: B1 = W2
// and the copies are W3 -> B0 after L1, W4 -> B1 after L2, W2 -> B1 after
// dX3 and (if another tile follows) W1 -> B0 after dX2; the next tile then
// finds W1 in B0 and W2 in B1.  Warpgroup 3, which has neither encoding nor
// dW1 work, draws the next tile's samples into a second sample buffer: the
// ids while warpgroups 0-2 encode (the sorted position and the target then
// arrive by asynchronous copies), the mean's copies after its last forward
// epilogue and the rays while warpgroups 0-2 add the dW1 tile, four MMA
// phases apart, so the two rounds of dependent global loads do not stall
// the tile.
constexpr int TR_THREADS = 512;
constexpr int TR_PSTRIDE = 60040;                // floats per partial (NPARAM + 1 rounded up to 8)
constexpr int TR_WB0 = 0;                        // 32768: weight buffer 0
constexpr int TR_WB1 = TR_WB0 + 32768;           // 32768: weight buffer 1
constexpr int TR_X0 = TR_WB1 + 32768;            // 20480
constexpr int TR_H1 = TR_X0 + 20480;             // 32768 each
constexpr int TR_H2 = TR_H1 + 32768;
constexpr int TR_H3 = TR_H2 + 32768;
constexpr int TR_DZ = TR_H3 + 32768;
// floats: b[4][128], w5[128], db[4][128], dw5[128], z5 partials [4][128]
// (then dw5 partials per warp), misc[16]
constexpr int TR_F = TR_DZ + 32768;
// samples of the current and the next tile: [2][7][128] floats (p, d, y;
// y < 0 marks a row beyond the minibatch)
constexpr int TR_SMP = TR_F + (4 * 128 + 128 + 4 * 128 + 128 + 4 * 128 + 16) * 4;
constexpr int TR_BAR = TR_SMP + 2 * 7 * 128 * 4;
constexpr int TR_SMEM_TOTAL = TR_BAR + 64;
static_assert(TR_SMEM_TOTAL <= 232448, "shared memory of the training kernel");
constexpr int TR_ROWB = 528;  // padded row of the dW staging area at the flush
static_assert(3 * 128 * TR_ROWB <= TR_F && TR_ROWB % 16 == 0, "dW staging below the float area");
static_assert(TR_PSTRIDE >= NPARAM + 1 && TR_PSTRIDE % 4 == 0, "partial stride");

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Bulk async copy global -> shared (16-byte aligned, size a multiple of 16);
// completes `bytes` of transaction count on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Programmatic dependent launch: wait until the grid launched before this
// one in the stream has completed and its memory is visible (immediate when
// this grid was launched without the attribute), and allow the grid
// launched after this one to start early.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dependents_launch() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Bulk async copy shared -> global (16-byte aligned, size a multiple of 16)
// in this thread's bulk group; bulk_commit_wait() waits for the group's
// copies to complete.
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit_wait() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// 13 features of one scalar x (held as the pair xh + xl, see encode()):
// x, then sin and cos of 2^k pi x for k = 0..5.
__device__ __forceinline__ void encode_scalar(float xh, float xl, float *f) {
    f[0] = xh;
#pragma unroll
    for (int k = 0; k < 6; k += 2) {
        float sv, cv;
        sincospi_k(xh, xl, k, sv, cv);
        f[1 + 2 * k] = sv;
        f[2 + 2 * k] = cv;
        f[3 + 2 * k] = 2.0f * (sv * cv);
        f[4 + 2 * k] = (cv - sv) * (cv + sv);
    }
}

// Features [26q, 26q + 26) of row r (warpgroups 0..2: scalars 2q and 2q + 1
// of (p_n, d)), written as bf16 pairs: the values of encode() +
// store_row_x0.  Warpgroup 2 also writes the pad columns as (1, 0): the
// weight images are zero there, so the forward is unchanged, and the dW1
// product's column 78 becomes the sum over samples of dz1, the gradient of
// the layer-1 bias; the B operand of the other layers' bias-gradient
// products is this tile's columns 64..79.
__device__ __forceinline__ void encode_part(uint8_t *x0, int r, int q, bool valid, float3 p, float3 d,
                                            const MlpDev &net) {
    if (q > 2) return;
    float xh[2] = {0.0f, 0.0f}, xl[2] = {0.0f, 0.0f};
    if (valid) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int c = 2 * q + j;
            if (c < 3) {
                const float pc = c == 0 ? p.x : c == 1 ? p.y : p.z;
                // selects, not net.lo[c]: a run-time index into the kernel
                // parameter makes the compiler copy it to local memory
                const float lo = c == 0 ? net.lo[0] : c == 1 ? net.lo[1] : net.lo[2];
                const float eh = c == 0 ? net.eh[0] : c == 1 ? net.eh[1] : net.eh[2];
                const float el = c == 0 ? net.el[0] : c == 1 ? net.el[1] : net.el[2];
                normalise_pair(pc, lo, eh, el, xh[j], xl[j]);
            } else {
                xh[j] = c == 3 ? d.x : c == 4 ? d.y : d.z;
            }
        }
    }
    float f[26];
    if (valid) {
        encode_scalar(xh[0], xl[0], f);
        encode_scalar(xh[1], xl[1], f + 13);
    } else {
#pragma unroll
        for (int k = 0; k < 26; ++k) f[k] = 0.0f;
    }
#pragma unroll
    for (int k = 0; k < 13; ++k)
        *reinterpret_cast<uint32_t *>(x0 + img_off(r, 26 * q + 2 * k, IN)) = pack_bf16(f[2 * k], f[2 * k + 1]);
    if (q == 2) *reinterpret_cast<uint32_t *>(x0 + img_off(r, IN_FEAT, IN)) = 0x3f80u;  // bf16 (1, 0)
}

// a[0..3] += (x, y, z, w) in global memory without a return value (one
// vector reduction; `a` 16-byte aligned), or a[0..3] = (x, y, z, w) when
// `store` (the first tile of a partial: no zero fill before it).
__device__ __forceinline__ void add_v4(float *a, float x, float y, float z, float w, bool store) {
    if (store)
        *reinterpret_cast<float4 *>(a) = make_float4(x, y, z, w);
    else
        asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(a), "f"(x), "f"(y), "f"(z), "f"(w)
                     : "memory");
}

__global__ void __launch_bounds__(TR_THREADS, 1) k_mlp_train(MlpDev net, SampleSrc S, int64_t m, float inv_batch,
                                                             float *partial, int *status) {
    extern __shared__ __align__(1024) uint8_t smem[];
    // buffers by index: arithmetic, not arrays (no local-memory copies)
    auto wb = [&](int b) { return smem + TR_WB0 + 32768 * b; };
    uint8_t *x0 = smem + TR_X0;
    auto hb = [&](int i) { return smem + TR_H1 + 32768 * i; };
    uint8_t *dz = smem + TR_DZ;
    float *fb = reinterpret_cast<float *>(smem + TR_F);
    float *bias = fb;             // [4][128]
    float *w5 = fb + 512;         // [128]
    float *dbias = fb + 640;      // [4][128]
    float *dw5 = fb + 1152;       // [128]
    float *z5p = fb + 1280;       // [4][128] per-warpgroup partial logits, then per-warp dw5 sums
    float *misc = fb + 1792;      // [0] db5, [1] loss; [8 + w], [12 + w]: warp w's loss, db5 sums
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + TR_BAR);  // MMA commits
    uint64_t *wbar = bar + 1;                                      // [2] weight copies; bar[3]: drain
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + TR_BAR + 32);
    float *smp = reinterpret_cast<float *>(smem + TR_SMP);  // [2][7][128]
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int r = t & 127, q = t >> 7, c0 = 32 * q;
    float *part = partial + (int64_t)blockIdx.x * TR_PSTRIDE;

    const int64_t ntiles = (m + 127) / 128;
    const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * per;
    const int64_t t1 = t0 + per < ntiles ? t0 + per : ntiles;
    if (t0 >= t1) return;  // no tiles: no partial (the reduction reads the first ceil(ntiles / per))
    // Until the grid-dependency wait below the kernel reads nothing that the
    // launch before it in the stream (the partial reduction and Adam step of
    // the previous training step, which may still be running under a
    // programmatic dependent launch) writes, and writes nothing it reads:
    // shared memory and TMEM set-up, the first tile's samples and encoding.
    if (t < 128) {
        dw5[t] = 0.0f;
#pragma unroll
        for (int l = 0; l < 4; ++l) dbias[128 * l + t] = 0.0f;
    }
    if (t < 16) misc[t] = 0.0f;
    if (t == 0) {
        mbar_init(bar, 1);
        mbar_init(wbar, 1);
        mbar_init(wbar + 1, 1);
        mbar_init(bar + 3, 1);
    }
    if (warp == 0) tmem_alloc(tslot, 512);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t tm_work = tmem;
    auto tm_dw = [&](int i) { return tmem + 128u * (uint32_t)(i + 1); };  // dW2, dW3, dW4
    const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
    const uint32_t s_wb0 = smem_u32(wb(0));
    auto s_wb = [&](int b) { return s_wb0 + 32768u * (uint32_t)b; };
    const uint32_t s_x0 = smem_u32(x0), s_dz = smem_u32(dz);
    const uint32_t s_h0 = smem_u32(hb(0));
    auto s_h = [&](int i) { return s_h0 + 32768u * (uint32_t)i; };
    const uint32_t id_fwd = tc_idesc_bf16(128, 128, false, false);
    const uint32_t id_dw = tc_idesc_bf16(128, 128, true, true);
    const uint32_t id_dw1 = tc_idesc_bf16(128, IN, true, true);
    const uint32_t id_dx = tc_idesc_bf16(128, 128, false, true);
    const uint32_t id_db = tc_idesc_bf16(128, 16, true, true);
    uint32_t phase = 0;
    bool ok = true;


    // weight copies (thread 0 only): bit b of `pend` / `wph` is buffer b's
    // pending flag / phase
    uint32_t pend = 0u, wph = 0u;
    bool wok = true;
    auto load_w = [&](int b, int img_off_bytes, int bytes) {
        if ((pend >> b) & 1u) return;  // only after a give-up: one copy per buffer and phase
        mbar_expect_tx(wbar + b, (uint32_t)bytes);
        bulk_g2s(wb(b), net.img + img_off_bytes, (uint32_t)bytes, wbar + b);
        pend |= 1u << b;
    };
    auto need_w = [&](int b) {
        if ((pend >> b) & 1u) {
            if (mbar_wait(wbar + b, (wph >> b) & 1u, net.wait_cycles)) {
                wph ^= 1u << b;
                pend &= ~(1u << b);
            } else {
                wok = false;
            }
        }
    };
    // row r's sample of tile `tile` into sample buffer b (warpgroup 3), in
    // three stages: ids (slots 0, 1: ray id; 3: direction index; 2: sorted
    // position and 6: target by asynchronous copy), the mean (slots 4, 5, 2
    // by asynchronous copy), the ray (slots 0-5)
    auto draw_ids = [&](int64_t tile, int b, int64_t step) {
        float *o = smp + b * 7 * 128 + r;
        const SampleIdx a = sample_index(S, tile * 128 + r, m, step);
        o[0] = __int_as_float((int)(a.rid & 0xffffffff));
        o[128] = __int_as_float((int)(a.rid >> 32));
        o[384] = __int_as_float(a.k);
        if (a.ok) {
            // the Gaussian's sorted position and the target land in shared
            // memory asynchronously; draw_ray waits for them
            if (S.mode != 0) cp_async4(o + 256, S.b.rank + a.g);
            if (S.mode == 0 ? S.y != nullptr : S.T_target != nullptr)
                cp_async4(o + 768, S.mode == 0 ? S.y + a.rid : S.T_target + a.rid);
            else
                o[768] = 0.0f;
            cp_async_commit();
        } else {
            o[768] = -1.0f;
        }
    };
    // second stage: the sorted position has landed; the Gaussian's mean
    // follows by three asynchronous copies into slots 4, 5 and 2
    auto draw_mean = [&](int b) {
        cp_async_wait_all();
        float *o = smp + b * 7 * 128 + r;
        if (S.mode != 0 && o[768] >= 0.0f) {
            const float *mu = reinterpret_cast<const float *>(S.b.gauss + 4 * (int64_t)__float_as_int(o[256]));
            cp_async4(o + 512, mu);
            cp_async4(o + 640, mu + 1);
            cp_async4(o + 256, mu + 2);
            cp_async_commit();
        }
    };
    // third stage: the ray
    auto draw_ray = [&](int b) {
        cp_async_wait_all();
        float *o = smp + b * 7 * 128 + r;
        const int64_t rid = (int64_t)(uint32_t)__float_as_int(o[0]) | ((int64_t)__float_as_int(o[128]) << 32);
        float3 p = make_float3(0.f, 0.f, 0.f), d = make_float3(0.f, 0.f, 1.f);
        if (o[768] >= 0.0f) {
            if (S.mode == 0) {
                p = make_float3(S.pos[3 * rid], S.pos[3 * rid + 1], S.pos[3 * rid + 2]);
                d = make_float3(S.dir[3 * rid], S.dir[3 * rid + 1], S.dir[3 * rid + 2]);
            } else {
                const int64_t g = S.rs.kind == RT_RAYS_HEMI ? rid / S.rs.K : 0;  // only hemisphere sets use it
                implicit_ray(S.rs, rid, __float_as_int(o[384]), g, make_float4(o[512], o[640], o[256], 0.0f), p,
                             d);
            }
        }
        o[0] = p.x;
        o[128] = p.y;
        o[256] = p.z;
        o[384] = d.x;
        o[512] = d.y;
        o[640] = d.z;
    };
    if (q == 3) {
        if (S.pf_use) {
            const float *pf = S.pf + (int64_t)blockIdx.x * 7 * 128 + r;
#pragma unroll
            for (int j = 0; j < 7; ++j) smp[128 * j + r] = pf[128 * j];
        } else {
            draw_ids(t0, 0, S.step);
            draw_mean(0);
            draw_ray(0);
        }
    }
    __syncthreads();
    if (q < 3) {  // the first tile's encoding (the loop encodes the others)
        const float *smr = smp + r;
        encode_part(x0, r, q, smr[768] >= 0.0f, make_float3(smr[0], smr[128], smr[256]),
                    make_float3(smr[384], smr[512], smr[640]), net);
    }
    grid_dependency_wait();
    if (t < 128) {
        bias[t] = net.params[OFF_B1 + t];
        bias[128 + t] = net.params[OFF_B2 + t];
        bias[256 + t] = net.params[OFF_B3 + t];
        bias[384 + t] = net.params[OFF_B4 + t];
        w5[t] = net.params[OFF_W5 + t];
    }
    const float b5 = net.params[OFF_B5];
    if (t == 0) {
        load_w(0, IMG_W1, 20480);
        load_w(1, IMG_W2, 32768);
    }
    __syncthreads();

    auto sync_mma = [&]() {
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
    };
    // a wait that gives up (thread 0: also a weight copy) marks this thread;
    // the thread still runs the tile's remaining steps (garbage values, no
    // early exit), so the CTA stays in step until it votes at the end of the
    // tile, then leaves together once its MMAs are done
    auto wait_mma = [&]() {
        if (!mbar_wait(bar, phase, net.wait_cycles)) ok = false;
        if (t == 0 && !wok) ok = false;
        phase ^= 1u;
        tc_fence_after();
    };

    for (int64_t tile = t0; tile < t1 && ok; ++tile) {
        const bool first = tile == t0;
        const int sb = (int)((tile - t0) & 1);
        // warpgroup 3 draws the samples of the CTA's next tile, or after the
        // last one those of its first tile in the next training step
        const bool more = tile + 1 < t1, ahead = more || S.pf_make;
        const float *smr = smp + sb * 7 * 128 + r;
        const float y = smr[768];
        const bool valid = y >= 0.0f;
        if (q < 3) {
            if (!first)
                encode_part(x0, r, q, valid, make_float3(smr[0], smr[128], smr[256]),
                            make_float3(smr[384], smr[512], smr[640]), net);
        } else if (ahead) {
            draw_ids(more ? tile + 1 : t0, sb ^ 1, more ? S.step : S.step + 1);  // completed in the dW1 phase
        }
        // ---- forward: layer l reads x_l (x0, h1, h2, h3) and W_{l+1} ----
        float h4[32];
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            sync_mma();
            if (t == 0) {
                tc_fence_after();
                const int b = l & 1;
                need_w(b);
                if (wok) {
                    const int K = l == 0 ? IN : H;
                    const uint32_t sbo = (uint32_t)(K / 8 * 128);
                    const uint32_t a = l == 0 ? s_x0 : s_h(l - 1);
                    issue_mma(tm_work, a, 128, sbo, 256, s_wb(b), 128, sbo, 256, id_fwd, K, false);
                }
                tc_commit(bar);
            }
            wait_mma();
            if (t == 0) {
                if (l == 0) load_w(0, IMG_W3, 32768);  // W1 read: B0 takes W3
                if (l == 1) load_w(1, IMG_W4, 32768);  // W2 read: B1 takes W4
            }
            // h = bf16(relu(x W^T + b)), the ReLU folded into the conversion;
            // the bias is added after the MMA in float32 (accumulating the
            // products onto a bias stored in TMEM measured a larger gradient
            // error, through ReLU decisions at pre-activations near 0)
            float v[32];
            tmem_ld32(tm_work + lane_off + c0, v);
#pragma unroll
            for (int k = 0; k < 32; ++k) v[k] += bias[128 * l + c0 + k];
            if (l < 3) {
                store_chunk_relu(hb(l), r, c0, v);
            } else {
                float zp = 0.0f;
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    h4[k] = bf16_round(fmaxf(v[k], 0.0f));
                    zp = fmaf(w5[c0 + k], h4[k], zp);
                }
                z5p[128 * q + r] = zp;
                // four MMA phases after the ids: their gathers have landed
                if (q == 3 && ahead) draw_mean(sb ^ 1);
            }
        }
        __syncthreads();
        // ---- loss and output layer (every warpgroup computes the row's
        // logit from the four partials in the same order) ----
        // L = -(w y log p + (1 - y) log(1 - p)), dL/dz = p (1 + (w - 1) y) - w y
        const float z5 = b5 + ((z5p[r] + z5p[128 + r]) + (z5p[256 + r] + z5p[384 + r]));
        const float pr = 1.0f / (1.0f + expf(-z5));
        const float wy = net.pos_w * y;
        const float dz5 = valid ? (pr * (wy + 1.0f - y) - wy) * inv_batch : 0.0f;
        if (q == 3) {  // the warpgroup with no encoding and no dW1 work
            float lv = valid ? (wy * (fmaxf(-z5, 0.0f) + log1pf(expf(-fabsf(z5)))) +
                                (1.0f - y) * (fmaxf(z5, 0.0f) + log1pf(expf(-fabsf(z5))))) * inv_batch
                             : 0.0f;
            float db5 = dz5;
            for (int off = 16; off > 0; off >>= 1) {
                lv += __shfl_xor_sync(FULL, lv, off);
                db5 += __shfl_xor_sync(FULL, db5, off);
            }
            if (lane == 0) {  // read by the first backward epilogue (after a barrier)
                misc[8 + (warp & 3)] = lv;
                misc[12 + (warp & 3)] = db5;
            }
        }
        // dz4 = bf16(dz5 * w5 * [h4 > 0]) (rounded by the store); this
        // warp's 32 rows of dz5 * h4, summed per column, go to z5p in the
        // first backward epilogue (z5p is still being read here)
        float dw5w;
        {
            float g[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                g[k] = h4[k] > 0.0f ? dz5 * w5[c0 + k] : 0.0f;
                h4[k] *= dz5;
            }
            store_chunk(dz, r, c0, g);
            dw5w = transpose_reduce32(h4, lane);
        }
        // ---- backward through layers 4, 3, 2: dz_{l+1} (dz or h_{l+1}'s
        // buffer) and W_{l+1} (B1, B0, B1) ----
#pragma unroll
        for (int l = 3; l >= 1; --l) {
            sync_mma();
            if (t == 0) {
                tc_fence_after();
                const int b = l == 2 ? 0 : 1;
                need_w(b);
                if (wok) {
                    const uint32_t s_dzl = l == 3 ? s_dz : s_h(l);
                    // dW_{l+1} += dz^T x_l : A = dz (MN-major), B = h_l (MN-major), K = samples
                    issue_mma(tm_dw(l - 1), s_dzl, 2048, 128, 4096, s_h(l - 1), 2048, 128, 4096, id_dw, 128,
                              !first);
                    // dX_l = dz W_{l+1} : A = dz (K-major), B = W (MN-major), K = units
                    issue_mma(tm_work, s_dzl, 128, 2048, 256, s_wb(b), 2048, 128, 4096, id_dx, 128, false);
                }
                tc_commit(bar);
            }
            wait_mma();
            if (t == 0) {
                if (l == 3) load_w(1, IMG_W2, 32768);                     // W4 read: B1 takes W2
                if (l == 2 && tile + 1 < t1) load_w(0, IMG_W1, 20480);    // W3 read: B0 takes W1
            }
            // sums over the tile's rows in a fixed order (no atomics): the
            // per-warp dw5 sums are stored after one barrier; warpgroup 3
            // adds them (and the loss and db5 sums) in the dW1 phase
            if (l == 3) z5p[128 * (warp & 3) + c0 + lane] = dw5w;
            // dz_l = bf16(dX_l) * [h_l > 0] on bf16 pairs, written over h_l
            uint8_t *hl = hb(l - 1);
            float v[32];
            uint32_t hp[16];
            tmem_ld32(tm_work + lane_off + c0, v);
            load_chunk_raw(hl, r, c0, hp);
#pragma unroll
            for (int k = 0; k < 16; ++k) hp[k] = pack_bf16(v[2 * k], v[2 * k + 1]) & bf16x2_pos_mask(hp[k]);
            store_chunk_raw(hl, r, c0, hp);
        }
        // ---- dW1 = dz1^T x0 (per tile, added to this CTA's partial) and the
        // bias gradients: x0's column 78 is all ones, so column 78 of dW1 is
        // db1 = sum over samples of dz1, and dz_l^T times x0's columns 64..79
        // gives db_l in its column 14 (db4, db3, db2 in work columns 94,
        // 110, 126) ----
        sync_mma();
        if (t == 0) {
            tc_fence_after();
            issue_mma(tm_work, s_h(0), 2048, 128, 4096, s_x0, 1280, 128, 2560, id_dw1, 128, false);
            issue_mma(tm_work + 80, s_dz, 2048, 128, 4096, s_x0 + 1024, 1280, 128, 2560, id_db, 128, false);
            issue_mma(tm_work + 96, s_h(2), 2048, 128, 4096, s_x0 + 1024, 1280, 128, 2560, id_db, 128, false);
            issue_mma(tm_work + 112, s_h(1), 2048, 128, 4096, s_x0 + 1024, 1280, 128, 2560, id_db, 128, false);
            tc_commit(bar);
        }
        wait_mma();
        // fire-and-forget vector adds (stores for the first tile): each
        // address of this CTA's partial is only ever written by this thread,
        // in tile order, so the sums are deterministic; warpgroup 3 has no
        // dW1 columns
        if (q < 2) {
            float *row = part + OFF_W1 + (int64_t)r * IN + c0;
            float v[32];
            tmem_ld32(tm_work + lane_off + c0, v);
#pragma unroll
            for (int k = 0; k < 8; ++k) add_v4(row + 4 * k, v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3], first);
        } else if (q == 2) {
            // columns 64..95: dW1 64..79 (78: db1), then db4's product (94)
            float *row = part + OFF_W1 + (int64_t)r * IN + c0;
            float v[32];
            tmem_ld32(tm_work + lane_off + c0, v);
            dbias[r] += v[14];
            dbias[384 + r] += v[30];
            v[14] = 0.0f;  // the pad weight's gradient
#pragma unroll
            for (int k = 0; k < 4; ++k) add_v4(row + 4 * k, v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3], first);
        } else {
            // columns 96..127: db3's and db2's products (110, 126)
            float v[32];
            tmem_ld32(tm_work + lane_off + c0, v);
            dbias[256 + r] += v[14];
            dbias[128 + r] += v[30];
            dw5[r] += (z5p[r] + z5p[128 + r]) + (z5p[256 + r] + z5p[384 + r]);
            if (r == 0) {
                misc[1] += (misc[8] + misc[9]) + (misc[10] + misc[11]);
                misc[0] += (misc[12] + misc[13]) + (misc[14] + misc[15]);
            }
            if (ahead) draw_ray(sb ^ 1);  // the next tile's rays, read after its first barrier
        }
        tc_fence_before();
        // the end-of-tile barrier doubles as the vote
        if (!__syncthreads_and(ok ? 1 : 0)) {
            ok = false;
            if (t == 0) {
                tc_commit(bar + 3);  // completes when all MMAs issued so far have
                rt_set_error(status, RT_ERR_TIMEOUT);
            }
            mbar_wait(bar + 3, 0, WAIT_CYCLES);
        }
    }
    // the partial reduction may be launched now; it waits for this grid
    // to complete before it reads the partials
    grid_dependents_launch();
    // weight copies still in flight (only after a give-up): let them land
    if (t == 0) {
#pragma unroll
        for (int b = 0; b < 2; ++b)
            if ((pend >> b) & 1u) mbar_wait(wbar + b, (wph >> b) & 1u, WAIT_CYCLES);
    }
    // ---- flush this CTA's partial gradient ----
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // the next step's first tile for the next launch
    if (S.pf_make && q == 3) {
        const float *o = smp + (int)((t1 - t0) & 1) * 7 * 128 + r;
        float *pf = S.pf + (int64_t)blockIdx.x * 7 * 128 + r;
#pragma unroll
        for (int j = 0; j < 7; ++j) pf[128 * j] = o[128 * j];
    }
    const bool any = ok;
    // dW2..dW4: TMEM -> shared memory rows (every activation and weight
    // buffer is dead now; rows padded to TR_ROWB bytes so that each 16-byte
    // store of a warp hits 8 distinct bank groups) -> one bulk copy per row
    // into the partial (stores straight from the row-per-thread registers
    // would write 16 bytes per 512-byte row stride across a warp)
    uint8_t *stage = smem;  // [3][128] rows
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        float4 *row = reinterpret_cast<float4 *>(stage + (l * 128 + r) * TR_ROWB + c0 * 4);
        float v[32];
        tmem_ld32(tm_dw(l) + lane_off + c0, v);
#pragma unroll
        for (int k = 0; k < 8; ++k)
            row[k] = any ? make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3])
                         : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    fence_async_smem();  // the rows, written by this proxy, are read by the bulk copies
    __syncthreads();
    if (q == 0) {
        const int offW[3] = {OFF_W2, OFF_W3, OFF_W4};
#pragma unroll
        for (int l = 0; l < 3; ++l) bulk_s2g(part + offW[l] + r * H, stage + (l * 128 + r) * TR_ROWB, H * 4);
        bulk_commit_wait();
    }
    if (t < 128) {
        part[OFF_B1 + t] = any ? dbias[t] : 0.0f;
        part[OFF_B2 + t] = any ? dbias[128 + t] : 0.0f;
        part[OFF_B3 + t] = any ? dbias[256 + t] : 0.0f;
        part[OFF_B4 + t] = any ? dbias[384 + t] : 0.0f;
        part[OFF_W5 + t] = any ? dw5[t] : 0.0f;
    }
    if (t == 0) {
        part[OFF_B5] = any ? misc[0] : 0.0f;
        part[NPARAM] = any ? misc[1] : 0.0f;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// Sum the CTA partials in a fixed order; either write the gradient or take
// an Adam step on the f32 master weights and re-pack the bf16 images.  A
// block of RA_GROUPS warps takes 32 consecutive parameters: warp w sums
// partials w, w + RA_GROUPS, ... (its loads all in flight), then warp 0 adds
// the RA_GROUPS sums in order.
constexpr int RA_GROUPS = 8;
__global__ void __launch_bounds__(32 * RA_GROUPS) k_mlp_reduce_adam(
    const float *partial, int nparts, float *grad_out, float *loss_out, float *params, float *mo, float *vo,
    uint8_t *img, float lr, float b1, float b2, float eps, float c1, float c2, int adam) {
    __shared__ float sums[RA_GROUPS][32];
    // the partials are complete; only then may the next training launch
    // start its set-up (which reads the sample buffer the training launch
    // before this one wrote)
    grid_dependency_wait();
    grid_dependents_launch();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int q = blockIdx.x * 32 + lane;
    float g = 0.0f;
    if (q <= NPARAM) {
        // the first RA_BATCH partials of this warp loaded before any is
        // added, so they are all in flight at once
        constexpr int RA_BATCH = 19;
        float x[RA_BATCH];
#pragma unroll
        for (int i = 0; i < RA_BATCH; ++i) {
            const int c = w + RA_GROUPS * i;
            x[i] = c < nparts ? __ldcg(partial + (int64_t)c * TR_PSTRIDE + q) : 0.0f;
        }
#pragma unroll
        for (int i = 0; i < RA_BATCH; ++i) g += x[i];
        for (int c = w + RA_GROUPS * RA_BATCH; c < nparts; c += RA_GROUPS)
            g += __ldcg(partial + (int64_t)c * TR_PSTRIDE + q);
    }
    sums[w][lane] = g;
    __syncthreads();
    if (w != 0 || q > NPARAM) return;
    g = sums[0][lane];
#pragma unroll
    for (int k = 1; k < RA_GROUPS; ++k) g += sums[k][lane];
    if (q == NPARAM) {
        if (loss_out) *loss_out = g;
        return;
    }
    if (!adam) {
        grad_out[q] = g;
        return;
    }
    const float m = b1 * mo[q] + (1.0f - b1) * g;
    const float v = b2 * vo[q] + (1.0f - b2) * g * g;
    mo[q] = m;
    vo[q] = v;
    const float wq = params[q] - lr * (m / c1) / (sqrtf(v / c2) + eps);
    params[q] = wq;
    // re-pack the bf16 image of weight matrices
    int base = -1, kin = 0, ioff = 0;
    if (q < OFF_B1) { base = OFF_W1; kin = IN; ioff = IMG_W1; }
    else if (q >= OFF_W2 && q < OFF_B2) { base = OFF_W2; kin = H; ioff = IMG_W2; }
    else if (q >= OFF_W3 && q < OFF_B3) { base = OFF_W3; kin = H; ioff = IMG_W3; }
    else if (q >= OFF_W4 && q < OFF_B4) { base = OFF_W4; kin = H; ioff = IMG_W4; }
    if (base >= 0) {
        const int e = q - base, r = e / kin, c = e % kin;
        *reinterpret_cast<__nv_bfloat16 *>(img + ioff + img_off(r, c, kin)) =
            __float2bfloat16_rn(base == OFF_W1 && c >= IN_FEAT ? 0.0f : wq);
    }
}
constexpr int RA_BLOCKS = (NPARAM + 1 + 31) / 32;

__global__ void k_mlp_pack(const float *params, uint8_t *img) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < OFF_B4; q += gridDim.x * blockDim.x) {
        int base = -1, kin = 0, ioff = 0;
        if (q < OFF_B1) { base = OFF_W1; kin = IN; ioff = IMG_W1; }
        else if (q >= OFF_W2 && q < OFF_B2) { base = OFF_W2; kin = H; ioff = IMG_W2; }
        else if (q >= OFF_W3 && q < OFF_B3) { base = OFF_W3; kin = H; ioff = IMG_W3; }
        else if (q >= OFF_W4 && q < OFF_B4) { base = OFF_W4; kin = H; ioff = IMG_W4; }
        if (base >= 0) {
            const int e = q - base, r = e / kin, c = e % kin;
            *reinterpret_cast<__nv_bfloat16 *>(img + ioff + img_off(r, c, kin)) =
                __float2bfloat16_rn(base == OFF_W1 && c >= IN_FEAT ? 0.0f : params[q]);
        }
    }
}

// He-uniform weights from Philox4x64-10 (counter (q,0,0,0), key (seed, 2)),
// zero biases; output layer uniform in +-sqrt(1/128).
__global__ void k_mlp_init(float *params, uint64_t seed) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < NPARAM; q += gridDim.x * blockDim.x) {
        uint64_t c[4] = {(uint64_t)q, 0ull, 0ull, 0ull};
        philox4x64_10(c, seed, 2ull);
        const float u = (float)(c[0] >> 40) * (1.0f / 16777216.0f) * 2.0f - 1.0f;
        float w = 0.0f;
        if (q < OFF_B1) w = u * sqrtf(6.0f / IN);
        else if ((q >= OFF_W2 && q < OFF_B2) || (q >= OFF_W3 && q < OFF_B3) || (q >= OFF_W4 && q < OFF_B4))
            w = u * sqrtf(6.0f / H);
        else if (q >= OFF_W5 && q < OFF_B5) w = u * sqrtf(1.0f / H);
        params[q] = w;
    }
}

__global__ void k_fill(float *p, int64_t n, float v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

}  // namespace

struct rt_surrogate {
    rt_mlp_cfg cfg;
    int64_t step;
    float lo[3], hi[3];
    void *block;
    float *params, *adam_m, *adam_v;
    uint8_t *img;
    float *partial;  // [nparts][TR_PSTRIDE]
    int nparts;
    float *scratch;   // [NPARAM+1] misc device scratch
    float *prefetch;  // [nparts][7][128]: the next training step's first tile per CTA
};

namespace {

std::atomic<long long> g_wait_cycles{WAIT_CYCLES};

MlpDev mlp_dev(const rt_surrogate *s) {
    MlpDev n;
    n.params = s->params;
    n.img = s->img;
    n.pos_w = s->cfg.pos_weight;
    n.wait_cycles = g_wait_cycles.load();
    for (int c = 0; c < 3; ++c) {
        // exact split of hi - lo (host float arithmetic is IEEE round-to-nearest)
        const volatile float hi = s->hi[c], lo = s->lo[c];
        const float sh = hi - lo;
        const float bb = sh - hi;
        n.lo[c] = lo;
        n.eh[c] = sh;
        n.el[c] = (hi - (sh - bb)) - (lo + bb);
    }
    return n;
}

bool g_attr_done = false;
rt_status set_smem_attrs() {
    if (g_attr_done) return RT_OK;
    if (cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, INF_SMEM_TOTAL) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, TR_SMEM_TOTAL) !=
            cudaSuccess) {
        cudaGetLastError();
        return RT_ERR_CUDA;
    }
    g_attr_done = true;
    return RT_OK;
}

// CTAs of a training launch over m samples, and how many of them have tiles
// (and so write a partial): the first ceil(ntiles / per), per = ceil(ntiles / grid)
int train_grid(const rt_surrogate *s, int64_t m) {
    const int64_t ntiles = (m + 127) / 128;
    const int grid = (int)(ntiles < s->nparts ? ntiles : s->nparts);
    return grid < 1 ? 1 : grid;
}
int train_parts(const rt_surrogate *s, int64_t m) {
    const int64_t ntiles = (m + 127) / 128, per = (ntiles + train_grid(s, m) - 1) / train_grid(s, m);
    return (int)((ntiles + per - 1) / per);
}

// Launch with programmatic stream serialisation: the kernel may start while
// the previous one in the stream finishes; it orders its own reads and
// writes against that kernel with griddepcontrol.wait.
template <typename... P, typename... A>
rt_status launch_dependent(void (*kernel)(P...), int grid, int block, size_t smem, cudaStream_t st, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, kernel, static_cast<P>(args)...) != cudaSuccess) {
        cudaGetLastError();
        return RT_ERR_CUDA;
    }
    return RT_OK;
}

// `dependent`: launched with programmatic stream serialisation (the training
// loop, where the launch before it is the partial reduction)
rt_status train_launch(const rt_surrogate *s, const SampleSrc &S, int64_t m, float inv_batch, cudaStream_t st,
                       bool dependent = false) {
    RT_TRY(set_smem_attrs());
    const int grid = train_grid(s, m);
    if (dependent)
        return launch_dependent(k_mlp_train, grid, TR_THREADS, TR_SMEM_TOTAL, st, mlp_dev(s), S, m, inv_batch,
                                s->partial, rt_status_ptr());
    k_mlp_train<<<grid, TR_THREADS, TR_SMEM_TOTAL, st>>>(mlp_dev(s), S, m, inv_batch, s->partial,
                                                         rt_status_ptr());
    RT_TRY(rt_check_launch());
    return RT_OK;
}

}  // namespace

extern "C" void rt_mlp_cfg_default(rt_mlp_cfg *c) {
    if (!c) return;
    c->lr = 1e-3f;
    c->beta1 = 0.9f;
    c->beta2 = 0.999f;
    c->eps = 1e-8f;
    c->batch = 262144;
    c->pos_weight = 1.0f;
}

extern "C" rt_status rt_set_wait_limit(int64_t max_cycles) {
    if (max_cycles < 0 || max_cycles > WAIT_CYCLES) return RT_ERR_INVALID_ARG;
    g_wait_cycles.store(max_cycles == 0 ? WAIT_CYCLES : (long long)max_cycles);
    return RT_OK;
}

extern "C" int64_t rt_surrogate_param_count(void) { return NPARAM; }

extern "C" rt_status rt_surrogate_create(const rt_mlp_cfg *cfg, uint64_t seed, rt_stream_t stream,
                                         rt_surrogate **out) {
    if (!out) return RT_ERR_INVALID_ARG;
    *out = nullptr;
    rt_mlp_cfg c;
    rt_mlp_cfg_default(&c);
    if (cfg) c = *cfg;
    if (!(c.lr > 0.f) || !(c.beta1 >= 0.f && c.beta1 < 1.f) || !(c.beta2 >= 0.f && c.beta2 < 1.f) ||
        !(c.eps > 0.f) || c.batch <= 0 || !(c.pos_weight > 0.f && c.pos_weight < 1e30f))
        return RT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    rt_surrogate *s = new rt_surrogate();
    s->cfg = c;
    s->step = 0;
    for (int k = 0; k < 3; ++k) {
        s->lo[k] = -1.f;
        s->hi[k] = 1.f;
    }
    s->nparts = rt_num_sms();
    const size_t pbytes = ((size_t)(NPARAM + 1) * 4 + 255) & ~(size_t)255;
    static_assert((((size_t)(NPARAM + 1) * 4 + 255) & ~(size_t)255) >= (size_t)TR_PSTRIDE * 4, "partial rows");
    const size_t total = 3 * pbytes + IMG_BYTES + (size_t)s->nparts * pbytes + pbytes +
                         (size_t)s->nparts * 7 * 128 * sizeof(float);
    rt_status r = rt_alloc(&s->block, total, stream);
    if (r != RT_OK) {
        delete s;
        return r;
    }
    char *b = (char *)s->block;
    s->params = (float *)b;
    s->adam_m = (float *)(b + pbytes);
    s->adam_v = (float *)(b + 2 * pbytes);
    s->img = (uint8_t *)(b + 3 * pbytes);
    s->partial = (float *)(b + 3 * pbytes + IMG_BYTES);
    s->scratch = (float *)(b + 3 * pbytes + IMG_BYTES + (size_t)s->nparts * pbytes);
    s->prefetch = (float *)(b + 3 * pbytes + IMG_BYTES + (size_t)s->nparts * pbytes + pbytes);
    // partial rows are TR_PSTRIDE floats apart (pbytes >= 4 * TR_PSTRIDE)
    k_mlp_init<<<64, 256, 0, st>>>(s->params, seed);
    k_fill<<<64, 256, 0, st>>>(s->adam_m, NPARAM, 0.f);
    k_fill<<<64, 256, 0, st>>>(s->adam_v, NPARAM, 0.f);
    k_mlp_pack<<<64, 256, 0, st>>>(s->params, s->img);
    if (rt_check_launch() != RT_OK || cudaStreamSynchronize(st) != cudaSuccess) {
        rt_free(s->block, stream);
        delete s;
        return RT_ERR_CUDA;
    }
    *out = s;
    return RT_OK;
}

extern "C" rt_status rt_surrogate_destroy(rt_surrogate *s, rt_stream_t stream) {
    if (!s) return RT_ERR_INVALID_ARG;
    rt_free(s->block, stream);
    delete s;
    return RT_OK;
}

extern "C" rt_status rt_surrogate_set_params(rt_surrogate *s, const float *params, rt_stream_t stream) {
    if (!s || !params) return RT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(s->params, params, NPARAM * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return RT_ERR_CUDA;
    k_fill<<<64, 256, 0, st>>>(s->adam_m, NPARAM, 0.f);
    k_fill<<<64, 256, 0, st>>>(s->adam_v, NPARAM, 0.f);
    k_mlp_pack<<<64, 256, 0, st>>>(s->params, s->img);
    s->step = 0;
    return rt_check_launch();
}

extern "C" rt_status rt_surrogate_get_params(const rt_surrogate *s, float *params, rt_stream_t stream) {
    if (!s || !params) return RT_ERR_INVALID_ARG;
    return cudaMemcpyAsync(params, s->params, NPARAM * 4, cudaMemcpyDeviceToDevice, (cudaStream_t)stream) ==
                   cudaSuccess
               ? RT_OK
               : RT_ERR_CUDA;
}

extern "C" rt_status rt_surrogate_get_state(const rt_surrogate *s, float *state, rt_stream_t stream) {
    if (!s || !state) return RT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    float stepf = (float)s->step;
    if (cudaMemcpyAsync(state, s->params, NPARAM * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(state + NPARAM, s->adam_m, NPARAM * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(state + 2 * NPARAM, s->adam_v, NPARAM * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(state + 3 * NPARAM, &stepf, 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return RT_ERR_CUDA;
    return RT_OK;
}

extern "C" rt_status rt_surrogate_set_state(rt_surrogate *s, const float *state, rt_stream_t stream) {
    if (!s || !state) return RT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    float stepf = 0.f;
    if (cudaMemcpyAsync(s->params, state, NPARAM * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(s->adam_m, state + NPARAM, NPARAM * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(s->adam_v, state + 2 * NPARAM, NPARAM * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(&stepf, state + 3 * NPARAM, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return RT_ERR_CUDA;
    if (!(stepf >= 0.f)) return RT_ERR_INVALID_ARG;
    s->step = (int64_t)stepf;
    k_mlp_pack<<<64, 256, 0, st>>>(s->params, s->img);
    return rt_check_launch();
}

extern "C" rt_status rt_surrogate_set_bounds(rt_surrogate *s, const float *lo, const float *hi) {
    if (!s || !lo || !hi) return RT_ERR_INVALID_ARG;
    for (int c = 0; c < 3; ++c) {
        if (!(hi[c] >= lo[c])) return RT_ERR_INVALID_ARG;
        s->lo[c] = lo[c];
        s->hi[c] = hi[c];
    }
    return RT_OK;
}

extern "C" rt_status rt_surrogate_forward(const rt_surrogate *s, const float *pos, const float *dir, int64_t m,
                                          float *p_out, rt_stream_t stream) {
    if (!s || m < 0) return RT_ERR_INVALID_ARG;
    if (m == 0) return RT_OK;
    if (!pos || !dir || !p_out) return RT_ERR_INVALID_ARG;
    RT_TRY(set_smem_attrs());
    SampleSrc S;
    memset(&S, 0, sizeof(S));
    S.mode = 0;
    S.pos = pos;
    S.dir = dir;
    int64_t ngroups = ((m + 127) / 128 + INF_WG - 1) / INF_WG;
    int grid = (int)(ngroups < rt_num_sms() ? ngroups : rt_num_sms());
    k_mlp_infer<<<grid, 128 * INF_WG, INF_SMEM_TOTAL, (cudaStream_t)stream>>>(mlp_dev(s), S, m, p_out, 0, 0.f,
                                                                              nullptr, nullptr, nullptr,
                                                                              rt_status_ptr());
    return rt_check_launch();
}

extern "C" rt_status rt_surrogate_loss_grad(const rt_surrogate *s, const float *pos, const float *dir,
                                            const float *y, int64_t m, float *grad_out, float *loss_out,
                                            rt_stream_t stream) {
    if (!s || m <= 0 || !pos || !dir || !y || !grad_out) return RT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    SampleSrc S;
    memset(&S, 0, sizeof(S));
    S.mode = 0;
    S.pos = pos;
    S.dir = dir;
    S.y = y;
    RT_TRY(train_launch(s, S, m, 1.0f / (float)m, st));
    const int nparts = train_parts(s, m);
    k_mlp_reduce_adam<<<RA_BLOCKS, 32 * RA_GROUPS, 0, st>>>(s->partial, nparts, grad_out, loss_out, nullptr,
                                                           nullptr, nullptr, nullptr, 0.f, 0.f, 0.f, 0.f, 1.f,
                                                           1.f, 0);
    return rt_check_launch();
}

extern "C" rt_status rt_surrogate_train(rt_surrogate *s, const rt_bvh *bvh, const rt_rayspec *samples,
                                        const float *T_target, int32_t steps, uint64_t seed, float *loss_curve,
                                        rt_stream_t stream) {
    if (!s || !bvh || !samples || !T_target || steps < 0) return RT_ERR_INVALID_ARG;
    if (samples->kind == RT_RAYS_EXPLICIT || samples->ray_ids) return RT_ERR_UNSUPPORTED;
    RaySetDev rs;
    int64_t R = 0;
    RT_TRY(rt_rayset_dev(bvh, samples, &rs, &R));
    if (R <= 0) return RT_ERR_INVALID_ARG;
    RT_TRY(rt_surrogate_set_bounds(s, bvh->lo, bvh->hi));
    cudaStream_t st = (cudaStream_t)stream;
    SampleSrc S;
    memset(&S, 0, sizeof(S));
    S.mode = 2;
    S.b = bvh_dev(bvh);
    S.rs = rs;
    S.T_target = T_target;
    S.seed = seed;
    S.R = R;
    const int64_t B = s->cfg.batch;
    const int nparts = train_parts(s, B);
    S.pf = s->prefetch;
    for (int32_t k = 0; k < steps; ++k) {
        S.step = s->step;
        S.pf_use = k > 0;             // drawn by the previous step's launch
        S.pf_make = k + 1 < steps;
        // the first launch follows whatever the stream ran before (no
        // early start); later ones may overlap the previous reduction
        RT_TRY(train_launch(s, S, B, 1.0f / (float)B, st, k > 0));
        s->step += 1;
        const double c1 = 1.0 - pow((double)s->cfg.beta1, (double)s->step);
        const double c2 = 1.0 - pow((double)s->cfg.beta2, (double)s->step);
        RT_TRY(launch_dependent(k_mlp_reduce_adam, RA_BLOCKS, 32 * RA_GROUPS, 0, st, s->partial, nparts,
                                (float *)nullptr, loss_curve ? loss_curve + k : (float *)nullptr, s->params,
                                s->adam_m, s->adam_v, s->img, s->cfg.lr, s->cfg.beta1, s->cfg.beta2,
                                s->cfg.eps, (float)c1, (float)c2, 1));
    }
    return RT_OK;
}

extern "C" rt_status rt_surrogate_infer(const rt_surrogate *s, const rt_bvh *bvh, const rt_rayspec *rays,
                                        float band, float *T_out, int64_t *n_fallback, rt_stream_t stream) {
    if (!s || !bvh || !rays || !(band >= 0.f && band <= 0.5f)) return RT_ERR_INVALID_ARG;
    if (rays->kind == RT_RAYS_EXPLICIT) return RT_ERR_UNSUPPORTED;
    RaySetDev rs;
    int64_t m = 0;
    RT_TRY(rt_rayset_dev(bvh, rays, &rs, &m));
    if (m == 0) {
        if (n_fallback && cudaMemsetAsync(n_fallback, 0, sizeof(int64_t), (cudaStream_t)stream) != cudaSuccess)
            return RT_ERR_CUDA;
        return RT_OK;
    }
    if (!T_out) return RT_ERR_INVALID_ARG;
    RT_TRY(set_smem_attrs());
    cudaStream_t st = (cudaStream_t)stream;
    SampleSrc S;
    memset(&S, 0, sizeof(S));
    S.mode = 1;
    S.b = bvh_dev(bvh);
    S.rs = rs;
    S.R = rs.n_rays;
    void *fb = nullptr;
    const bool use_fb = band > 0.f;
    int64_t *fb_rid = nullptr, *fb_pos = nullptr;
    unsigned long long *fb_count = nullptr, *work = nullptr;
    if (use_fb) {
        RT_TRY(rt_alloc(&fb, 16 * (size_t)m + 512, stream));
        fb_rid = (int64_t *)fb;
        fb_pos = fb_rid + m;
        fb_count = (unsigned long long *)(fb_pos + m);
        work = fb_count + 4;
        if (cudaMemsetAsync(fb_count, 0, 8, st) != cudaSuccess) {
            rt_free(fb, stream);
            return RT_ERR_CUDA;
        }
    }
    int64_t ngroups = ((m + 127) / 128 + INF_WG - 1) / INF_WG;
    int grid = (int)(ngroups < rt_num_sms() ? ngroups : rt_num_sms());
    k_mlp_infer<<<grid, 128 * INF_WG, INF_SMEM_TOTAL, st>>>(mlp_dev(s), S, m, T_out, 1, band, fb_rid, fb_pos,
                                                            fb_count, rt_status_ptr());
    rt_status r = rt_check_launch();
    if (r == RT_OK && use_fb) {
        r = rt_trace_launch_list(bvh, rays, fb_rid, fb_pos, fb_count, m, T_out, stream, work);
        if (r == RT_OK && n_fallback &&
            cudaMemcpyAsync(n_fallback, fb_count, 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            r = RT_ERR_CUDA;
    } else if (r == RT_OK && n_fallback) {
        if (cudaMemsetAsync(n_fallback, 0, 8, st) != cudaSuccess) r = RT_ERR_CUDA;
    }
    if (fb) rt_free(fb, stream);
    return r;
}

// ---------------------------------------------------------------------------
// Failure path of the bounded waits
// ---------------------------------------------------------------------------
namespace {
// One thread waits on an mbarrier that nothing ever completes, with the same
// bounded wait the surrogate kernels use; on giving up it records
// RT_ERR_TIMEOUT in the status word and returns.
__global__ void k_wait_selftest(long long max_cycles, int *status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        if (!mbar_wait(&bar, 0, max_cycles)) rt_set_error(status, RT_ERR_TIMEOUT);
    }
}
}  // namespace

extern "C" rt_status rt_selftest_wait_timeout(int64_t max_cycles, rt_stream_t stream) {
    if (max_cycles <= 0 || max_cycles > 4000000000LL) return RT_ERR_INVALID_ARG;
    k_wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>((long long)max_cycles, rt_status_ptr());
    return rt_check_launch();
}

// ---------------------------------------------------------------------------
// Inference without device allocation
// ---------------------------------------------------------------------------
// Some callers cannot let a library allocate device memory during a call:
// engines that reserve the whole device budget up front and forbid
// allocation inside their frame loop, and hosts whose device memory is owned
// by another runtime's allocator.  For them the fallback lists and counters of
// rt_surrogate_infer live in a fixed array that is part of the library image
// (reserved on every device that loads the library, until the process exits).
namespace {

constexpr int64_t kNoAllocMaxRays = 1 << 20;
// [0, M): fallback ray ids, [M, 2M): their output positions, then the fallback
// count and the trace work counter (M = kNoAllocMaxRays): 16 MiB + 256 B.
static __device__ __align__(256) int64_t g_noalloc_scratch[2 * kNoAllocMaxRays + 32];

std::mutex g_noalloc_mu;

// The array's device address is a property of the module loaded into a CUDA
// context.  A device reset destroys that context (and the module with it);
// the next context gets a new unique id (cuCtxGetId), so addresses are cached
// per context id and an address from a destroyed context is never reused.
typedef int (*ctx_get_current_fn)(void **);
typedef int (*ctx_get_id_fn)(void *, unsigned long long *);
ctx_get_current_fn g_ctx_current = nullptr;
ctx_get_id_fn g_ctx_id = nullptr;
bool g_ctx_fns_done = false;
constexpr int kNoAllocCache = 16;
unsigned long long g_noalloc_ctx[kNoAllocCache] = {0};
int64_t *g_noalloc_ptr[kNoAllocCache] = {nullptr};
int g_noalloc_next = 0;

// Unique id of the current CUDA context, 0 if none is current or the driver
// does not provide the calls (then nothing is cached).  Caller holds the lock.
unsigned long long current_ctx_id() {
    if (!g_ctx_fns_done) {
        g_ctx_fns_done = true;
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) ==
                cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            g_ctx_current = (ctx_get_current_fn)f1;
            g_ctx_id = (ctx_get_id_fn)f2;
        }
        cudaGetLastError();
    }
    if (!g_ctx_current || !g_ctx_id) return 0;
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_current(&ctx) != 0 || !ctx || g_ctx_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of the scratch array in the current context (the host-side
// symbol is only a stand-in, never a device address): looked up once per
// context with cudaGetSymbolAddress; a failed lookup is returned as an error
// and leaves nothing cached.
rt_status noalloc_scratch(int64_t **out) {
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    unsigned long long id = current_ctx_id();
    if (id != 0) {
        for (int k = 0; k < kNoAllocCache; ++k) {
            if (g_noalloc_ctx[k] == id && g_noalloc_ptr[k]) {
                *out = g_noalloc_ptr[k];
                return RT_OK;
            }
        }
    }
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return RT_ERR_CUDA;
    }
    if (id == 0) id = current_ctx_id();  // the lookup made the primary context current
    if (id != 0) {
        g_noalloc_ctx[g_noalloc_next] = id;
        g_noalloc_ptr[g_noalloc_next] = (int64_t *)p;
        g_noalloc_next = (g_noalloc_next + 1) % kNoAllocCache;
    }
    *out = (int64_t *)p;
    return RT_OK;
}

}  // namespace

extern "C" rt_status rt_surrogate_infer_noalloc(const rt_surrogate *s, const rt_bvh *bvh, const rt_rayspec *rays,
                                                float band, float *T_out, int64_t *n_fallback,
                                                rt_stream_t stream) {
    if (!s || !bvh || !rays || !(band >= 0.f && band <= 0.5f)) return RT_ERR_INVALID_ARG;
    if (rays->kind == RT_RAYS_EXPLICIT) return RT_ERR_UNSUPPORTED;
    RaySetDev rs;
    int64_t m = 0;
    RT_TRY(rt_rayset_dev(bvh, rays, &rs, &m));
    if (m > kNoAllocMaxRays) return RT_ERR_INVALID_ARG;  // beyond the fixed scratch capacity
    if (m == 0) {
        if (n_fallback && cudaMemsetAsync(n_fallback, 0, sizeof(int64_t), (cudaStream_t)stream) != cudaSuccess)
            return RT_ERR_CUDA;
        return RT_OK;
    }
    if (!T_out) return RT_ERR_INVALID_ARG;
    int64_t *scratch = nullptr;
    RT_TRY(noalloc_scratch(&scratch));
    RT_TRY(set_smem_attrs());
    cudaStream_t st = (cudaStream_t)stream;
    int64_t *fb_rid = scratch;
    int64_t *fb_pos = scratch + kNoAllocMaxRays;
    unsigned long long *fb_count = (unsigned long long *)(scratch + 2 * kNoAllocMaxRays);
    unsigned long long *work = fb_count + 4;
    const bool use_fb = band > 0.f;
    // the array keeps the previous call's contents: the count must start at 0
    if (use_fb && cudaMemsetAsync(fb_count, 0, sizeof(unsigned long long), st) != cudaSuccess) return RT_ERR_CUDA;
    SampleSrc S;
    memset(&S, 0, sizeof(S));
    S.mode = 1;
    S.b = bvh_dev(bvh);
    S.rs = rs;
    S.R = rs.n_rays;
    int64_t ngroups = ((m + 127) / 128 + INF_WG - 1) / INF_WG;
    int grid = (int)(ngroups < rt_num_sms() ? ngroups : rt_num_sms());
    k_mlp_infer<<<grid, 128 * INF_WG, INF_SMEM_TOTAL, st>>>(mlp_dev(s), S, m, T_out, 1, band, use_fb ? fb_rid : nullptr,
                                                   use_fb ? fb_pos : nullptr, use_fb ? fb_count : nullptr,
                                                   rt_status_ptr());
    RT_TRY(rt_check_launch());
    if (use_fb) {
        RT_TRY(rt_trace_launch_list(bvh, rays, fb_rid, fb_pos, fb_count, m, T_out, stream, work));
        if (n_fallback && cudaMemcpyAsync(n_fallback, fb_count, 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return RT_ERR_CUDA;
    } else if (n_fallback && cudaMemsetAsync(n_fallback, 0, 8, st) != cudaSuccess) {
        return RT_ERR_CUDA;
    }
    return RT_OK;
}
