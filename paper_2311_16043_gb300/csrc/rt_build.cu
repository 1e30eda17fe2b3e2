// rt_build.cu -- LBVH construction on the device (Sec. 4.1: a binary radix
// tree over the Gaussians in the manner of Karras 2012, leaves = tight boxes
// of single Gaussians, internal nodes = union of their children).
//
// Steps (all kernels below, one stream):
//   k_bounds       per-axis min/max of the means (order-preserving uint atomics)
//   k_morton       30-bit Morton codes, float32 IEEE quantisation (no FMA)
//   k_radix_*      stable LSD radix sort of (code, index), 8-bit digits, 4 passes
//   k_perm         permutation, inverse permutation, 64-bit keys code<<32|index
//   k_prep         per-Gaussian record (mean, opacity, whitening W = S^-1 R^T)
//                  and its leaf box, written in sorted order
//   k_karras       internal-node children by the longest-common-prefix split
//   k_refit        bottom-up child boxes; the second thread to reach a node
//                  (atomic arrival count) forms its box and climbs on
#include <math.h>
#include <stdio.h>

#include "rt_internal.cuh"

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 keys per block
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;

__device__ __forceinline__ uint32_t f2ord(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// Input check: every value finite, scales > 0, a non-zero quaternion and
// opacity in [0, 1]; *bad becomes non-zero otherwise.
__global__ void k_validate(const float *__restrict__ mean, const float *__restrict__ scale,
                           const float *__restrict__ quat, const float *__restrict__ opacity, int64_t n,
                           unsigned *bad) {
    bool ok = true;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float qn = 0.0f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float m = mean[3 * i + c], sc = scale[3 * i + c];
            ok = ok && isfinite(m) && isfinite(sc) && sc > 0.0f;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float q = quat[4 * i + c];
            ok = ok && isfinite(q);
            qn += q * q;
        }
        const float o = opacity[i];
        ok = ok && qn > 0.0f && o >= 0.0f && o <= 1.0f;
    }
    if (!ok) atomicOr(bad, 1u);
}

// Records a failed input check in the status word (asynchronous callers).
__global__ void k_report_invalid(const unsigned *bad, int *status) {
    if (*bad) rt_set_error(status, RT_ERR_INVALID_ARG);
}

// bounds_u[0..2] = ordered min, [3..5] = ordered max (pre-set to 0xff.. / 0)
__global__ void k_bounds(const float *__restrict__ mean, int64_t n, uint32_t *bounds_u) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float v = mean[3 * i + c];
            lo[c] = fminf(lo[c], v);
            hi[c] = fmaxf(hi[c], v);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        for (int off = 16; off > 0; off >>= 1) {
            lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], off));
            hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], off));
        }
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            atomicMin(&bounds_u[c], f2ord(lo[c]));
            atomicMax(&bounds_u[3 + c], f2ord(hi[c]));
        }
    }
}

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// Quantisation with separately rounded float32 operations:
// u = (mu - lo) / (hi - lo), q = clamp(floor(u * 1024), 0, 1023); 0 if hi == lo.
__global__ void k_morton(const float *__restrict__ mean, int64_t n, const uint32_t *bounds_u,
                         float *bounds_out, uint32_t *codes, int32_t *vals) {
    float lo[3], ext[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        lo[c] = ord2f(bounds_u[c]);
        float hi = ord2f(bounds_u[3 + c]);
        ext[c] = __fsub_rn(hi, lo[c]);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            bounds_out[c] = lo[c];
            bounds_out[3 + c] = hi;
        }
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t q[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (ext[c] == 0.0f) {
                q[c] = 0;
                continue;
            }
            float u = __fdiv_rn(__fsub_rn(mean[3 * i + c], lo[c]), ext[c]);
            float v = __fmul_rn(u, 1024.0f);
            int qi = (int)floorf(v);
            qi = qi < 0 ? 0 : (qi > 1023 ? 1023 : qi);
            q[c] = (uint32_t)qi;
        }
        codes[i] = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
        vals[i] = (int32_t)i;
    }
}

// counts[d * nblk + b] = number of keys of tile b with digit d
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t *__restrict__ keys,
                                                             int64_t n, int shift, int nblk,
                                                             uint32_t *counts) {
    __shared__ uint32_t hist[kRadix];
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) hist[d] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
    for (int it = 0; it < kSortItems; ++it) {
        int64_t i = base + it * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&hist[(keys[i] >> shift) & (kRadix - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) counts[(int64_t)d * nblk + blockIdx.x] = hist[d];
}

// In-place exclusive scan of m counts, one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_radix_scan(uint32_t *counts, int64_t m) {
    __shared__ uint32_t part[1024];
    int t = threadIdx.x;
    int64_t chunk = (m + 1023) / 1024;
    int64_t b = t * chunk, e = b + chunk < m ? b + chunk : m;
    uint32_t s = 0;
    for (int64_t i = b; i < e; ++i) s += counts[i];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {  // Hillis-Steele inclusive
        uint32_t v = t >= off ? part[t - off] : 0u;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    uint32_t run = part[t] - s;  // exclusive prefix of this chunk
    for (int64_t i = b; i < e; ++i) {
        uint32_t c = counts[i];
        counts[i] = run;
        run += c;
    }
}

// The counts' exclusive scan in parallel: k_scan_sums totals each segment
// of kScanSeg counts, k_radix_scan scans the totals (one block), and
// k_scan_apply scans each segment from its total's prefix.  (One block
// scanning all kRadix * nblk counts took 6.8 ms a pass at 64M keys.)
constexpr int kScanThreads = 256, kScanItems = 16, kScanSeg = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_sum256(uint32_t v, uint32_t *ws) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    uint32_t t = 0;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; ++w) t += ws[w];
    return t;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(const uint32_t *__restrict__ counts, int64_t m,
                                                            uint32_t *sums) {
    __shared__ uint32_t ws[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanSeg;
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int64_t i = base + j * kScanThreads + threadIdx.x;
        if (i < m) s += counts[i];
    }
    s = block_sum256(s, ws);
    if (threadIdx.x == 0) sums[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(uint32_t *counts, int64_t m,
                                                             const uint32_t *__restrict__ offs) {
    __shared__ uint32_t ws[kScanThreads / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int64_t base = (int64_t)blockIdx.x * kScanSeg + (int64_t)t * kScanItems;  // this thread's run
    uint32_t v[kScanItems], s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = base + j < m ? counts[base + j] : 0u;
        s += v[j];
    }
    // exclusive prefix of s over the block (warp scan, then the warps' totals)
    uint32_t inc = s;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += u;
    }
    if (lane == 31) ws[w] = inc;
    __syncthreads();
    uint32_t run = offs[blockIdx.x] + inc - s;
    for (int ww = 0; ww < w; ++ww) run += ws[ww];
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < m) counts[base + j] = run;
        run += v[j];
    }
}

// Stable scatter: within a tile, keys are ranked in index order (round,
// warp, lane), so equal digits keep their relative order.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const uint32_t *__restrict__ keys_in, const int32_t *__restrict__ vals_in, int64_t n, int shift,
    int nblk, const uint32_t *__restrict__ offsets, uint32_t *keys_out, int32_t *vals_out) {
    constexpr int kWarps = kSortThreads / 32;
    __shared__ uint32_t goff[kRadix];
    __shared__ uint32_t wcnt[kWarps][kRadix];
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    for (int d = t; d < kRadix; d += kSortThreads) goff[d] = offsets[(int64_t)d * nblk + blockIdx.x];
    const uint32_t lt_mask = (1u << lane) - 1u;
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int it = 0; it < kSortItems; ++it) {
        for (int j = t; j < kWarps * kRadix; j += kSortThreads) (&wcnt[0][0])[j] = 0;
        __syncthreads();
        int64_t i = base + it * kSortThreads + t;
        bool valid = i < n;
        uint32_t key = valid ? keys_in[i] : 0u;
        int32_t val = valid ? vals_in[i] : 0;
        uint32_t d = valid ? ((key >> shift) & (kRadix - 1)) : 0xffffffffu;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t rank = __popc(peers & lt_mask);
        if (valid && rank == 0) wcnt[w][d] = __popc(peers);
        __syncthreads();
        for (int dd = t; dd < kRadix; dd += kSortThreads) {  // prefix over warps, per digit
            uint32_t run = goff[dd];
            for (int ww = 0; ww < kWarps; ++ww) {
                uint32_t c = wcnt[ww][dd];
                wcnt[ww][dd] = run;
                run += c;
            }
            goff[dd] = run;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = wcnt[w][d] + rank;
            keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
    }
}

__global__ void k_perm(const uint32_t *__restrict__ codes, const int32_t *__restrict__ vals,
                       int64_t n, int32_t *perm, int32_t *rank, uint64_t *keys) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        int32_t i = vals[p];
        perm[p] = i;
        rank[i] = (int32_t)p;
        keys[p] = ((uint64_t)codes[p] << 32) | (uint32_t)i;
    }
}

// Per-Gaussian record and leaf box in sorted order.
__global__ void k_prep(const float *__restrict__ mean, const float *__restrict__ scale,
                       const float *__restrict__ quat, const float *__restrict__ opacity,
                       const int32_t *__restrict__ perm, int64_t n, rt_params prm,
                       const uint32_t *bounds_u, float4 *gauss, float *leafbox) {
    // absolute box margin: 1e-6 of the scene's coordinate scale
    float L = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float lo = ord2f(bounds_u[c]), hi = ord2f(bounds_u[3 + c]);
        L = fmaxf(L, fmaxf(fabsf(lo), fmaxf(fabsf(hi), hi - lo)));
    }
    const float margin = 1e-6f * L;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        int32_t i = perm[p];
        float qw = quat[4 * i], qx = quat[4 * i + 1], qy = quat[4 * i + 2], qz = quat[4 * i + 3];
        float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
        qw /= qn; qx /= qn; qy /= qn; qz /= qn;
        float R[3][3];
        R[0][0] = 1.f - 2.f * (qy * qy + qz * qz); R[0][1] = 2.f * (qx * qy - qw * qz); R[0][2] = 2.f * (qx * qz + qw * qy);
        R[1][0] = 2.f * (qx * qy + qw * qz); R[1][1] = 1.f - 2.f * (qx * qx + qz * qz); R[1][2] = 2.f * (qy * qz - qw * qx);
        R[2][0] = 2.f * (qx * qz - qw * qy); R[2][1] = 2.f * (qy * qz + qw * qx); R[2][2] = 1.f - 2.f * (qx * qx + qy * qy);
        float s[3] = {scale[3 * i], scale[3 * i + 1], scale[3 * i + 2]};
        float mu[3] = {mean[3 * i], mean[3 * i + 1], mean[3 * i + 2]};
        float o = opacity[i];
        float W[3][3];  // row k = column k of R divided by s_k
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) W[k][c] = __fdiv_rn(R[c][k], s[k]);
        gauss[4 * p + 0] = make_float4(mu[0], mu[1], mu[2], o);
        gauss[4 * p + 1] = make_float4(W[0][0], W[0][1], W[0][2], __int_as_float(i));
        gauss[4 * p + 2] = make_float4(W[1][0], W[1][1], W[1][2], 0.f);
        gauss[4 * p + 3] = make_float4(W[2][0], W[2][1], W[2][2], 0.f);
        // support radius: k_sigma, or the opacity-aware radius (same accepted set)
        float K = prm.k_sigma;
        bool empty = false;
        if (prm.box_mode == 1) {
            if (o < prm.alpha_min) empty = true;
            else {
                float kk = 2.0f * logf(o / prm.alpha_min);
                kk = kk * (1.0f + 1e-4f) + 1e-6f;  // outward margin for logf rounding
                if (kk < K * K) K = sqrtf(kk);
            }
        }
        float *bx = leafbox + 6 * p;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            // half-extent along world axis c: K sqrt(sum_k (R_ck s_k)^2), widened by
            // 1e-4 relative plus a few ulps of |mu| so the float box contains the
            // exact support and the slab test never misses an accepted peak
            float a0 = R[c][0] * s[0], a1 = R[c][1] * s[1], a2 = R[c][2] * s[2];
            float h = K * sqrtf(a0 * a0 + a1 * a1 + a2 * a2);
            h = h * (1.0f + 1e-4f) + 4.0f * 1.1920929e-7f * fabsf(mu[c]) + margin + 1e-30f;
            bx[c] = empty ? __int_as_float(0x7fc00000) : __fsub_rd(mu[c], h);
            bx[3 + c] = empty ? __int_as_float(0x7fc00000) : __fadd_ru(mu[c], h);
        }
    }
}

__device__ __forceinline__ int lcp(const uint64_t *keys, int64_t n, int64_t i, int64_t j) {
    if (j < 0 || j >= n) return -1;
    return __clzll(keys[i] ^ keys[j]);
}

// Internal node i: direction d toward the longer common prefix, range end j
// by exponential + binary search, split gamma by binary search; children
// gamma and gamma+1 are leaves when they are the range's ends.
__global__ void k_karras(const uint64_t *__restrict__ keys, int64_t n, float4 *nodes, int32_t *parent) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n - 1;
         i += (int64_t)gridDim.x * blockDim.x) {
        int d = (lcp(keys, n, i, i + 1) - lcp(keys, n, i, i - 1)) >= 0 ? 1 : -1;
        int dmin = lcp(keys, n, i, i - d);
        int64_t lmax = 2;
        while (lcp(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
        int64_t l = 0;
        for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
            if (lcp(keys, n, i, i + (l + t) * d) > dmin) l += t;
        int64_t j = i + l * d;
        int dnode = lcp(keys, n, i, j);
        int64_t s = 0, t = l;
        for (;;) {
            t = (t + 1) >> 1;
            if (lcp(keys, n, i, i + (s + t) * d) > dnode) s += t;
            if (t == 1) break;
        }
        int64_t gamma = i + s * d + (d < 0 ? -1 : 0);
        int64_t first = i < j ? i : j, last = i < j ? j : i;
        uint32_t lref, rref;
        if (first == gamma) {
            lref = RT_LEAF_BIT | (uint32_t)gamma;
            parent[(n - 1) + gamma] = (int32_t)i;
        } else {
            lref = (uint32_t)gamma;
            parent[gamma] = (int32_t)i;
        }
        if (last == gamma + 1) {
            rref = RT_LEAF_BIT | (uint32_t)(gamma + 1);
            parent[(n - 1) + gamma + 1] = (int32_t)i;
        } else {
            rref = (uint32_t)(gamma + 1);
            parent[gamma + 1] = (int32_t)i;
        }
        nodes[4 * i + 3] = make_float4(__uint_as_float(lref), __uint_as_float(rref), 0.f, 0.f);
        if (i == 0) parent[0] = -1;
    }
}

__device__ __forceinline__ void store_child_box(float4 *nodes, int32_t node, bool right, const float b[6]) {
    float *nd = reinterpret_cast<float *>(nodes + 4 * (int64_t)node);
    if (!right) {
        __stcg(nd + 0, b[0]); __stcg(nd + 1, b[3]); __stcg(nd + 2, b[1]);
        __stcg(nd + 3, b[4]); __stcg(nd + 4, b[2]); __stcg(nd + 5, b[5]);
    } else {
        __stcg(nd + 6, b[0]); __stcg(nd + 7, b[3]); __stcg(nd + 8, b[1]);
        __stcg(nd + 9, b[4]); __stcg(nd + 10, b[2]); __stcg(nd + 11, b[5]);
    }
}

// One thread per leaf climbs toward the root.  At each internal node it
// stores its subtree's box into the node's child slot, fences, and bumps the
// node's arrival count: the first arrival stops, the second (which then sees
// both slots) forms the union and continues.  No thread ever waits.
__global__ void k_refit(const float *__restrict__ leafbox, const int32_t *__restrict__ parent,
                        int64_t n, float4 *nodes, uint32_t *arrivals) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        float b[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) b[c] = leafbox[6 * p + c];
        uint32_t child = RT_LEAF_BIT | (uint32_t)p;
        int32_t node = parent[(n - 1) + p];
        while (node >= 0) {
            float4 refs = __ldcg(nodes + 4 * (int64_t)node + 3);
            bool right = __float_as_uint(refs.x) != child;
            store_child_box(nodes, node, right, b);
            __threadfence();
            if (atomicAdd(&arrivals[node], 1u) == 0) break;
            __threadfence();
            const float *nd = reinterpret_cast<const float *>(nodes + 4 * (int64_t)node);
            float l[12];
#pragma unroll
            for (int c = 0; c < 12; ++c) l[c] = __ldcg(nd + c);
            // slots: (L.lo.x, L.hi.x, L.lo.y, L.hi.y, L.lo.z, L.hi.z, R.lo.x, ...)
            b[0] = fminf(l[0], l[6]);  b[3] = fmaxf(l[1], l[7]);
            b[1] = fminf(l[2], l[8]);  b[4] = fmaxf(l[3], l[9]);
            b[2] = fminf(l[4], l[10]); b[5] = fmaxf(l[5], l[11]);
            child = (uint32_t)node;
            node = parent[node];
        }
    }
}

// Surface area of a box stored (lo.x, hi.x, lo.y, hi.y, lo.z, hi.z); -1 for NaN.
__device__ __forceinline__ float box_area(const float b[6]) {
    const float dx = b[1] - b[0], dy = b[3] - b[2], dz = b[5] - b[4];
    const float a = dx * dy + dy * dz + dz * dx;
    return a == a ? a : -1.0f;
}

// One level of the collapse into a 4-wide tree.  Each frontier entry is a
// binary internal node that becomes wide node w: its children are expanded
// greedily (the internal child of largest surface area is replaced by its two
// children) until four; children that are still internal binary nodes become
// wide nodes of the next level.
__global__ void k_collapse4(const float4 *__restrict__ nodes, const int2 *__restrict__ front_in,
                            const unsigned *__restrict__ n_in, int2 *front_out, unsigned *n_out,
                            unsigned *n_wide, float4 *wide) {
    const unsigned cnt = *n_in;
    for (unsigned f = blockIdx.x * blockDim.x + threadIdx.x; f < cnt; f += gridDim.x * blockDim.x) {
        const int2 e = front_in[f];
        uint32_t ref[4];
        float box[4][6];
        int m = 0;
        auto add_children = [&](int32_t b) {
            const float4 a = nodes[4 * (int64_t)b], c = nodes[4 * (int64_t)b + 1], d = nodes[4 * (int64_t)b + 2],
                         r = nodes[4 * (int64_t)b + 3];
            ref[m] = __float_as_uint(r.x);
            box[m][0] = a.x; box[m][1] = a.y; box[m][2] = a.z; box[m][3] = a.w; box[m][4] = c.x; box[m][5] = c.y;
            ++m;
            ref[m] = __float_as_uint(r.y);
            box[m][0] = c.z; box[m][1] = c.w; box[m][2] = d.x; box[m][3] = d.y; box[m][4] = d.z; box[m][5] = d.w;
            ++m;
        };
        add_children(e.x);
        while (m < 4) {
            int best = -1;
            float best_a = -2.0f;
            for (int c = 0; c < m; ++c) {
                if (ref[c] & RT_LEAF_BIT) continue;
                const float a = box_area(box[c]);
                if (a > best_a) {
                    best_a = a;
                    best = c;
                }
            }
            if (best < 0) break;
            const int32_t b = (int32_t)ref[best];
            // move the last entry into the expanded slot, then append both children
            ref[best] = ref[m - 1];
#pragma unroll
            for (int k = 0; k < 6; ++k) box[best][k] = box[m - 1][k];
            --m;
            add_children(b);
        }
        float4 *w = wide + 8 * (int64_t)e.y;
        float v[6][4];
        uint32_t out_ref[4];
        for (int c = 0; c < 4; ++c) {
            if (c < m) {
#pragma unroll
                for (int k = 0; k < 6; ++k) v[k][c] = box[c][k];
                if (ref[c] & RT_LEAF_BIT) {
                    out_ref[c] = ref[c];
                } else {
                    const unsigned idx = atomicAdd(n_wide, 1u);
                    const unsigned slot = atomicAdd(n_out, 1u);
                    front_out[slot] = make_int2((int32_t)ref[c], (int32_t)idx);
                    out_ref[c] = idx;
                }
            } else {
#pragma unroll
                for (int k = 0; k < 6; ++k) v[k][c] = __int_as_float(0x7fc00000);
                out_ref[c] = RT_EMPTY;
            }
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) w[k] = make_float4(v[k][0], v[k][1], v[k][2], v[k][3]);
        w[6] = make_float4(__uint_as_float(out_ref[0]), __uint_as_float(out_ref[1]), __uint_as_float(out_ref[2]),
                           __uint_as_float(out_ref[3]));
        w[7] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Refit links of the 4-wide tree: where each leaf and each wide node sits in
// its wide parent (4*w + slot; the root has none).
__global__ void k_wide_links(const float4 *__restrict__ wide, int64_t n_wide, int32_t *leaf_slot,
                             int32_t *wide_parent) {
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < n_wide;
         w += (int64_t)gridDim.x * blockDim.x) {
        const float4 r = wide[8 * w + 6];
        const uint32_t ref[4] = {__float_as_uint(r.x), __float_as_uint(r.y), __float_as_uint(r.z),
                                 __float_as_uint(r.w)};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (ref[c] == RT_EMPTY) continue;
            if (ref[c] & RT_LEAF_BIT) leaf_slot[ref[c] & ~RT_LEAF_BIT] = (int32_t)(4 * w + c);
            else wide_parent[ref[c]] = (int32_t)(4 * w + c);
        }
        if (w == 0) wide_parent[0] = -1;
    }
}

// Bottom-up refit of the 4-wide tree with its slots kept: each leaf stores its
// box into its slot and bumps the node's arrival count; the arrival that
// completes the node's children forms the union and climbs to the node's own
// slot in its parent.  No thread waits (as k_refit).
__global__ void k_refit_wide(const float *__restrict__ leafbox, const int32_t *__restrict__ leaf_slot,
                             const int32_t *__restrict__ wide_parent, int64_t n, float4 *wide,
                             uint32_t *arrivals) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        float b[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) b[c] = leafbox[6 * p + c];  // lo xyz, hi xyz
        int32_t slot = leaf_slot[p];
        while (slot >= 0) {
            const int64_t w = slot >> 2;
            const int c = slot & 3;
            float *wf = reinterpret_cast<float *>(wide + 8 * w);
            // SoA rows: lo.x, hi.x, lo.y, hi.y, lo.z, hi.z
            __stcg(wf + 0 + c, b[0]); __stcg(wf + 4 + c, b[3]);
            __stcg(wf + 8 + c, b[1]); __stcg(wf + 12 + c, b[4]);
            __stcg(wf + 16 + c, b[2]); __stcg(wf + 20 + c, b[5]);
            __threadfence();
            const float4 r = __ldcg(wide + 8 * w + 6);
            const uint32_t ref[4] = {__float_as_uint(r.x), __float_as_uint(r.y), __float_as_uint(r.z),
                                     __float_as_uint(r.w)};
            uint32_t m = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) m += ref[k] != RT_EMPTY;
            if (atomicAdd(&arrivals[w], 1u) + 1u < m) break;
            __threadfence();
            float u[6] = {__int_as_float(0x7fc00000), __int_as_float(0x7fc00000), __int_as_float(0x7fc00000),
                          __int_as_float(0x7fc00000), __int_as_float(0x7fc00000), __int_as_float(0x7fc00000)};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (ref[k] == RT_EMPTY) continue;
                u[0] = fminf(u[0], __ldcg(wf + 0 + k)); u[3] = fmaxf(u[3], __ldcg(wf + 4 + k));
                u[1] = fminf(u[1], __ldcg(wf + 8 + k)); u[4] = fmaxf(u[4], __ldcg(wf + 12 + k));
                u[2] = fminf(u[2], __ldcg(wf + 16 + k)); u[5] = fmaxf(u[5], __ldcg(wf + 20 + k));
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) b[k] = u[k];
            slot = wide_parent[w];
        }
    }
}

__global__ void k_export_boxes(const float4 *__restrict__ nodes, int64_t m, float *boxes,
                               int32_t *left, int32_t *right) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        float4 a = nodes[4 * i], b = nodes[4 * i + 1], c = nodes[4 * i + 2], r = nodes[4 * i + 3];
        if (boxes) {
            float *o = boxes + 12 * i;
            o[0] = a.x; o[1] = a.z; o[2] = b.x; o[3] = a.y; o[4] = a.w; o[5] = b.y;
            o[6] = b.z; o[7] = c.x; o[8] = c.z; o[9] = b.w; o[10] = c.y; o[11] = c.w;
        }
        if (left) left[i] = (int32_t)__float_as_uint(r.x);
        if (right) right[i] = (int32_t)__float_as_uint(r.y);
    }
}

// In-place exclusive scan of the m radix counts; sums: scan_sums_len(m)
// scratch words.
int64_t scan_sums_len(int64_t m) { return (m + kScanSeg - 1) / kScanSeg; }
void scan_counts(uint32_t *counts, int64_t m, uint32_t *sums, cudaStream_t st) {
    const int64_t P = scan_sums_len(m);
    k_scan_sums<<<(unsigned)P, kScanThreads, 0, st>>>(counts, m, sums);
    k_radix_scan<<<1, 1024, 0, st>>>(sums, P);
    k_scan_apply<<<(unsigned)P, kScanThreads, 0, st>>>(counts, m, sums);
}

int grid_for(int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    int64_t cap = (int64_t)rt_num_sms() * 16;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

rt_status rt_sort_pairs_u32(uint32_t *keys, int32_t *vals, int64_t n, int bits, rt_stream_t stream) {
    if (n <= 1 || bits <= 0) return RT_OK;
    if (n > (int64_t(1) << 31)) return RT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int nblk = (int)((n + kSortTile - 1) / kSortTile);
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    const int64_t mc = (int64_t)kRadix * nblk;
    const size_t bk = up(size_t(n) * 4), bc = up(size_t(mc) * 4), bs = up(size_t(scan_sums_len(mc)) * 4);
    void *blk = nullptr;
    RT_TRY(rt_alloc(&blk, 2 * bk + bc + bs, stream));
    uint32_t *k0 = keys, *k1 = (uint32_t *)blk, *counts = (uint32_t *)((char *)blk + 2 * bk),
             *sums = (uint32_t *)((char *)blk + 2 * bk + bc);
    int32_t *v0 = vals, *v1 = (int32_t *)((char *)blk + bk);
    const int passes = bits >= 32 ? 4 : (bits + kRadixBits - 1) / kRadixBits;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = pass * kRadixBits;
        k_radix_hist<<<nblk, kSortThreads, 0, st>>>(k0, n, shift, nblk, counts);
        scan_counts(counts, mc, sums, st);
        k_radix_scatter<<<nblk, kSortThreads, 0, st>>>(k0, v0, n, shift, nblk, counts, k1, v1);
        uint32_t *tk = k0; k0 = k1; k1 = tk;
        int32_t *tv = v0; v0 = v1; v1 = tv;
    }
    rt_status r = rt_check_launch();
    if (r == RT_OK && k0 != keys &&
        (cudaMemcpyAsync(keys, k0, size_t(n) * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
         cudaMemcpyAsync(vals, v0, size_t(n) * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)) {
        cudaGetLastError();
        r = RT_ERR_CUDA;
    }
    rt_free(blk, stream);
    return r;
}

extern "C" rt_status rt_build_bvh(const float *mean, const float *scale, const float *quat,
                                  const float *opacity, int64_t n, const rt_params *params,
                                  rt_stream_t stream, rt_bvh **out) {
    if (!out) return RT_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 0 || n >= (int64_t)0x7fffffff) return RT_ERR_INVALID_ARG;
    if (n > 0 && (!mean || !scale || !quat || !opacity)) return RT_ERR_INVALID_ARG;
    rt_params prm;
    rt_params_default(&prm);
    if (params) prm = *params;
    if (!(prm.k_sigma > 0.f) || !(prm.alpha_min > 0.f && prm.alpha_min < 1.f) ||
        !(prm.t_min >= 0.f && prm.t_min < 1.f) || !(prm.origin_eps >= 0.f) ||
        (prm.box_mode != 0 && prm.box_mode != 1) || (prm.deterministic != 0 && prm.deterministic != 1))
        return RT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;

    rt_bvh *b = new rt_bvh();
    b->n = n;
    b->params = prm;
    const int64_t ni = n > 1 ? n - 1 : 0;
    size_t off_g = 0;
    size_t off_nd = off_g + align256(sizeof(float4) * 4 * (size_t)n);
    size_t off_perm = off_nd + align256(sizeof(float4) * 4 * (size_t)ni);
    size_t off_rank = off_perm + align256(sizeof(int32_t) * (size_t)n);
    size_t off_keys = off_rank + align256(sizeof(int32_t) * (size_t)n);
    size_t off_par = off_keys + align256(sizeof(uint64_t) * (size_t)n);
    size_t off_bnd = off_par + align256(sizeof(int32_t) * (size_t)(n > 0 ? 2 * n - 1 : 0));
    size_t off_wide = off_bnd + 256;
    size_t total = off_wide + align256(sizeof(float4) * 8 * (size_t)ni);
    rt_status s = rt_alloc(&b->block, total, stream);
    if (s != RT_OK) {
        delete b;
        return s;
    }
    char *base = (char *)b->block;
    b->bytes = (int64_t)total;
    b->gauss = (float4 *)(base + off_g);
    b->nodes = (float4 *)(base + off_nd);
    b->perm = (int32_t *)(base + off_perm);
    b->rank = (int32_t *)(base + off_rank);
    b->keys = (uint64_t *)(base + off_keys);
    b->parent = (int32_t *)(base + off_par);
    b->bounds = (float *)(base + off_bnd);
    b->wide = (float4 *)(base + off_wide);
    b->n_wide = 0;
    b->links = nullptr;
    b->leaf_slot = b->wide_parent = nullptr;
    b->wide_arrivals = nullptr;
    for (int c = 0; c < 3; ++c) b->lo[c] = b->hi[c] = 0.f;
    if (n == 0) {
        *out = b;
        return RT_OK;
    }

    // scratch: bounds(6 u32) | codes, vals x2 | counts | leafbox | arrivals
    const int nblk = (int)((n + kSortTile - 1) / kSortTile);
    size_t s_bu = 0;
    size_t s_k0 = s_bu + 256;
    size_t s_v0 = s_k0 + align256(4 * (size_t)n);
    size_t s_k1 = s_v0 + align256(4 * (size_t)n);
    size_t s_v1 = s_k1 + align256(4 * (size_t)n);
    size_t s_cnt = s_v1 + align256(4 * (size_t)n);
    size_t s_sums = s_cnt + align256(4 * (size_t)kRadix * nblk);
    size_t s_leaf = s_sums + align256(4 * (size_t)scan_sums_len((int64_t)kRadix * nblk));
    size_t s_arr = s_leaf + align256(24 * (size_t)n);
    size_t s_f0 = s_arr + align256(4 * (size_t)ni);
    size_t s_f1 = s_f0 + align256(8 * (size_t)(ni + 1));
    size_t s_cnt2 = s_f1 + align256(8 * (size_t)(ni + 1));
    size_t s_total = s_cnt2 + 512;  // 64 level counts + the wide-node count (+ pad)
    void *scratch = nullptr;
    s = rt_alloc(&scratch, s_total, stream);
    if (s != RT_OK) {
        rt_free(b->block, stream);
        delete b;
        return s;
    }
    char *sb = (char *)scratch;
    uint32_t *bounds_u = (uint32_t *)(sb + s_bu);
    uint32_t *k0 = (uint32_t *)(sb + s_k0), *k1 = (uint32_t *)(sb + s_k1);
    int32_t *v0 = (int32_t *)(sb + s_v0), *v1 = (int32_t *)(sb + s_v1);
    uint32_t *counts = (uint32_t *)(sb + s_cnt);
    uint32_t *sums = (uint32_t *)(sb + s_sums);
    float *leafbox = (float *)(sb + s_leaf);
    uint32_t *arrivals = (uint32_t *)(sb + s_arr);
    int2 *front[2] = {(int2 *)(sb + s_f0), (int2 *)(sb + s_f1)};
    unsigned *wcnt = (unsigned *)(sb + s_cnt2);  // [0..63] level counts, [64] wide-node count (512 B region)

    rt_status result = RT_OK;
    unsigned bad = 0;  // host copy of the input check (read with the bounds)
    do {
        if (cudaMemsetAsync(bounds_u, 0xff, 12, st) != cudaSuccess ||
            cudaMemsetAsync(bounds_u + 3, 0, 20, st) != cudaSuccess) {
            result = RT_ERR_CUDA;
            break;
        }
        k_validate<<<grid_for(n, 256), 256, 0, st>>>(mean, scale, quat, opacity, n, bounds_u + 7);
        k_bounds<<<grid_for(n, 256), 256, 0, st>>>(mean, n, bounds_u);
        k_morton<<<grid_for(n, 256), 256, 0, st>>>(mean, n, bounds_u, b->bounds, k0, v0);
        for (int pass = 0; pass < 4; ++pass) {
            int shift = pass * kRadixBits;
            k_radix_hist<<<nblk, kSortThreads, 0, st>>>(k0, n, shift, nblk, counts);
            scan_counts(counts, (int64_t)kRadix * nblk, sums, st);
            k_radix_scatter<<<nblk, kSortThreads, 0, st>>>(k0, v0, n, shift, nblk, counts, k1, v1);
            uint32_t *tk = k0; k0 = k1; k1 = tk;
            int32_t *tv = v0; v0 = v1; v1 = tv;
        }
        k_perm<<<grid_for(n, 256), 256, 0, st>>>(k0, v0, n, b->perm, b->rank, b->keys);
        k_prep<<<grid_for(n, 128), 128, 0, st>>>(mean, scale, quat, opacity, b->perm, n, prm, bounds_u,
                                                 b->gauss, leafbox);
        if (n == 1) {
            int32_t m1 = -1;
            if (cudaMemcpyAsync(b->parent, &m1, sizeof(int32_t), cudaMemcpyHostToDevice, st) != cudaSuccess)
                result = RT_ERR_CUDA;
        } else {
            k_karras<<<grid_for(ni, 256), 256, 0, st>>>(b->keys, n, b->nodes, b->parent);
            if (cudaMemsetAsync(arrivals, 0, 4 * (size_t)ni, st) != cudaSuccess) {
                result = RT_ERR_CUDA;
                break;
            }
            k_refit<<<grid_for(n, 256), 256, 0, st>>>(leafbox, b->parent, n, b->nodes, arrivals);
            // collapse into the 4-wide tree, one level per launch (the tree has at
            // most 64 levels; launches past the last level find an empty frontier)
            const int2 root = make_int2(0, 0);
            const unsigned one = 1u;
            if (cudaMemsetAsync(wcnt, 0, 512, st) != cudaSuccess ||
                cudaMemcpyAsync(front[0], &root, sizeof(int2), cudaMemcpyHostToDevice, st) != cudaSuccess ||
                cudaMemcpyAsync(wcnt, &one, sizeof(unsigned), cudaMemcpyHostToDevice, st) != cudaSuccess ||
                cudaMemcpyAsync(wcnt + 64, &one, sizeof(unsigned), cudaMemcpyHostToDevice, st) != cudaSuccess) {
                result = RT_ERR_CUDA;
                break;
            }
            int grid_c = grid_for(ni, 128);
            for (int lvl = 0; lvl < 63; ++lvl)
                k_collapse4<<<grid_c, 128, 0, st>>>(b->nodes, front[lvl & 1], wcnt + lvl, front[(lvl + 1) & 1],
                                                     wcnt + lvl + 1, wcnt + 64, b->wide);
            unsigned nw = 0, left_over = 0;
            if (cudaMemcpyAsync(&nw, wcnt + 64, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaMemcpyAsync(&left_over, wcnt + 63, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                result = RT_ERR_CUDA;
                break;
            }
            // a frontier left after the last level would mean an unfinished wide
            // tree (impossible for keys of <= 61 significant bits); then only
            // the binary tree is used
            b->n_wide = (left_over || nw > (unsigned)ni) ? 0 : nw;
        }
        if (rt_check_launch() != RT_OK) {
            result = RT_ERR_CUDA;
            break;
        }
        if (cudaMemcpyAsync(b->lo, b->bounds, 3 * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(b->hi, b->bounds + 3, 3 * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&bad, bounds_u + 7, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess) {
            result = RT_ERR_CUDA;
            break;
        }
    } while (0);
    if (result == RT_OK && cudaStreamSynchronize(st) != cudaSuccess) result = RT_ERR_CUDA;
    rt_free(scratch, stream);
    if (result == RT_OK && bad) result = RT_ERR_INVALID_ARG;
    if (result != RT_OK) {
        rt_free(b->block, stream);
        delete b;
        return result;
    }
    *out = b;
    return RT_OK;
}

extern "C" rt_status rt_bvh_refit(rt_bvh *b, const float *mean, const float *scale, const float *quat,
                                  const float *opacity, rt_stream_t stream) {
    if (!b) return RT_ERR_INVALID_ARG;
    const int64_t n = b->n;
    if (n == 0) return RT_OK;
    if (!mean || !scale || !quat || !opacity) return RT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t ni = n > 1 ? n - 1 : 0;
    if (b->n_wide > 0 && !b->links) {
        const size_t o_par = align256(4 * (size_t)n), o_arr = o_par + align256(4 * (size_t)b->n_wide);
        RT_TRY(rt_alloc(&b->links, o_arr + align256(4 * (size_t)b->n_wide), stream));
        b->leaf_slot = (int32_t *)b->links;
        b->wide_parent = (int32_t *)((char *)b->links + o_par);
        b->wide_arrivals = (uint32_t *)((char *)b->links + o_arr);
        // -1 everywhere first: a slot the links never set ends the climb
        rt_status r = RT_OK;
        if (cudaMemsetAsync(b->links, 0xff, o_arr, st) != cudaSuccess) r = RT_ERR_CUDA;
        if (r == RT_OK) {
            k_wide_links<<<grid_for(b->n_wide, 256), 256, 0, st>>>(b->wide, b->n_wide, b->leaf_slot,
                                                                    b->wide_parent);
            r = rt_check_launch();
        }
        if (r != RT_OK) {
            rt_free(b->links, stream);
            b->links = nullptr;
            return r;
        }
    }
    // scratch: bounds (6 u32) | leaf boxes | binary arrivals
    const size_t s_leaf = 256, s_arr = s_leaf + align256(24 * (size_t)n);
    void *scratch = nullptr;
    RT_TRY(rt_alloc(&scratch, s_arr + align256(4 * (size_t)ni) + 256, stream));
    char *sb = (char *)scratch;
    uint32_t *bounds_u = (uint32_t *)sb;
    float *leafbox = (float *)(sb + s_leaf);
    uint32_t *arrivals = (uint32_t *)(sb + s_arr);
    rt_status result = RT_OK;
    do {
        if (cudaMemsetAsync(bounds_u, 0xff, 12, st) != cudaSuccess ||
            cudaMemsetAsync(bounds_u + 3, 0, 20, st) != cudaSuccess) {
            result = RT_ERR_CUDA;
            break;
        }
        k_validate<<<grid_for(n, 256), 256, 0, st>>>(mean, scale, quat, opacity, n, bounds_u + 7);
        k_report_invalid<<<1, 1, 0, st>>>(bounds_u + 7, rt_status_ptr());
        k_bounds<<<grid_for(n, 256), 256, 0, st>>>(mean, n, bounds_u);
        k_prep<<<grid_for(n, 128), 128, 0, st>>>(mean, scale, quat, opacity, b->perm, n, b->params, bounds_u,
                                                 b->gauss, leafbox);
        if (n > 1) {
            if (cudaMemsetAsync(arrivals, 0, 4 * (size_t)ni, st) != cudaSuccess) {
                result = RT_ERR_CUDA;
                break;
            }
            k_refit<<<grid_for(n, 256), 256, 0, st>>>(leafbox, b->parent, n, b->nodes, arrivals);
        }
        if (b->n_wide > 0) {
            if (cudaMemsetAsync(b->wide_arrivals, 0, 4 * (size_t)b->n_wide, st) != cudaSuccess) {
                result = RT_ERR_CUDA;
                break;
            }
            k_refit_wide<<<grid_for(n, 256), 256, 0, st>>>(leafbox, b->leaf_slot, b->wide_parent, n, b->wide,
                                                           b->wide_arrivals);
        }
        result = rt_check_launch();
    } while (0);
    rt_free(scratch, stream);
    return result;
}

extern "C" rt_status rt_bvh_destroy(rt_bvh *bvh, rt_stream_t stream) {
    if (!bvh) return RT_ERR_INVALID_ARG;
    if (bvh->links) rt_free(bvh->links, stream);
    rt_free(bvh->block, stream);
    delete bvh;
    return RT_OK;
}

extern "C" rt_status rt_bvh_info(const rt_bvh *bvh, int64_t *n, float *lo, float *hi, int64_t *bytes) {
    if (!bvh) return RT_ERR_INVALID_ARG;
    if (n) *n = bvh->n;
    for (int c = 0; c < 3; ++c) {
        if (lo) lo[c] = bvh->lo[c];
        if (hi) hi[c] = bvh->hi[c];
    }
    if (bytes) *bytes = bvh->bytes;
    return RT_OK;
}

extern "C" rt_status rt_bvh_export(const rt_bvh *bvh, uint64_t *keys, int32_t *left, int32_t *right,
                                   int32_t *parent, float *boxes, rt_stream_t stream) {
    if (!bvh) return RT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int64_t n = bvh->n;
    if (n == 0) return RT_OK;
    if (keys && cudaMemcpyAsync(keys, bvh->keys, 8 * (size_t)n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return RT_ERR_CUDA;
    if (parent && cudaMemcpyAsync(parent, bvh->parent, 4 * (size_t)(2 * n - 1), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return RT_ERR_CUDA;
    if (n > 1 && (boxes || left || right)) {
        k_export_boxes<<<grid_for(n - 1, 256), 256, 0, st>>>(bvh->nodes, n - 1, boxes, left, right);
        return rt_check_launch();
    }
    return RT_OK;
}
