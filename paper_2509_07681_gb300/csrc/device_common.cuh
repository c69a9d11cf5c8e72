// Device building blocks of the FUnc-SNE iteration on sm_103a: the Philox
// generator, index mappings, (distance, index) keys, warp-wide bitonic
// networks, distance kernels for FP32 / BF16 / FP8 rows and the warp
// bisection of the bandwidth (Eq. 1).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_fp16.h>

#include "params.h"

namespace fsne {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint64_t kSentinel = ~0ull;  // larger than every valid (d2, idx) key

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw (SC'11): ten rounds of two 32x32->64-bit
// multiplies; the 64-bit key is bumped by the Weyl constants between rounds.
__device__ __forceinline__ void philox_round(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3, uint32_t k0,
                                             uint32_t k1) {
    const uint32_t ha = __umulhi(kPhiloxM0, c0), la = kPhiloxM0 * c0;
    const uint32_t hb = __umulhi(kPhiloxM1, c2), lb = kPhiloxM1 * c2;
    c0 = hb ^ c1 ^ k0;
    c1 = lb;
    c2 = ha ^ c3 ^ k1;
    c3 = la;
}
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t seed) {
    uint32_t k0 = static_cast<uint32_t>(seed);
    uint32_t k1 = static_cast<uint32_t>(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += kPhiloxW0;
            k1 += kPhiloxW1;
        }
        philox_round(c0, c1, c2, c3, k0, k1);
    }
    return make_uint4(c0, c1, c2, c3);
}
// The same block with the round keys precomputed (philox_keys).
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, const PhiloxKeys& K) {
#pragma unroll
    for (int r = 0; r < 10; ++r) philox_round(c0, c1, c2, c3, K.k0[r], K.k1[r]);
    return make_uint4(c0, c1, c2, c3);
}

// uniform integer in [0, m): high word of u * m.
__device__ __forceinline__ uint32_t map_index(uint32_t u, uint32_t m) { return __umulhi(u, m); }

// uniform index in [0, n) without i.
__device__ __forceinline__ uint32_t map_other(uint32_t u, uint32_t n, uint32_t i) {
    const uint32_t j = __umulhi(u, n - 1u);
    return j + (j >= i ? 1u : 0u);
}

// ---------------------------------------------------------------- keys
// (d2, idx) packed so that unsigned order equals the lexicographic order
// (d2 >= 0, so its IEEE bits are monotone).
__device__ __forceinline__ uint64_t make_key(float d2, uint32_t idx) {
    return (static_cast<uint64_t>(__float_as_uint(d2)) << 32) | idx;
}
__device__ __forceinline__ uint32_t key_idx(uint64_t k) { return static_cast<uint32_t>(k); }
__device__ __forceinline__ float key_d2(uint64_t k) {
    return __uint_as_float(static_cast<uint32_t>(k >> 32));
}

__device__ __forceinline__ uint64_t shfl64(uint64_t v, int src) {
    const uint32_t lo = __shfl_sync(kFull, static_cast<uint32_t>(v), src);
    const uint32_t hi = __shfl_sync(kFull, static_cast<uint32_t>(v >> 32), src);
    return (static_cast<uint64_t>(hi) << 32) | lo;
}
__device__ __forceinline__ uint64_t shfl_xor64(uint64_t v, int m) {
    const uint32_t lo = __shfl_xor_sync(kFull, static_cast<uint32_t>(v), m);
    const uint32_t hi = __shfl_xor_sync(kFull, static_cast<uint32_t>(v >> 32), m);
    return (static_cast<uint64_t>(hi) << 32) | lo;
}

// Element e of a warp-distributed array of 32*R values (lane e%32, register e/32).
template <int R, typename T>
__device__ __forceinline__ T warp_get(const T (&v)[R], uint32_t e) {
    T out = v[0];
    const int src = static_cast<int>(e & 31u);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const T x = __shfl_sync(kFull, v[r], src);
        if (static_cast<uint32_t>(r) == (e >> 5)) out = x;
    }
    return out;
}

template <int R>
__device__ __forceinline__ uint64_t warp_get64(const uint64_t (&v)[R], uint32_t e) {
    uint64_t out = v[0];
    const int src = static_cast<int>(e & 31u);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint64_t x = shfl64(v[r], src);
        if (static_cast<uint32_t>(r) == (e >> 5)) out = x;
    }
    return out;
}

// ---------------------------------------------------------------- bitonic networks
// Ascending sort of 32*R keys held as element e = r*32 + lane.
template <int R>
__device__ __forceinline__ void cmpx_stage(uint64_t (&k)[R], int lane, int size, int stride) {
    if (stride >= 32) {
        const int rs = stride >> 5;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if ((r & rs) == 0) {
                const int e = r * 32 + lane;
                const bool asc = (e & size) == 0;
                const uint64_t a = k[r], b = k[r | rs];
                // out of order for the stage's direction (equal keys may swap)
                const bool sw = (b < a) == asc;
                k[r] = sw ? b : a;
                k[r | rs] = sw ? a : b;
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = r * 32 + lane;
            const uint64_t o = shfl_xor64(k[r], stride);
            const bool asc = (e & size) == 0;
            const bool lower = (lane & stride) == 0;
            // keep the minimum (lower == asc) or the maximum of the pair:
            // take the partner's key when it is smaller or larger respectively
            // (one 64-bit compare, one select)
            const bool take = (o < k[r]) == (lower == asc);
            k[r] = take ? o : k[r];
        }
    }
}

template <int R>
__device__ __forceinline__ void warp_sort(uint64_t (&k)[R], int lane) {
#pragma unroll
    for (int size = 2; size <= 32 * R; size <<= 1)
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) cmpx_stage<R>(k, lane, size, stride);
}

// Sorts a bitonic sequence of 32*R keys ascending.
template <int R>
__device__ __forceinline__ void warp_bitonic_merge(uint64_t (&k)[R], int lane) {
#pragma unroll
    for (int stride = 16 * R; stride > 0; stride >>= 1) cmpx_stage<R>(k, lane, 32 * R, stride);
}

// Top 32*R of (sorted old list, 32 candidates): old[0..32R-33] always stay,
// the last 32 slots take the 32 smallest of (old tail, candidates).
template <int R>
__device__ __forceinline__ void merge_candidates(uint64_t (&old)[R], uint64_t cand, int lane) {
    uint64_t c[1] = {cand};
    warp_sort<1>(c, lane);
    const uint64_t crev = shfl64(c[0], 31 - lane);
    uint64_t b[1] = {old[R - 1] < crev ? old[R - 1] : crev};
    warp_bitonic_merge<1>(b, lane);
    if constexpr (R == 1) {
        old[0] = b[0];
    } else {
        uint64_t m[2] = {old[0], shfl64(b[0], 31 - lane)};
        warp_bitonic_merge<2>(m, lane);
        old[0] = m[0];
        old[1] = m[1];
    }
}

__device__ __forceinline__ uint64_t shfl_up64(uint64_t v, int d) {
    const uint32_t lo = __shfl_up_sync(kFull, static_cast<uint32_t>(v), d);
    const uint32_t hi = __shfl_up_sync(kFull, static_cast<uint32_t>(v >> 32), d);
    return (static_cast<uint64_t>(hi) << 32) | lo;
}

// Inserts the candidate keys that precede thr (one per lane) into a sorted
// warp list of 32*R keys, one at a time: each insertion finds its position by
// a ballot and shifts the tail up by one element. Afterwards the first k
// entries are the k smallest of (list, candidates) whenever thr is the
// list's k-th key. Cheap when few candidates qualify.
template <int R>
__device__ __forceinline__ void insert_candidates(uint64_t (&lst)[R], uint64_t cand, uint64_t thr, int lane) {
    unsigned m = __ballot_sync(kFull, cand < thr);
    while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const uint64_t c = shfl64(cand, src);
        int pos = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) pos += __popc(__ballot_sync(kFull, lst[r] < c));
        uint64_t prev[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint64_t up = shfl_up64(lst[r], 1);
            const uint64_t tail = r > 0 ? shfl64(lst[r > 0 ? r - 1 : 0], 31) : up;
            prev[r] = lane == 0 ? tail : up;
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = r * 32 + lane;
            lst[r] = e < pos ? lst[r] : (e == pos ? c : prev[r]);
        }
    }
}

// ---------------------------------------------------------------- packed FP32 pairs
// sm_100 and later execute two FP32 operations in one instruction (FFMA2,
// FMUL2); each half is rounded exactly as its scalar counterpart, so a pair
// costs one issue slot instead of two. A squared distance summed this way
// keeps two chains (even and odd components) and adds them at the end.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 bcast2(float s) { return make_float2(s, s); }
// x - y rounded once, as __fsub_rn(x, y): fma(y, -1, x).
__device__ __forceinline__ float2 sub2(float2 x, float2 y) { return __ffma2_rn(y, make_float2(-1.f, -1.f), x); }
__device__ __forceinline__ float hsum2(float2 a) { return __fadd_rn(a.x, a.y); }
// Squared distance between the float4 u and v in two chains:
// (d0^2 + d2^2) + (d1^2 + d3^2).
__device__ __forceinline__ float2 sqdiff2_f4(const float4 u, const float4 v, float2 acc) {
    const float2 d01 = sub2(make_float2(u.x, u.y), make_float2(v.x, v.y));
    const float2 d23 = sub2(make_float2(u.z, u.w), make_float2(v.z, v.w));
    acc = fma2(d01, d01, acc);
    return fma2(d23, d23, acc);
}
// The same two chains started from the first pair: (d0^2 + d2^2, d1^2 + d3^2).
__device__ __forceinline__ float2 sq2_f4(const float4 u, const float4 v) {
    const float2 d01 = sub2(make_float2(u.x, u.y), make_float2(v.x, v.y));
    const float2 d23 = sub2(make_float2(u.z, u.w), make_float2(v.z, v.w));
    return fma2(d23, d23, mul2(d01, d01));
}

// ---------------------------------------------------------------- warp reductions
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(kFull, v, m);
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(kFull, v, m);
    return v;
}

// Reduce-scatter of v[OFF .. OFF+32): afterwards lane l holds the warp sum
// of v[OFF + l] (31 shuffles).
template <int OFF = 0, int N>
__device__ __forceinline__ float warp_reduce_scatter32(float (&v)[N], int lane) {
    static_assert(OFF + 32 <= N, "reduce-scatter window out of range");
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const bool up = (lane & w) != 0;
#pragma unroll
        for (int k = 0; k < w; ++k) {
            const float send = up ? v[OFF + k] : v[OFF + k + w];
            const float keep = up ? v[OFF + k + w] : v[OFF + k];
            v[OFF + k] = keep + __shfl_xor_sync(kFull, send, w);
        }
    }
    return v[OFF];
}

// ---------------------------------------------------------------- rows
template <int DP>
__device__ __forceinline__ void load_row(const float* __restrict__ src, float (&v)[DP]) {
    if constexpr (DP % 4 == 0) {
        const float4* s = reinterpret_cast<const float4*>(src);
#pragma unroll
        for (int q = 0; q < DP / 4; ++q) {
            const float4 a = __ldg(s + q);
            v[4 * q] = a.x;
            v[4 * q + 1] = a.y;
            v[4 * q + 2] = a.z;
            v[4 * q + 3] = a.w;
        }
    } else {
        const float2* s = reinterpret_cast<const float2*>(src);
#pragma unroll
        for (int q = 0; q < DP / 2; ++q) {
            const float2 a = __ldg(s + q);
            v[2 * q] = a.x;
            v[2 * q + 1] = a.y;
        }
    }
}

template <int DP>
__device__ __forceinline__ float sqdist_ld(const float (&a)[DP], const float (&b)[DP]) {
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < DP; ++c) {
        const float d = __fsub_rn(a[c], b[c]);
        acc = __fmaf_rn(d, d, acc);
    }
    return acc;
}

// Vector atomic add of DP floats (DP = 2, 4, 8, 16, 32; rows 8-byte aligned
// for DP = 2 and 16-byte aligned otherwise).
template <int DP>
__device__ __forceinline__ void atomic_add_row(float* dst, const float (&v)[DP], float scale) {
    if constexpr (DP == 2) {
        atomicAdd(reinterpret_cast<float2*>(dst), make_float2(scale * v[0], scale * v[1]));
    } else {
#pragma unroll
        for (int q = 0; q < DP / 4; ++q)
            atomicAdd(reinterpret_cast<float4*>(dst) + q,
                      make_float4(scale * v[4 * q], scale * v[4 * q + 1], scale * v[4 * q + 2],
                                  scale * v[4 * q + 3]));
    }
}

// ---------------------------------------------------------------- HD distances
// Exact FP32 squared distance, one lane per candidate: the squares of the
// even and of the odd features each summed in feature order (two packed
// chains), then the two sums added (zero padding adds nothing). Every FP32 HD
// distance of the library is summed in this order. xs: the own row in
// shared memory.
__device__ __forceinline__ float dist_f32(const float* __restrict__ xs,
                                          const float* __restrict__ xc, int n4) {
    const float4* a = reinterpret_cast<const float4*>(xs);
    const float4* b = reinterpret_cast<const float4*>(xc);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int q = 0; q < n4; ++q) acc = sqdiff2_f4(a[q], __ldg(b + q), acc);
    return hsum2(acc);
}

struct ApproxDist {
    float d2;    // FP32 distance to the dequantised row
    float band;  // bound on |d2 - exact FP32 distance to the master row|
};

// Band of a distance to a dequantised row. acc: the FP32 sum of
// (x_i - x~_c)^2 with the own row x_i exact; E: an upper bound of the
// candidate row's own dequantisation error ||x_c - x~_c||, stored with the
// row when it was quantised. Expanding ||(x_i - x~_c) - (x_c - x~_c)||^2
// and Cauchy-Schwarz give |d2 - d~2| <= 2 ||x_i - x~_c|| E + E^2; the terms
// in gamma cover the FP32 rounding of this sum and of the exact FP32
// distance it is compared with.
__device__ __forceinline__ ApproxDist band_from_row_error(float acc, float E, float gamma) {
    const float b0 = 2.f * sqrtf(acc * (1.f + gamma)) * E + E * E;
    ApproxDist r;
    r.d2 = acc;
    r.band = b0 * (1.f + 4.f * gamma) + gamma * (2.f * acc + 2.f * b0) + 1e-30f;
    return r;
}

// FP8-E4M3 rows with a per-row FP32 scale stored after the codes:
// 16 codes per 16-byte chunk, x~ = code * scale.
__device__ __forceinline__ void fp8x4_to_float(uint32_t w, float s, float (&o)[4]) {
    const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(w & 0xffffu), __NV_E4M3);
    const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(w >> 16), __NV_E4M3);
    const float2 a = mul2(__half22float2(*reinterpret_cast<const __half2*>(&lo)), bcast2(s));
    const float2 b = mul2(__half22float2(*reinterpret_cast<const __half2*>(&hi)), bcast2(s));
    o[0] = a.x;
    o[1] = a.y;
    o[2] = b.x;
    o[3] = b.y;
}


// ------------------------------------------------------- row-group distances
// A warp scores the candidates of its 32 lanes (lane l owns candidate l) by
// groups of G lanes per row (G = 1, 2, 4 or 8): R = 32 / G rows per pass. Lane l works in group l / G on the
// 16-byte chunks s, s + G, s + 2G, ... of the row, s = l mod G, and an xor
// butterfly inside the group adds the partial sums (the butterfly is
// symmetric, so every lane of the group holds the same bits). G = 1 is the
// plain lane-per-row loop of dist_f32. Narrow rows are gathered fastest one
// lane per row, 128-byte rows four lanes per row, rows of several hundred
// bytes eight lanes per row (wide lane-per-row gathers thrash L1).
constexpr uint32_t kNoRow = 0xffffffffu;

__device__ __forceinline__ float group_sum_rt(float v, int G) {
    for (int m = 1; m < G; m <<= 1) v += __shfl_xor_sync(kFull, v, m);
    return v;
}

__device__ __forceinline__ float part_f32(const float* __restrict__ xs, const float* __restrict__ xc, int n4,
                                          int s, int G) {
    const float4* a = reinterpret_cast<const float4*>(xs);
    const float4* b = reinterpret_cast<const float4*>(xc);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int q = s; q < n4; q += G) acc = sqdiff2_f4(a[q], __ldg(b + q), acc);
    return hsum2(acc);
}

// The same sum as part_f32 (same order, same bits) with the loads of up to
// kBatch chunks issued before any is used: one memory round trip per kBatch
// chunks instead of one per four. Pays off for narrow rows read by one or
// two lanes, where the plain loop waits twice per row.
constexpr int kBatch = 8;

template <int G>
__device__ __forceinline__ float part_f32_batched(const float* __restrict__ xs, const float* __restrict__ xc,
                                                  int n4, int s) {
    const float4* a = reinterpret_cast<const float4*>(xs);
    const float4* b = reinterpret_cast<const float4*>(xc);
    float2 acc = make_float2(0.f, 0.f);
    for (int q0 = s; q0 < n4; q0 += kBatch * G) {
        float4 v[kBatch];
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
            const int q = q0 + k * G;
            v[k] = q < n4 ? __ldg(b + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
            const int q = q0 + k * G;
            if (q < n4) acc = sqdiff2_f4(a[q], v[k], acc);
        }
    }
    return hsum2(acc);
}

// FP32 squared distance from the staged own row xs to row cv of X32, for the
// candidate of every lane (0 where cv == kNoRow). All lanes must call it.
template <int G>
__device__ __forceinline__ float group_dist_f32(const float* __restrict__ xs, const float* __restrict__ X32,
                                                int xpitch, int n4, uint32_t cv, int lane) {
    constexpr int R = 32 / G;
    const int g = lane / G, s = lane & (G - 1);
    float mine = 0.f;
#pragma unroll
    for (int p = 0; p < G; ++p) {
        const uint32_t cj = __shfl_sync(kFull, cv, p * R + g);
        float acc = 0.f;
        if (cj != kNoRow) {
            const float* row = X32 + static_cast<int64_t>(cj) * xpitch;
            if constexpr (G <= 2)
                acc = part_f32_batched<G>(xs, row, n4, s);
            else
                acc = part_f32(xs, row, n4, s, G);
        }
        acc = group_sum_rt(acc, G);
        const float v = __shfl_sync(kFull, acc, (lane & (R - 1)) * G);
        if (lane / R == p) mine = v;
    }
    return mine;
}

// Position of the set bit of rank k (0-based, from bit 0) of m; m must have
// more than k set bits. Binary search on prefix population counts.
__device__ __forceinline__ int nth_set_bit(uint32_t m, int k) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const uint32_t low = m & ((1u << w) - 1u);  // bits [pos, pos + w) of the window
        const int c = __popc(low);
        if (c <= k) {
            k -= c;
            m >>= w;
            pos += w;
        } else {
            m = low;
        }
    }
    return pos;
}

// The same FP32 distances (same grouping and summation order, hence the
// same bits) for only the lanes with need == true, packed R to a pass. All
// lanes must call it. NARROW: rows read by one or two lanes load all their
// chunks at once (one round trip; spectrum-1m BF16 refinement 1.161 to 1.129
// ms); callers whose reduced-precision rows take four or more lanes keep the
// plain loop, which their code generation prefers (swissroll-200k 0.368 to
// 0.356 ms).
template <bool NARROW = true>
__device__ __forceinline__ float group_rerank_f32(const float* __restrict__ xs, const float* __restrict__ X32,
                                                  int xpitch, int n4, uint32_t c, bool need, int lane, int G) {
    const uint32_t m = __ballot_sync(kFull, need);
    const int nn = __popc(m);
    const int R = 32 / G, g = lane / G, s = lane & (G - 1);
    const int rank = __popc(m & ((1u << lane) - 1u));
    float mine = 0.f;
    for (int base = 0; base < nn; base += R) {
        const int k = base + g;  // this group scores the k-th flagged lane's row
        const int src = (k < nn) ? nth_set_bit(m, k) : 0;
        const uint32_t cj = __shfl_sync(kFull, c, src);
        float acc = 0.f;
        if (k < nn) {
            const float* row = X32 + static_cast<int64_t>(cj) * xpitch;
            if (NARROW && G == 2)
                acc = part_f32_batched<2>(xs, row, n4, s);
            else if (NARROW && G == 1)
                acc = part_f32_batched<1>(xs, row, n4, s);
            else
                acc = part_f32(xs, row, n4, s, G);
        }
        acc = group_sum_rt(acc, G);
        const int r = rank - base;
        const bool mine_here = need && r >= 0 && r < R;
        const float v = __shfl_sync(kFull, acc, (mine_here ? r : 0) * G);
        if (mine_here) mine = v;
    }
    return mine;
}

// Adds the squared differences between own-row floats 8q .. 8q + 7 and the
// eight BF16 values of chunk q to the two chains of acc (even and odd
// features), in order. A BF16 pair widens to FP32 by a shift and a mask.
__device__ __forceinline__ float2 bf16_pair(uint32_t w) {
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
__device__ __forceinline__ float2 bf16_chunk_acc(const float* __restrict__ xs, const uint4 raw, int q, float2 acc) {
    const float4 x0 = reinterpret_cast<const float4*>(xs)[2 * q];
    const float4 x1 = reinterpret_cast<const float4*>(xs)[2 * q + 1];
    float2 d = sub2(make_float2(x0.x, x0.y), bf16_pair(raw.x));
    acc = fma2(d, d, acc);
    d = sub2(make_float2(x0.z, x0.w), bf16_pair(raw.y));
    acc = fma2(d, d, acc);
    d = sub2(make_float2(x1.x, x1.y), bf16_pair(raw.z));
    acc = fma2(d, d, acc);
    d = sub2(make_float2(x1.z, x1.w), bf16_pair(raw.w));
    return fma2(d, d, acc);
}

// BF16 rows by groups: the distance to the dequantised row and its band
// (band_from_row_error), for the candidate of every lane. BF16 rows hold nq
// chunks of 8 values, then a 16-byte chunk whose first four bytes hold the
// row's error bound E_c >= ||x_c - x~_c||.
// A lane issues the loads of KB of its chunks before using any.
template <int G, int KB>
__device__ __forceinline__ ApproxDist group_dist_bf16(const float* __restrict__ xs,
                                                      const uint8_t* __restrict__ Xq, int qpitch, int nq,
                                                      uint32_t cv, int lane, float gamma) {
    constexpr int R = 32 / G;
    const int g = lane / G, s = lane & (G - 1);
    const int sn = nq & (G - 1);  // the lane of a group that reads the norm chunk
    float my_acc = 0.f, my_nrm = 0.f;
#pragma unroll
    for (int p = 0; p < G; ++p) {
        const uint32_t cj = __shfl_sync(kFull, cv, p * R + g);
        float2 acc2 = make_float2(0.f, 0.f);
        float nrm = 0.f;
        if (cj != kNoRow) {
            const uint4* b = reinterpret_cast<const uint4*>(Xq + static_cast<int64_t>(cj) * qpitch);
            // all of a batch's chunk loads in flight before any is used
            for (int q0 = s; q0 < nq; q0 += KB * G) {
                uint4 raw[KB];
#pragma unroll
                for (int k = 0; k < KB; ++k) {
                    const int q = q0 + k * G;
                    raw[k] = q < nq ? __ldg(b + q) : make_uint4(0u, 0u, 0u, 0u);
                }
#pragma unroll
                for (int k = 0; k < KB; ++k) {
                    const int q = q0 + k * G;
                    if (q < nq) acc2 = bf16_chunk_acc(xs, raw[k], q, acc2);
                }
            }
            if (s == sn) nrm = __ldg(reinterpret_cast<const float*>(b + nq));
        }
        const float acc = group_sum_rt(hsum2(acc2), G);
        const int src = (lane & (R - 1)) * G;
        const float va = __shfl_sync(kFull, acc, src);
        const float vn = __shfl_sync(kFull, nrm, src + sn);
        if (lane / R == p) {
            my_acc = va;
            my_nrm = vn;
        }
    }
    return band_from_row_error(my_acc, my_nrm, gamma);
}

// FP8-E4M3 rows by groups: distance to the dequantised row and its band
// (band_from_row_error), for the candidate of every lane. FP8 rows hold nw
// words of 4 codes, then the row's error bound E_c >= ||x_c - x~_c|| four
// bytes before the scale (scale_off).
template <int G>
__device__ __forceinline__ ApproxDist group_dist_fp8(const float* __restrict__ xs,
                                                     const uint8_t* __restrict__ Xq, int qpitch, int nw,
                                                     int scale_off, uint32_t cv, int lane, float gamma) {
    constexpr int R = 32 / G;
    const int g = lane / G, s = lane & (G - 1);
    const int nch = (nw + 3) >> 2;
    float my_acc = 0.f, my_err = 0.f;
#pragma unroll
    for (int p = 0; p < G; ++p) {
        const uint32_t cj = __shfl_sync(kFull, cv, p * R + g);
        float2 acc2 = make_float2(0.f, 0.f);
        float err = 0.f;
        if (cj != kNoRow) {
            const uint8_t* row = Xq + static_cast<int64_t>(cj) * qpitch;
            const float sc = __ldg(reinterpret_cast<const float*>(row + scale_off));
            if (s == 0) err = __ldg(reinterpret_cast<const float*>(row + scale_off - 4));
            const uint4* b = reinterpret_cast<const uint4*>(row);
            for (int q = s; q < nch; q += G) {
                const uint4 raw = __ldg(b + q);
                const uint32_t w4[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    if (4 * q + m < nw) {
                        float v[4];
                        fp8x4_to_float(w4[m], sc, v);
                        const float4 xi = reinterpret_cast<const float4*>(xs)[4 * q + m];
                        acc2 = sqdiff2_f4(xi, make_float4(v[0], v[1], v[2], v[3]), acc2);
                    }
                }
            }
        }
        const float acc = group_sum_rt(hsum2(acc2), G);
        const int src = (lane & (R - 1)) * G;
        const float va = __shfl_sync(kFull, acc, src);
        const float ve = __shfl_sync(kFull, err, src);
        if (lane / R == p) {
            my_acc = va;
            my_err = ve;
        }
    }
    return band_from_row_error(my_acc, my_err, gamma);
}

// ---------------------------------------------------------------- range checks
// With FUNCSNE_CHECKED defined (the library's range-checked build), every
// point index read from memory and then used to address a row or a list is
// checked against [0, n): an index outside it sets kErrIndex in the device
// error word (reported by funcsne_sync as FUNCSNE_E_RANGE) and is replaced by
// `fallback`, a valid index, so the access stays in bounds. Never traps.
// Without it the macros cost nothing.
#ifdef FUNCSNE_CHECKED
__device__ __forceinline__ uint32_t checked_index(uint32_t j, uint32_t n, uint32_t fallback, uint32_t* err) {
    if (j < n) return j;
    atomicOr(err, kErrIndex);
    return fallback;
}
#define FSNE_IDX(j, n, fallback, err) ::fsne::checked_index((j), (n), (fallback), (err))
// a candidate that the kernel drops when it is out of range: only reported
#define FSNE_FLAG_RANGE(j, n, err) \
    do {                                \
        if (!((j) < (n))) atomicOr((err), kErrIndex); \
    } while (0)
#else
#define FSNE_IDX(j, n, fallback, err) (j)
#define FSNE_FLAG_RANGE(j, n, err) \
    do {                                \
    } while (0)
#endif

// ---------------------------------------------------------------- asynchronous copies
// 16-byte global-to-shared copies that complete in the background
// (cp.async, L2 only): issued for the next point while the current one is
// processed, then waited for by group.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
    const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N of this thread's committed groups are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// ---------------------------------------------------------------- warp hash sets
// Open-addressing set of point indices in shared memory (256 slots, linear
// probing, EMPTY = 0xffffffff). At most 96 entries are ever inserted, so an
// empty slot always exists and every probe sequence ends.
constexpr uint32_t kHashEmpty = 0xffffffffu;

// Open addressing with linear probing over S slots (a power of two, at least
// 128): the top log2(S) bits of a Fibonacci hash pick the first slot.
template <int S = kHashSlots>
__device__ __forceinline__ uint32_t hash_slot(uint32_t x) {
    static_assert(S >= 128 && (S & (S - 1)) == 0, "hash set size");
    constexpr int kShift = 32 - __builtin_ctz(S);
    return (x * 2654435761u) >> kShift;
}

template <int S = kHashSlots>
__device__ __forceinline__ void hset_clear(uint32_t* tab, int lane) {
    const uint4 e = make_uint4(kHashEmpty, kHashEmpty, kHashEmpty, kHashEmpty);
#pragma unroll
    for (int q = 0; q < S / 128; ++q) reinterpret_cast<uint4*>(tab)[lane + 32 * q] = e;
}

template <int S = kHashSlots>
__device__ __forceinline__ void hset_insert(uint32_t* tab, uint32_t x) {
    uint32_t h = hash_slot<S>(x);
    for (int probe = 0; probe < S; ++probe) {
        const uint32_t prev = atomicCAS(tab + h, kHashEmpty, x);
        if (prev == kHashEmpty || prev == x) return;
        h = (h + 1u) & (S - 1);
    }
}

template <int S = kHashSlots>
__device__ __forceinline__ bool hset_has(const uint32_t* tab, uint32_t x) {
    uint32_t h = hash_slot<S>(x);
    for (int probe = 0; probe < S; ++probe) {
        const uint32_t v = tab[h];
        if (v == x) return true;
        if (v == kHashEmpty) return false;
        h = (h + 1u) & (S - 1);
    }
    return false;
}

// ---------------------------------------------------------------- bisection (Eq. 1)
// Warp-wide calibration of beta = 1/(2 sigma^2) for a sorted list of k
// squared distances held as element e = r*32 + lane. With sh = d - d0,
// S = sum exp(-beta sh), U = sum exp(.) sh, V = sum exp(.) sh^2:
// H = ln S + beta U/S and dH/dbeta = -beta (V/S - (U/S)^2) < 0.
// Start from beta0 (> 0: warm restart) or 1/mean(sh); keep a bracket
// [lo, hi] on the root of H = ln perp; take the Newton step when it stays
// inside the bracket, else double (no upper bound yet) or halve the bracket;
// stop when |H - ln perp| < tol, after one last Newton step from the sums of
// that evaluation. The oracle reaches its tolerance by plain bisection.
template <int R>
__device__ __forceinline__ float warp_bisect(const float (&d2)[R], int k, float log_perp,
                                             float beta0, float (&p)[R], int lane) {
    const float d0 = __shfl_sync(kFull, d2[0], 0);
    float sh[R];
#pragma unroll
    for (int r = 0; r < R; ++r) sh[r] = (r * 32 + lane < k) ? (d2[r] - d0) : 0.f;
    const float inv_k = 1.f / static_cast<float>(k);
    if (logf(static_cast<float>(k)) <= log_perp) {
#pragma unroll
        for (int r = 0; r < R; ++r) p[r] = (r * 32 + lane < k) ? inv_k : 0.f;
        return 0.f;
    }
    float beta = beta0;
    if (!(beta > 0.f)) {
        float m = 0.f;
#pragma unroll
        for (int r = 0; r < R; ++r) m += sh[r];
        m = warp_sum(m) * inv_k;
        beta = m > 0.f ? 1.f / m : 1.f;
    }
    constexpr float kLog2e = 1.4426950408889634f;
    float lo = 0.f, hi = INFINITY;
    for (int it = 0; it < kBisectMaxIt; ++it) {
        float S = 0.f, U = 0.f, V = 0.f;
        const float nb = -beta * kLog2e;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (r * 32 + lane < k) {
                const float e = exp2f(nb * sh[r]);
                S += e;
                const float es = e * sh[r];
                U += es;
                V = __fmaf_rn(es, sh[r], V);
            }
        }
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) {
            S += __shfl_xor_sync(kFull, S, m);
            U += __shfl_xor_sync(kFull, U, m);
            V += __shfl_xor_sync(kFull, V, m);
        }
        const float invS = __fdividef(1.f, S);
        const float mu = U * invS;
        const float H = logf(S) + beta * mu;
        const float f = H - log_perp;
        const float slope = -beta * (V * invS - mu * mu);
        if (fabsf(f) < kBisectTol) {
            // converged: one more Newton step from the sums at hand (no new
            // evaluation) takes the entropy error from below the tolerance
            // down to the FP32 evaluation noise
            const float nb2 = beta - __fdividef(f, slope);
            if (slope < 0.f && nb2 > 0.f && isfinite(nb2)) beta = nb2;
            break;
        }
        if (f > 0.f)
            lo = beta;
        else
            hi = beta;
        float nxt = beta - __fdividef(f, slope);
        if (!(slope < 0.f) || !(nxt > lo) || !(nxt < hi)) nxt = isinf(hi) ? 2.f * beta : 0.5f * (lo + hi);
        beta = nxt;
    }
    float S = 0.f;
    const float nb = -beta * kLog2e;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        p[r] = (r * 32 + lane < k) ? exp2f(nb * sh[r]) : 0.f;
        S += p[r];
    }
    S = warp_sum(S);
    const float invS = 1.f / S;
#pragma unroll
    for (int r = 0; r < R; ++r) p[r] *= invS;
    return beta;
}

// Negative sample s of a point: the MurmurHash3 finalizer (fmix32) of words
// 1 and 3 of the point's Philox block for slot s mod 32, salted by s div 32.
__device__ __forceinline__ uint32_t negative_word(uint32_t w1, uint32_t w3, uint32_t pass) {
    uint32_t h = w1 ^ (w3 + (pass + 1u) * 0x9E3779B9u);
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

// Coin of iteration t: HD refinement iff u < p0 + p1 E, by default
// p0 = 0.05 and p1 = 1 - p0 = 0.95 (Section 3). FP64 with explicit rounding
// so host and device agree bit for bit.
__device__ __forceinline__ bool hd_coin(uint32_t t, double E, uint64_t seed, int mode, double p0, double p1) {
    if (mode == kHdAlways) return true;
    if (mode == kHdNever) return false;
    const uint4 w = philox(t, 0u, kStreamCoin, 0u, seed);
    const double p = __dadd_rn(p0, __dmul_rn(p1, E));
    const double u = __dmul_rn(static_cast<double>(w.x), 2.3283064365386962890625e-10);
    return u < p;
}

}  // namespace fsne
