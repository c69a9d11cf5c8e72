// Insertion of new points into a running FUnc-SNE state (Section 3: the
// iteration admits new points without a pre-computation phase).
//
// For each new point i (indices n_old .. N-1), at iteration t:
//   1. k_hd distinct existing points from counter (t, i, INSERT, l), offsets
//      in [0, n_old) with linear probing (one thread per point);
//   2. a warp per point: FP32 distances, (d2, idx) order, then q.rounds
//      rounds (option insert_rounds, default 64) of 32 candidates, round r
//      slot s from counter (t, i, INSERT, 64+32r+s):
//      slots 0-23 a neighbour of a listed neighbour (an existing point's list
//      of iteration t), slots 24-31 a uniform existing point; top-k merge;
//   3. cold-start bisection (beta, P);
//   4. y_i = mean of the HD neighbours' y; v_i = 0; A, R rows cleared;
//   5. LD list = the first k_ld HD neighbours, completed when k_ld > k_hd by
//      distinct random existing points from counter (t, i, INSERT, 2^30+l),
//      above the slots of every round.
#include "device_common.cuh"
#include "launch.h"

namespace fsne {

constexpr int kInsertNnSlots = 24;

__global__ void insert_lists_kernel(InsertParams q) {
    const int64_t i = q.n_old + static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= q.N) return;
    uint32_t off[64];
    const uint32_t m = static_cast<uint32_t>(q.n_old);
    for (int l = 0; l < q.k_hd; ++l) {
        const uint4 w = philox(q.t, static_cast<uint32_t>(i), kStreamInsert, static_cast<uint32_t>(l), q.seed);
        uint32_t o = map_index(w.x, m);
        for (;;) {
            bool taken = false;
            for (int a = 0; a < l; ++a) taken |= (off[a] == o);
            if (!taken) break;
            o = (o + 1u == m) ? 0u : o + 1u;
        }
        off[l] = o;
        q.hd_idx[i * q.k_hd + l] = static_cast<int32_t>(o);
    }
}

template <int DP, int RH>
__global__ void __launch_bounds__(256) insert_refine_kernel(InsertParams q) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float* xs = reinterpret_cast<float*>(smem) + wib * (q.xpitch + 64);
    int32_t* s_list = reinterpret_cast<int32_t*>(xs + q.xpitch);  // 64 entries
    const int k = q.k_hd;
    const int64_t gi = q.n_old + static_cast<int64_t>(blockIdx.x) * 8 + wib;
    if (gi >= q.N) return;
    const uint32_t i = static_cast<uint32_t>(gi);
    const float* xrow = q.X32 + gi * q.xpitch;
    for (int f = lane * 4; f < q.xpitch; f += 128)
        *reinterpret_cast<float4*>(xs + f) = __ldg(reinterpret_cast<const float4*>(xrow + f));
    __syncwarp();
    uint64_t key[RH];
#pragma unroll
    for (int r = 0; r < RH; ++r) {
        const int e = r * 32 + lane;
        key[r] = kSentinel;
        const uint32_t j = e < k ? static_cast<uint32_t>(q.hd_idx[gi * k + e]) : kNoRow;
        const float d = group_rerank_f32(xs, q.X32, q.xpitch, q.n4, j, e < k, lane, q.g);
        if (e < k) key[r] = make_key(d, j);
    }
    warp_sort<RH>(key, lane);
    const uint32_t m = static_cast<uint32_t>(q.n_old);
    for (int round = 0; round < q.rounds; ++round) {
        uint32_t li[RH];
#pragma unroll
        for (int r = 0; r < RH; ++r) li[r] = key_idx(key[r]);
        const uint4 w = philox(q.t, i, kStreamInsert, static_cast<uint32_t>(64 + 32 * round + lane), q.seed);
        const uint32_t a = warp_get<RH>(li, map_index(w.x, k));
        uint32_t c;
        if (lane < kInsertNnSlots)
            c = static_cast<uint32_t>(q.hd_idx[static_cast<int64_t>(a) * k + map_index(w.y, k)]);
        else
            c = map_index(w.x, m);
        bool valid = c < m;
#pragma unroll
        for (int r = 0; r < RH; ++r)
            for (int s = 0; s < 32; ++s) valid &= (__shfl_sync(kFull, li[r], s) != c);
        const unsigned same = __match_any_sync(kFull, c);
        valid &= (same & ((1u << lane) - 1u)) == 0u;
        const float dc = group_rerank_f32(xs, q.X32, q.xpitch, q.n4, c, valid, lane, q.g);
        const uint64_t ck = valid ? make_key(dc, c) : kSentinel;
        merge_candidates<RH>(key, ck, lane);
    }
    float d2[RH], pv[RH];
#pragma unroll
    for (int r = 0; r < RH; ++r) d2[r] = key_d2(key[r]);
    const float b = warp_bisect<RH>(d2, k, q.log_perp, 0.f, pv, lane);
    // write the HD list, P, beta; stage the list for the LD seeding
    float ysum[DP];
#pragma unroll
    for (int c = 0; c < DP; ++c) ysum[c] = 0.f;
#pragma unroll
    for (int r = 0; r < RH; ++r) {
        const int e = r * 32 + lane;
        if (e < k) {
            const uint32_t j = key_idx(key[r]);
            q.hd_idx[gi * k + e] = static_cast<int32_t>(j);
            q.hd_d2[gi * k + e] = d2[r];
            q.P[gi * k + e] = pv[r];
            s_list[e] = static_cast<int32_t>(j);
            float yj[DP];
            load_row<DP>(q.Y + static_cast<int64_t>(j) * DP, yj);
#pragma unroll
            for (int c = 0; c < DP; ++c) ysum[c] += yj[c];
        }
    }
    if (lane == 0) q.beta[gi] = b;
#pragma unroll
    for (int c = 0; c < DP; ++c) ysum[c] = warp_sum(ysum[c]);
    if (lane < DP) {
        float v = ysum[0];
#pragma unroll
        for (int c = 1; c < DP; ++c)
            if (lane == c) v = ysum[c];
        q.Y[gi * DP + lane] = v / static_cast<float>(k);
        q.V[gi * DP + lane] = 0.f;
        q.A[gi * DP + lane] = 0.f;
        q.R[gi * DP + lane] = 0.f;
    }
    __syncwarp();
    if (lane == 0) {
        const int kl = q.k_ld;
        const int mcopy = kl < k ? kl : k;
        for (int l = 0; l < mcopy; ++l) q.ld_idx[gi * kl + l] = s_list[l];
        for (int l = mcopy; l < kl; ++l) {
            const uint4 w = philox(q.t, i, kStreamInsert, 0x40000000u + static_cast<uint32_t>(l), q.seed);
            uint32_t o = map_index(w.x, m);
            for (;;) {
                bool taken = false;
                for (int s = 0; s < l; ++s) taken |= (static_cast<uint32_t>(q.ld_idx[gi * kl + s]) == o);
                if (!taken) break;
                o = (o + 1u == m) ? 0u : o + 1u;
            }
            q.ld_idx[gi * kl + l] = static_cast<int32_t>(o);
        }
    }
}

cudaError_t launch_insert(const InsertParams& q, int DP, cudaStream_t s) {
    const int64_t n_new = q.N - q.n_old;
    if (n_new <= 0) return cudaSuccess;
    insert_lists_kernel<<<static_cast<int>((n_new + 127) / 128), 128, 0, s>>>(q);
    const int blocks = static_cast<int>((n_new + 7) / 8);
    const size_t smem = static_cast<size_t>(8) * (q.xpitch + 64) * sizeof(float);
#define FSNE_INS(dp, rh)                                                                                       \
    if (DP == dp && (q.k_hd <= 32 ? 1 : 2) == rh) {                                                            \
        cudaFuncSetAttribute(insert_refine_kernel<dp, rh>, cudaFuncAttributeMaxDynamicSharedMemorySize,        \
                             static_cast<int>(smem));                                                          \
        insert_refine_kernel<dp, rh><<<blocks, 256, smem, s>>>(q);                                             \
        return cudaGetLastError();                                                                             \
    }
    FSNE_INS(2, 1) FSNE_INS(4, 1) FSNE_INS(8, 1) FSNE_INS(16, 1) FSNE_INS(32, 1)
    FSNE_INS(2, 2) FSNE_INS(4, 2) FSNE_INS(8, 2) FSNE_INS(16, 2) FSNE_INS(32, 2)
#undef FSNE_INS
    return cudaErrorInvalidValue;
}

}  // namespace fsne
