// The FUnc-SNE iteration as three phase kernels (one warp per point,
// persistent grids) plus the update kernel (update_kernel.cu).
//
// Iteration t, Jacobi order (all reads see state t; writes go to the t+1
// list buffers, to P/beta of the point itself, or to accumulators):
//   hd_refine_kernel  (Section 3) when the coin of t fires: 32 candidates
//     (slots 0-15 HD neighbour of an HD neighbour, 16-19 LD neighbour,
//     20-23 LD neighbour of an LD neighbour, 24-31 random; words 0-1 of the
//     slot's Philox block), dedup against the list / self / earlier slots,
//     FP32 distances (or dequantised BF16 / FP8 distances with an error band
//     and an exact FP32 re-rank of every candidate that can enter), top-k on
//     (d2, idx), new-neighbour flag, warm-restart bandwidth calibration;
//   ld_refine_kernel  every iteration: 32 candidates (slots 0-15 LD
//     neighbour of an LD neighbour, 16-23 HD neighbour of iteration t, 24-31
//     random; words 2-3), distances at Y_t of the old list and the
//     candidates, top-k_ld on (d2, idx);
//   forces_kernel     over the lists of t+1 at Y_t: attraction
//     4 (p_{j|i}/2N) w^{1/alpha} (y_i - y_j) added to A_i and subtracted from
//     A_j; repulsion 4 (w_ij / Zhat_t) w^{1/alpha} (y_i - y_j) over
//     S_i = HD u LD and over n_neg Philox-seeded negatives outside S_i
//     scaled by (N-1)/n_neg; per-point Z_t terms summed per block in FP64.
// hd_refine and ld_refine only read state t, so they may run concurrently.
#pragma once

#include "device_common.cuh"

namespace fsne {

constexpr int kWarpsPerBlock = 8;
// Up to this many qualifying candidates are merged by single insertions;
// more go through the bitonic network (HD and LD refinement).
constexpr int kInsertMaxHd = 12;
constexpr int kInsertMaxLd = 8;

struct ListView {
    const int32_t* __restrict__ hd_idx_c;
    const float* __restrict__ hd_d2_c;
    int32_t* __restrict__ hd_idx_n;
    float* __restrict__ hd_d2_n;
    const int32_t* __restrict__ ld_idx_c;
    int32_t* __restrict__ ld_idx_n;
};

__device__ __forceinline__ ListView list_view(const StepParams& p, int hc, int lc) {
    ListView v;
    v.hd_idx_c = hc ? p.hd_idx1 : p.hd_idx0;
    v.hd_d2_c = hc ? p.hd_d21 : p.hd_d20;
    v.hd_idx_n = hc ? p.hd_idx0 : p.hd_idx1;
    v.hd_d2_n = hc ? p.hd_d20 : p.hd_d21;
    v.ld_idx_c = lc ? p.ld_idx1 : p.ld_idx0;
    v.ld_idx_n = lc ? p.ld_idx0 : p.ld_idx1;
    return v;
}

// ------------------------------------------------------------------ HD refinement
// Resident blocks per SM the registers are sized for. The kernel waits mostly
// on memory; the registers hold the batches of row chunks in flight
// (group_dist_bf16) and, in the pipelined variant (PF), the next point's
// lists. Five blocks (48 registers) pay for FP32 rows read by up to four
// lanes with k_hd <= 32 (spectrum-1m 1.116 to 1.096 ms, swissroll-200k 0.321
// to 0.308 ms); the reduced-precision, wide-row and k_hd = 64 variants are
// faster with four (64 registers): five made pixels-70k BF16 0.517 to 0.575
// ms and spectrum-1m BF16 1.169 to 1.190 ms.
template <int XM, int RH, int G>
constexpr int hd_refine_min_blocks() { return (XM == 0 && RH == 1 && G <= 4) ? 5 : 4; }

// G: lanes per gathered row, of the FP32 rows (XM = 0) or of the BF16 / FP8
// rows (the exact re-rank then takes the FP32 rows' p.gf at run time).
// PF: software pipelining over the points of a warp: the next point's lists
// are loaded into registers and its own row is copied into the second of two
// shared-memory row buffers (cp.async) while the current point is scored,
// which takes two memory round trips off every point's chain of dependent
// loads.
template <int RH, int XM, int G, bool PF>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, hd_refine_min_blocks<XM, RH, G>())
hd_refine_kernel(const StepParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    float* const xbuf = reinterpret_cast<float*>(smem + wib * p.smem_per_warp);
    uint32_t* tab = reinterpret_cast<uint32_t*>(xbuf + (PF ? 2 : 1) * p.xs_floats);
    __shared__ unsigned long long s_cnt[kWarpsPerBlock][3];

    const DevScalars* sc = p.sc;
    const uint32_t t = sc->t;
    // the coin refines every point; without it, only the points of the
    // insertion window (if one is open) are refined (uniform over the grid)
    const bool fire = hd_coin(t, sc->E, p.seed, p.hd_mode, p.coin_p0, p.coin_p1);
    if (!fire && !fresh_only(sc, t, fire, p.N)) return;
    const int64_t lo = fire ? 0 : sc->fresh_lo;
    const ListView L = list_view(p, sc->hd_cur, sc->ld_cur);
    const uint32_t N = static_cast<uint32_t>(p.N);
    const int k_hd = p.k_hd, k_ld = p.k_ld;

    for (int f = p.xpitch + lane; f < p.xs_floats; f += 32) {
        xbuf[f] = 0.f;
        if (PF) xbuf[p.xs_floats + f] = 0.f;
    }
    // per-lane counts: a lane scores at most one candidate a point, so each
    // stays below N < 2^31; widened for the block sums
    uint32_t c_new = 0, c_scored = 0, c_rerank = 0;

    // the lists of point g (HD indices and distances, LD indices)
    auto load_lists = [&](int64_t g, uint32_t (&hi)[RH], float (&h2)[RH], uint32_t& li) {
#pragma unroll
        for (int r = 0; r < RH; ++r) {
            const int e = r * 32 + lane;
            hi[r] = e < k_hd ? static_cast<uint32_t>(__ldg(L.hd_idx_c + g * k_hd + e)) : 0xffffffffu;
            h2[r] = e < k_hd ? __ldg(L.hd_d2_c + g * k_hd + e) : __uint_as_float(0x7f800000u);
        }
        li = lane < k_ld ? static_cast<uint32_t>(__ldg(L.ld_idx_c + g * k_ld + lane)) : 0xffffffffu;
    };
    // point g's own FP32 row into the row buffer dst, asynchronously; one
    // commit group per call on every lane (empty for g >= N)
    auto stage_row = [&](int64_t g, float* dst) {
        if (g < p.N) {
            const float* xrow = p.X32 + g * p.xpitch;
            for (int f = lane * 4; f < p.xpitch; f += 128) cp_async16(dst + f, xrow + f);
        }
        cp_async_commit();
    };
    const int64_t tw = static_cast<int64_t>(gridDim.x) * kWarpsPerBlock;
    const int64_t g0 = lo + static_cast<int64_t>(blockIdx.x) * kWarpsPerBlock + wib;
    uint32_t n_hidx[RH];
    float n_hd2[RH];
    uint32_t n_lidx = 0;
    int buf = 0;
    if constexpr (PF) {
        if (g0 < p.N) load_lists(g0, n_hidx, n_hd2, n_lidx);
        stage_row(g0, xbuf);
    }
    for (int64_t gi = g0; gi < p.N; gi += tw) {
        const uint32_t i = static_cast<uint32_t>(gi);
        uint32_t hidx[RH];
        float hd2[RH];
        uint32_t lidx;
        float* xs = xbuf;
        if constexpr (PF) {
#pragma unroll
            for (int r = 0; r < RH; ++r) {
                hidx[r] = n_hidx[r];
                hd2[r] = n_hd2[r];
            }
            lidx = n_lidx;
            const int64_t gn = gi + tw;
            if (gn < p.N) load_lists(gn, n_hidx, n_hd2, n_lidx);
            stage_row(gn, xbuf + (buf ^ 1) * p.xs_floats);
            xs = xbuf + buf * p.xs_floats;
        } else {
            load_lists(gi, hidx, hd2, lidx);
        }
        const uint4 w = philox(t, i, kStreamRefine, static_cast<uint32_t>(lane), p.pk);
        if constexpr (PF) {
            cp_async_wait<1>();  // this point's row has landed
        } else {
            __syncwarp();
            const float* xrow = p.X32 + gi * p.xpitch;
            for (int f = lane * 4; f < p.xpitch; f += 128)
                *reinterpret_cast<float4*>(xs + f) = __ldg(reinterpret_cast<const float4*>(xrow + f));
        }
        hset_clear(tab, lane);
        __syncwarp();
#pragma unroll
        for (int r = 0; r < RH; ++r)
            if (r * 32 + lane < k_hd) hset_insert(tab, hidx[r]);
        const uint32_t e0 = lane < kHdNnEnd ? map_index(w.x, k_hd) : map_index(w.x, k_ld);
        // hv and lv are shuffled warp-wide; each lane uses (and, in the
        // checked build, range-checks) only the one its slot reads
        const uint32_t hv = warp_get<RH>(hidx, e0);
        const uint32_t lv = __shfl_sync(kFull, lidx, static_cast<int>(e0 & 31u));
        uint32_t c;
        if (lane < kHdNnEnd)
            c = static_cast<uint32_t>(__ldg(L.hd_idx_c + static_cast<int64_t>(FSNE_IDX(hv, N, i, &p.sc->err)) * k_hd +
                                            map_index(w.y, k_hd)));
        else if (lane < kHdLdNbEnd)
            c = lv;
        else if (lane < kHdLdNnEnd)
            c = static_cast<uint32_t>(__ldg(L.ld_idx_c + static_cast<int64_t>(FSNE_IDX(lv, N, i, &p.sc->err)) * k_ld +
                                            map_index(w.y, k_ld)));
        else
            c = map_other(w.x, N, i);
        __syncwarp();
        FSNE_FLAG_RANGE(c, N, &p.sc->err);
        bool valid = (c != i) && (c < N) && !hset_has(tab, c);
        valid &= (__match_any_sync(kFull, c) & ((1u << lane) - 1u)) == 0u;

        uint64_t ck = kSentinel;
        const uint32_t cv = valid ? c : kNoRow;
        if constexpr (XM == 0) {
            const float d = group_dist_f32<G>(xs, p.X32, p.xpitch, p.n4, cv, lane);
            if (valid) ck = make_key(d, c);
        } else {
            const float thr = warp_get<RH>(hd2, static_cast<uint32_t>(k_hd - 1));
            ApproxDist a;
            if constexpr (XM == 1)
                // a lane's row chunks in flight: 8 with the lists of the
                // k_hd > 32 variant, 4 otherwise (eight made the 784-d rows
                // of pixels-70k 26% slower)
                a = group_dist_bf16<G, RH == 2 ? 8 : 4>(xs, p.Xq, p.qpitch, p.nq, cv, lane, p.q_gamma);
            else  // nq = code words for FP8
                a = group_dist_fp8<G>(xs, p.Xq, p.qpitch, p.nq, p.qscale_off, cv, lane, p.q_gamma);
            const bool need = valid && __fsub_rd(a.d2, a.band) <= thr;
            c_scored += valid ? 1 : 0;
            c_rerank += need ? 1 : 0;
            // candidates that can enter: the exact FP32 distance, computed as
            // in FP32 mode (same grouping), so the lists equal FP32 mode's
            const float d = group_rerank_f32<(G <= 2)>(xs, p.X32, p.xpitch, p.n4, c, need, lane, p.gf);
            if (need) ck = make_key(d, c);
        }
        // flag: some candidate precedes the old k-th entry
        uint64_t keys[RH];
#pragma unroll
        for (int r = 0; r < RH; ++r) keys[r] = (r * 32 + lane < k_hd) ? make_key(hd2[r], hidx[r]) : kSentinel;
        const uint64_t kth = warp_get64<RH>(keys, static_cast<uint32_t>(k_hd - 1));
        const int nqual = __popc(__ballot_sync(kFull, ck < kth));
        if (nqual > 0) {
            if (nqual > kInsertMaxHd)
                merge_candidates<RH>(keys, ck, lane);
            else
                insert_candidates<RH>(keys, ck, kth, lane);
        }
        float nd2[RH];
#pragma unroll
        for (int r = 0; r < RH; ++r) {
            const int e = r * 32 + lane;
            nd2[r] = key_d2(keys[r]);
            if (e < k_hd) {
                L.hd_idx_n[gi * k_hd + e] = static_cast<int32_t>(key_idx(keys[r]));
                L.hd_d2_n[gi * k_hd + e] = nd2[r];
            }
        }
        if (nqual > 0) {
            float pv[RH];
            const float b = warp_bisect<RH>(nd2, k_hd, p.log_perp, p.beta[gi], pv, lane);
#pragma unroll
            for (int r = 0; r < RH; ++r) {
                const int e = r * 32 + lane;
                if (e < k_hd) p.P[gi * k_hd + e] = pv[r];
            }
            if (lane == 0) p.beta[gi] = b;
            ++c_new;
        }
        __syncwarp();
        buf ^= 1;
    }
    if constexpr (PF) cp_async_wait<0>();
    unsigned long long cs = c_scored, cr = c_rerank;
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
        cs += __shfl_xor_sync(kFull, cs, m);
        cr += __shfl_xor_sync(kFull, cr, m);
    }
    if (lane == 0) {
        s_cnt[wib][0] = static_cast<unsigned long long>(c_new);
        s_cnt[wib][1] = cs;
        s_cnt[wib][2] = cr;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long a = 0, b = 0, c = 0;
        for (int v = 0; v < kWarpsPerBlock; ++v) {
            a += s_cnt[v][0];
            b += s_cnt[v][1];
            c += s_cnt[v][2];
        }
        p.cnt[3 * blockIdx.x + 0] = a;
        p.cnt[3 * blockIdx.x + 1] = b;
        p.cnt[3 * blockIdx.x + 2] = c;
    }
}

// LD rows are gathered by groups of G = DP/CW lanes (CW = 4 floats per lane,
// 2 when DP = 2): one 16-byte load per lane, R = 32/G rows per warp
// instruction. Lane l owns components [CW (l mod G), CW (l mod G) + CW) of
// every row its group touches.
template <int DP, int CWP = 4>
struct RowSplit {
    static constexpr int CW = DP >= CWP ? CWP : DP;  // floats per lane
    static constexpr int G = DP / CW;                 // lanes per row
    static constexpr int R = 32 / G;                  // rows per pass
};

// 32 bytes of read-only global data in one load (a 256-bit load, sm_100
// and later); src must be 32-byte aligned.
__device__ __forceinline__ void ldg_v8(const float* __restrict__ src, float* v) {
    asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "l"(src));
}

// CW consecutive floats of a row. A chunk of 8 (32-byte aligned: LD rows of
// 8 floats and more) is one 256-bit load, so two lanes cover a 64-byte row in
// one warp load: 1.395 to 1.381 ms for the forces and 0.957 to 0.935 ms for
// the two-lane LD refinement on 1M points at d = 16. Chunks of 16 stay on
// 128-bit loads (two 256-bit loads made the d = 32 LD refinement slower,
// 2.62 to 2.91 ms).
template <int CW>
__device__ __forceinline__ void load_chunk(const float* __restrict__ src, float (&v)[CW]) {
    if constexpr (CW == 8) {
        ldg_v8(src, v);
    } else if constexpr (CW % 4 == 0) {
#pragma unroll
        for (int q = 0; q < CW / 4; ++q) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(src) + q);
            v[4 * q] = a.x;
            v[4 * q + 1] = a.y;
            v[4 * q + 2] = a.z;
            v[4 * q + 3] = a.w;
        }
    } else {
        const float2 a = __ldg(reinterpret_cast<const float2*>(src));
        v[0] = a.x;
        v[1] = a.y;
    }
}

// Adds scale * v (CW floats as CW/2 pairs) to dst with vector atomics.
template <int CW>
__device__ __forceinline__ void atomic_add_chunk(float* dst, const float2 (&v)[CW / 2], float scale) {
    if constexpr (CW % 4 == 0) {
#pragma unroll
        for (int q = 0; q < CW / 4; ++q) {
            const float2 a = mul2(bcast2(scale), v[2 * q]), b = mul2(bcast2(scale), v[2 * q + 1]);
            atomicAdd(reinterpret_cast<float4*>(dst) + q, make_float4(a.x, a.y, b.x, b.y));
        }
    } else {
        atomicAdd(reinterpret_cast<float2*>(dst), mul2(bcast2(scale), v[0]));
    }
}

// Sum over the G lanes of a row group (xor butterfly inside the group).
template <int G>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int m = 1; m < G; m <<= 1) v += __shfl_xor_sync(kFull, v, m);
    return v;
}

// ------------------------------------------------------------------ LD refinement
// Squared LD distances from y_i to row cv of Y for the candidate of every
// lane (0 where cv == kNoRow), rows read by groups of G lanes: lane l holds
// the CW = DP / G components CW (l mod G) ... of y_i in yi. All lanes call it.
template <int DP, int G>
__device__ __forceinline__ float group_ld_dist(const float (&yi)[DP / G], const float* __restrict__ Y,
                                               uint32_t cv, int lane) {
    constexpr int CW = DP / G, R = 32 / G;
    const int g = lane / G, s = lane % G;
    float mine = 0.f;
#pragma unroll
    for (int p = 0; p < G; ++p) {
        const uint32_t cj = __shfl_sync(kFull, cv, p * R + g);
        float v[CW];
        if (cj != kNoRow) {
            load_chunk<CW>(Y + static_cast<int64_t>(cj) * DP + CW * s, v);
        } else {
#pragma unroll
            for (int c = 0; c < CW; ++c) v[c] = yi[c];
        }
        float2 acc2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < CW; c += 2) {
            const float2 d = sub2(make_float2(yi[c], yi[c + 1]), make_float2(v[c], v[c + 1]));
            acc2 = fma2(d, d, acc2);
        }
        const float acc = group_sum<G>(hsum2(acc2));
        const float val = __shfl_sync(kFull, acc, (lane % R) * G);
        if (lane / R == p) mine = val;
    }
    return mine;
}

// Lanes per LD row in the LD refinement: rows of 32 bytes and more are read
// two lanes per row (both 16-byte halves of a 32-byte sector in one request).
template <int DP>
__host__ __device__ constexpr int ld_lanes() { return DP >= 8 ? 2 : 1; }

// Reduce-scatter of G values over the G lanes of a row group (xor partners
// G/2, ..., 1, recursive halving): afterwards v[0] of lane s of the group
// holds the group sum of element s.
template <int G, int C = G>
__device__ __forceinline__ void group_reduce_scatter(float (&v)[G], int s) {
    if constexpr (C > 1) {
        constexpr int H = C / 2;
        const bool up = (s & H) != 0;
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const float send = up ? v[k] : v[k + H];
            const float keep = up ? v[k + H] : v[k];
            v[k] = keep + __shfl_xor_sync(kFull, send, H);
        }
        group_reduce_scatter<G, H>(v, s);
    }
}

// Squared LD distances from y_i to row cv of Y for the row of every lane
// (0 where cv == kNoRow), rows of DP >= 8 floats read by G = DP/4 lanes with
// one 16-byte load each: G warp loads of R1 = 32/G whole rows each (one
// cache-line wavefront per row). Lane l holds components 4 (l mod G) ... of
// y_i in yi. The partial sums are reduce-scattered inside each group and one
// shuffle hands every lane its own row's sum. All lanes call it.
template <int DP>
__device__ __forceinline__ float ld_dist_rows(const float4 yi, const float* __restrict__ Y, uint32_t cv,
                                              int lane) {
    constexpr int G = DP / 4, R1 = 32 / G;
    const int g = lane / G, s = lane % G;
    float ps[G];
#pragma unroll
    for (int q = 0; q < G; ++q) {
        const uint32_t cj = __shfl_sync(kFull, cv, q * R1 + g);
        const float4 v = cj != kNoRow ? __ldg(reinterpret_cast<const float4*>(Y + static_cast<int64_t>(cj) * DP + 4 * s))
                                      : yi;
        ps[q] = hsum2(sq2_f4(yi, v));
    }
    group_reduce_scatter<G>(ps, s);
    // lane (g, s) now holds row s R1 + g; row l sits on lane (l mod R1) G + l / R1
    return __shfl_sync(kFull, ps[0], (lane % R1) * G + lane / R1);
}

// PAIR: rows of 8 or more floats are gathered by ld_dist_rows (DP/4 lanes
// per row, one 16-byte load each), and the neighbour-of-neighbour index
// loads are issued before the old list's rows are gathered, so the two
// memory round trips overlap. Otherwise group_ld_dist with ld_lanes lanes.
// The Philox block of a lane in the LD refinement, with the round keys from
// the launch parameters for rows of 16 floats and bumped in the kernel
// otherwise. With the parameter keys the compiler keeps some of them in
// registers; measured after a 200-iteration burn-in, that paid at d = 16
// (spectrum-1m: 0.821 to 0.790 ms) and cost at d = 8 and d = 32
// (swissroll-200k 0.131 to 0.135 ms, lowrank-2m 2.08 to 2.18 ms).
template <int DP>
__device__ __forceinline__ uint4 ld_philox(uint32_t t, uint32_t i, int lane, const StepParams& p) {
    if constexpr (DP == 16)
        return philox(t, i, kStreamRefine, static_cast<uint32_t>(lane), p.pk);
    else
        return philox(t, i, kStreamRefine, static_cast<uint32_t>(lane), p.seed);
}

template <int DP, int RH, bool PAIR>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 4)
ld_refine_kernel(const StepParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    uint32_t* tab = reinterpret_cast<uint32_t*>(smem) + wib * kHashSlots;

    const DevScalars* sc = p.sc;
    const uint32_t t = sc->t;
    const ListView L = list_view(p, sc->hd_cur, sc->ld_cur);
    const uint32_t N = static_cast<uint32_t>(p.N);
    const int k_hd = p.k_hd, k_ld = p.k_ld;
    const float* __restrict__ Y = p.Y;

    const int64_t tw = static_cast<int64_t>(gridDim.x) * kWarpsPerBlock;
    for (int64_t gi = static_cast<int64_t>(blockIdx.x) * kWarpsPerBlock + wib; gi < p.N; gi += tw) {
        const uint32_t i = static_cast<uint32_t>(gi);
        uint32_t hidx[RH];
#pragma unroll
        for (int r = 0; r < RH; ++r) {
            const int e = r * 32 + lane;
            hidx[r] = e < k_hd ? static_cast<uint32_t>(__ldg(L.hd_idx_c + gi * k_hd + e)) : 0xffffffffu;
        }
        const uint32_t lidx = lane < k_ld ? static_cast<uint32_t>(__ldg(L.ld_idx_c + gi * k_ld + lane)) : 0xffffffffu;
        float d_old, d_c;
        uint32_t cand_c;
        bool cand_valid;
        if constexpr (PAIR) {
            const float4 yi = __ldg(reinterpret_cast<const float4*>(Y + gi * DP + 4 * (lane % (DP / 4))));
            const uint4 w = ld_philox<DP>(t, i, lane, p);
            const uint32_t e0 = lane < kLdNnEnd ? map_index(w.z, k_ld) : map_index(w.z, k_hd);
            const uint32_t lv = __shfl_sync(kFull, lidx, static_cast<int>(e0 & 31u));
            const uint32_t hv = warp_get<RH>(hidx, e0);
            // in flight while the old list's rows are gathered
            const uint32_t cnn =
                lane < kLdNnEnd ? static_cast<uint32_t>(__ldg(L.ld_idx_c +
                                                              static_cast<int64_t>(FSNE_IDX(lv, N, i, &p.sc->err)) * k_ld +
                                                              map_index(w.w, k_ld)))
                                : 0u;
            d_old = ld_dist_rows<DP>(yi, Y, lane < k_ld ? FSNE_IDX(lidx, N, i, &p.sc->err) : kNoRow, lane);
            hset_clear(tab, lane);
            __syncwarp();
            if (lane < k_ld) hset_insert(tab, lidx);
            const uint32_t c = lane < kLdNnEnd ? cnn : (lane < kLdHdNbEnd ? hv : map_other(w.z, N, i));
            FSNE_FLAG_RANGE(c, N, &p.sc->err);
            __syncwarp();
            bool valid = (c != i) && (c < N) && !hset_has(tab, c);
            valid &= (__match_any_sync(kFull, c) & ((1u << lane) - 1u)) == 0u;
            d_c = ld_dist_rows<DP>(yi, Y, valid ? c : kNoRow, lane);
            cand_c = c;
            cand_valid = valid;
        } else {
            constexpr int GL = ld_lanes<DP>();
            float yi[DP / GL];
            load_chunk<DP / GL>(Y + gi * DP + (DP / GL) * (lane % GL), yi);
            const uint4 w = ld_philox<DP>(t, i, lane, p);
            hset_clear(tab, lane);
            __syncwarp();
            if (lane < k_ld) hset_insert(tab, lidx);
            const uint32_t e0 = lane < kLdNnEnd ? map_index(w.z, k_ld) : map_index(w.z, k_hd);
            const uint32_t lv = __shfl_sync(kFull, lidx, static_cast<int>(e0 & 31u));
            const uint32_t hv = warp_get<RH>(hidx, e0);
            uint32_t c;
            if (lane < kLdNnEnd)
                c = static_cast<uint32_t>(__ldg(L.ld_idx_c + static_cast<int64_t>(FSNE_IDX(lv, N, i, &p.sc->err)) * k_ld +
                                                map_index(w.w, k_ld)));
            else if (lane < kLdHdNbEnd)
                c = hv;
            else
                c = map_other(w.z, N, i);
            __syncwarp();
            bool valid = (c != i) && (c < N) && !hset_has(tab, c);
            valid &= (__match_any_sync(kFull, c) & ((1u << lane) - 1u)) == 0u;
            FSNE_FLAG_RANGE(c, N, &p.sc->err);
            d_old = group_ld_dist<DP, GL>(yi, Y, lane < k_ld ? FSNE_IDX(lidx, N, i, &p.sc->err) : kNoRow, lane);
            d_c = group_ld_dist<DP, GL>(yi, Y, valid ? c : kNoRow, lane);
            cand_c = c;
            cand_valid = valid;
        }
        const uint32_t c = cand_c;
        const bool valid = cand_valid;
        uint64_t lk[1] = {lane < k_ld ? make_key(d_old, lidx) : kSentinel};
        const uint64_t ck = valid ? make_key(d_c, c) : kSentinel;
        // the old list ordered under the distances at Y_t, then the candidates
        warp_sort<1>(lk, lane);
        const uint64_t thr = shfl64(lk[0], k_ld - 1);
        const int nqual = __popc(__ballot_sync(kFull, ck < thr));
        if (nqual > kInsertMaxLd)
            merge_candidates<1>(lk, ck, lane);
        else if (nqual > 0)
            insert_candidates<1>(lk, ck, thr, lane);
        if (lane < k_ld) L.ld_idx_n[gi * k_ld + lane] = static_cast<int32_t>(key_idx(lk[0]));
        __syncwarp();
    }
}

// Reduce-scatter of V-element vectors over the lanes that share lane mod G
// (xor partners at distances 16, 8, ..., G): while a lane holds more than one
// element it keeps half and sends half (recursive halving), later stages add
// single elements. Afterwards v[0 .. C) holds elements [base, base + C) of
// the sum, C = scatter_count<V, G>(); `owner` is false on the lanes that hold
// a copy of another lane's elements.
template <int V, int G>
__host__ __device__ constexpr int scatter_count() {
    int c = V;
    for (int m = 16; m >= G; m >>= 1)
        if (c > 1) c >>= 1;
    return c;
}

template <int V, int C, int M, int G>
__device__ __forceinline__ void reduce_scatter_stages(float (&v)[V], int lane, int& base, bool& owner) {
    if constexpr (M >= G && M >= 1) {
        if constexpr (C > 1) {
            constexpr int H = C / 2;
            const bool up = (lane & M) != 0;
#pragma unroll
            for (int k = 0; k < H; ++k) {
                const float send = up ? v[k] : v[k + H];
                const float keep = up ? v[k + H] : v[k];
                v[k] = keep + __shfl_xor_sync(kFull, send, M);
            }
            if (up) base += H;
            reduce_scatter_stages<V, H, M / 2, G>(v, lane, base, owner);
        } else {
            v[0] += __shfl_xor_sync(kFull, v[0], M);
            if (lane & M) owner = false;
            reduce_scatter_stages<V, 1, M / 2, G>(v, lane, base, owner);
        }
    }
}

template <int DP>
constexpr int forces_min_blocks() { return 4; }

template <int DP, int RH, int CWP>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, forces_min_blocks<DP>())
forces_kernel(const StepParams p) {
    using S = RowSplit<DP, CWP>;
    constexpr int CW = S::CW, G = S::G, R = S::R;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    uint32_t* tab = reinterpret_cast<uint32_t*>(smem) + wib * kForceHashSlots;
    __shared__ double s_z[kWarpsPerBlock];

    const DevScalars* sc = p.sc;
    const uint32_t t = sc->t;
    const bool fire = hd_coin(t, sc->E, p.seed, p.hd_mode, p.coin_p0, p.coin_p1);
    // lists of iteration t+1: the HD buffer flips only when the coin fired
    // (the rows of an insertion window refined alone were copied back into
    // the current buffer by fresh_lists_kernel)
    const int32_t* __restrict__ hd_new = (sc->hd_cur ^ (fire ? 1 : 0)) ? p.hd_idx1 : p.hd_idx0;
    const int32_t* __restrict__ ld_new = sc->ld_cur ? p.ld_idx0 : p.ld_idx1;
    const float invZ = static_cast<float>(1.0 / sc->Zhat);
    const uint32_t N = static_cast<uint32_t>(p.N);
    const int k_hd = p.k_hd, k_ld = p.k_ld;
    const float* __restrict__ Y = p.Y;
    const float alpha = p.alpha, inv_alpha = p.inv_alpha;
    const int gq = lane / G;          // row slot of this lane within a pass
    const int co = CW * (lane % G);   // first component owned by this lane

    double z_acc = 0.0;
    const int64_t tw = static_cast<int64_t>(gridDim.x) * kWarpsPerBlock;
    for (int64_t gi = static_cast<int64_t>(blockIdx.x) * kWarpsPerBlock + wib; gi < p.N; gi += tw) {
        const uint32_t i = static_cast<uint32_t>(gi);
        uint32_t nh[RH];
        float pv[RH];
#pragma unroll
        for (int r = 0; r < RH; ++r) {
            const int e = r * 32 + lane;
            nh[r] = e < k_hd ? FSNE_IDX(static_cast<uint32_t>(__ldg(hd_new + gi * k_hd + e)), N, i, &p.sc->err)
                             : 0xffffffffu;
            pv[r] = e < k_hd ? p.P[gi * k_hd + e] : 0.f;
        }
        const uint32_t nl =
            lane < k_ld ? FSNE_IDX(static_cast<uint32_t>(__ldg(ld_new + gi * k_ld + lane)), N, i, &p.sc->err)
                        : 0xffffffffu;
        float yi[CW];
        load_chunk<CW>(Y + gi * DP + co, yi);
        const uint4 wq = philox(t, i, kStreamRefine, static_cast<uint32_t>(lane), p.pk);
        // S_i = HD u LD lists of t+1 as a warp hash set
        hset_clear<kForceHashSlots>(tab, lane);
        __syncwarp();
#pragma unroll
        for (int r = 0; r < RH; ++r)
            if (r * 32 + lane < k_hd) hset_insert<kForceHashSlots>(tab, nh[r]);
        __syncwarp();
        const bool ld_in_hd = lane < k_ld && hset_has<kForceHashSlots>(tab, nl);
        __syncwarp();
        if (lane < k_ld) hset_insert<kForceHashSlots>(tab, nl);
        __syncwarp();

        // this lane's components as pairs (packed arithmetic)
        constexpr int CH = CW / 2;
        float2 yi2[CH], att[CH], rep[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            yi2[c] = make_float2(yi[2 * c], yi[2 * c + 1]);
            att[c] = make_float2(0.f, 0.f);
            rep[c] = make_float2(0.f, 0.f);
        }
        float z = 0.f;
        // One interaction per row group: w, w^{1/alpha} and this lane's
        // components of y_i - y_j. Every lane of the warp executes it (the
        // group reduction is a warp shuffle); lanes with on == false read no
        // row and contribute nothing.
        auto interact = [&](uint32_t j, bool on, float2 (&dy)[CH], float& w, float& winv) {
            float yj[CW];
            if (on) {
                load_chunk<CW>(Y + static_cast<int64_t>(j) * DP + co, yj);
            } else {
#pragma unroll
                for (int c = 0; c < CW; ++c) yj[c] = yi[c];
            }
            float2 r2v = make_float2(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                dy[c] = sub2(yi2[c], make_float2(yj[2 * c], yj[2 * c + 1]));
                r2v = fma2(dy[c], dy[c], r2v);
            }
            const float r2 = group_sum<G>(hsum2(r2v));
            winv = on ? __fdividef(1.f, __fmaf_rn(r2, inv_alpha, 1.f)) : 0.f;
            w = (alpha == 1.f || !on) ? winv : exp2f(alpha * __log2f(winv));
        };
        // HD neighbours: attraction (both directions of p_ij) and repulsion
        for (int b = 0; b < k_hd; b += R) {
            const int e = b + gq;
            const uint32_t j = warp_get<RH>(nh, static_cast<uint32_t>(e));
            const float pe = warp_get<RH>(pv, static_cast<uint32_t>(e));
            const bool on = e < k_hd;
            float2 dy[CH];
            float w, winv;
            interact(j, on, dy, w, winv);
            const float fa = 4.f * pe * p.inv2N * winv;
            const float fr = 4.f * w * invZ * winv;
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                att[c] = fma2(bcast2(fa), dy[c], att[c]);
                rep[c] = fma2(bcast2(fr), dy[c], rep[c]);
            }
            if (lane % G == 0) z += w;
            if (on) atomic_add_chunk<CW>(p.A + static_cast<int64_t>(j) * DP + co, dy, -fa);
        }
        // LD neighbours outside the HD list: repulsion (an entry that is in
        // the HD list travels as kNoRow: one shuffle a row)
        const uint32_t nl_rep = (lane < k_ld && !ld_in_hd) ? nl : kNoRow;
        for (int b = 0; b < k_ld; b += R) {
            const int l = b + gq;
            const uint32_t j = __shfl_sync(kFull, nl_rep, l & 31);
            const bool on = l < k_ld && j != kNoRow;
            float2 dy[CH];
            float w, winv;
            interact(j, on, dy, w, winv);
            const float fr = 4.f * w * invZ * winv;
#pragma unroll
            for (int c = 0; c < CH; ++c) rep[c] = fma2(bcast2(fr), dy[c], rep[c]);
            if (lane % G == 0) z += w;
        }
        // Philox-seeded negatives outside S_i, scaled by (N-1)/n_neg: lane l
        // draws and checks negative s0 + l of each block of 32 once (from its
        // own Philox words), and the passes fetch them by one shuffle a row
        for (int s0 = 0; s0 < p.n_neg; s0 += 32) {
            const uint32_t jn = map_other(negative_word(wq.y, wq.w, static_cast<uint32_t>(s0 >> 5)), N, i);
            const uint32_t jneg = (s0 + lane < p.n_neg && !hset_has<kForceHashSlots>(tab, jn)) ? jn : kNoRow;
            const int cnt = min(32, p.n_neg - s0);
            for (int b = 0; b < cnt; b += R) {
                const int e = b + gq;
                const uint32_t j = __shfl_sync(kFull, jneg, e & 31);
                const bool on = e < cnt && j != kNoRow;
                float2 dy[CH];
                float w, winv;
                interact(j, on, dy, w, winv);
                const float fr = p.neg_scale * 4.f * w * invZ * winv;
#pragma unroll
                for (int c = 0; c < CH; ++c) rep[c] = fma2(bcast2(fr), dy[c], rep[c]);
                if (lane % G == 0) z = __fmaf_rn(p.neg_scale, w, z);
            }
        }
        // sum over the row groups, scattered: each lane ends with C elements
        // of (A_i, R_i) restricted to its components, which it adds to A_i
        // (the reverse attraction of other points lands there too) or stores
        // into R_i
        constexpr int V = 2 * CW;
        float v[V];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            v[2 * c] = att[c].x;
            v[2 * c + 1] = att[c].y;
            v[CW + 2 * c] = rep[c].x;
            v[CW + 2 * c + 1] = rep[c].y;
        }
        int base = 0;
        bool owner = true;
        reduce_scatter_stages<V, V, 16, G>(v, lane, base, owner);
        if (owner) {
#pragma unroll
            for (int q = 0; q < scatter_count<V, G>(); ++q) {
                const int e = base + q;
                if (e < CW)
                    atomicAdd(p.A + gi * DP + co + e, v[q]);
                else
                    p.R[gi * DP + co + e - CW] = v[q];
            }
        }
        z = warp_sum(z);
        z_acc += static_cast<double>(z);
        __syncwarp();
    }
    if (lane == 0) s_z[wib] = z_acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double zb = 0.0;
        for (int v = 0; v < kWarpsPerBlock; ++v) zb += s_z[v];
        p.zpart[blockIdx.x] = zb;
    }
}

// ------------------------------------------------------------------ forces, row-pair layout
// The same forces as forces_kernel, laid out for the L1 data pipe, which
// bounds this kernel: every gathered LD row (DP floats) is read by G = DP/4
// lanes with one 16-byte load each, so one warp load touches R1 = 32/G whole
// rows (one cache-line wavefront per row instead of one per 16-byte column
// of a row), and each lane takes two rows per pass (slots m = 0, 1 at rows
// b + m R1 + lane/G), which keeps the rows per pass of the two-lane split.
// The repulsion-only rows (LD neighbours outside the HD list, then the
// negatives outside S_i) are appended to a per-warp queue in shared memory
// as they are found and consumed R rows at a time, so slots that contribute
// nothing cost no pass.
template <int DP>
struct PairSplit {
    static constexpr int G = DP / 4;    // lanes per row, one float4 each
    static constexpr int R1 = 32 / G;   // rows per warp load
    static constexpr int R = 2 * R1;    // rows per pass (two slots per lane)
};

template <int DP, int RH>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 4)
forces_pair_kernel(const StepParams p) {
    using S = PairSplit<DP>;
    constexpr int G = S::G, R1 = S::R1, R = S::R;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    uint32_t* tab = reinterpret_cast<uint32_t*>(smem) + wib * (kForceHashSlots + kRepRing);
    uint32_t* ring = tab + kForceHashSlots;
    __shared__ double s_z[kWarpsPerBlock];

    const DevScalars* sc = p.sc;
    const uint32_t t = sc->t;
    const bool fire = hd_coin(t, sc->E, p.seed, p.hd_mode, p.coin_p0, p.coin_p1);
    // lists of iteration t+1: the HD buffer flips only when the coin fired
    // (the rows of an insertion window refined alone were copied back into
    // the current buffer by fresh_lists_kernel)
    const int32_t* __restrict__ hd_new = (sc->hd_cur ^ (fire ? 1 : 0)) ? p.hd_idx1 : p.hd_idx0;
    const int32_t* __restrict__ ld_new = sc->ld_cur ? p.ld_idx0 : p.ld_idx1;
    const float invZ = static_cast<float>(1.0 / sc->Zhat);
    const uint32_t N = static_cast<uint32_t>(p.N);
    const int k_hd = p.k_hd, k_ld = p.k_ld;
    const float* __restrict__ Y = p.Y;
    const float alpha = p.alpha, inv_alpha = p.inv_alpha;
    const int gq = lane / G;          // row slot of this lane within a warp load
    const int co = 4 * (lane % G);    // first component owned by this lane
    const bool leader = (lane % G) == 0;
    const unsigned lt_mask = (1u << lane) - 1u;

    double z_acc = 0.0;
    const int64_t tw = static_cast<int64_t>(gridDim.x) * kWarpsPerBlock;
    for (int64_t gi = static_cast<int64_t>(blockIdx.x) * kWarpsPerBlock + wib; gi < p.N; gi += tw) {
        const uint32_t i = static_cast<uint32_t>(gi);
        uint32_t nh[RH];
        float pv[RH];
#pragma unroll
        for (int r = 0; r < RH; ++r) {
            const int e = r * 32 + lane;
            nh[r] = e < k_hd ? FSNE_IDX(static_cast<uint32_t>(__ldg(hd_new + gi * k_hd + e)), N, i, &p.sc->err)
                             : 0xffffffffu;
            pv[r] = e < k_hd ? p.P[gi * k_hd + e] : 0.f;
        }
        const uint32_t nl =
            lane < k_ld ? FSNE_IDX(static_cast<uint32_t>(__ldg(ld_new + gi * k_ld + lane)), N, i, &p.sc->err)
                        : 0xffffffffu;
        const float4 yi = __ldg(reinterpret_cast<const float4*>(Y + gi * DP + co));
        const uint4 wq = philox(t, i, kStreamRefine, static_cast<uint32_t>(lane), p.pk);
        // S_i = HD u LD lists of t+1 as a warp hash set
        hset_clear<kForceHashSlots>(tab, lane);
        __syncwarp();
#pragma unroll
        for (int r = 0; r < RH; ++r)
            if (r * 32 + lane < k_hd) hset_insert<kForceHashSlots>(tab, nh[r]);
        __syncwarp();
        const bool ld_in_hd = lane < k_ld && hset_has<kForceHashSlots>(tab, nl);
        __syncwarp();
        if (lane < k_ld) hset_insert<kForceHashSlots>(tab, nl);

        // this lane's four components as two pairs (packed arithmetic)
        float2 att[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        float2 rep[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        float z = 0.f;
        // Two rows per lane: r2, w and w^{1/alpha} of rows j[0], j[1]
        // (kNoRow: no row, contributes nothing) and this lane's components
        // of y_i - y_j. Every lane executes it (group reductions are shuffles).
        auto interact2 = [&](const uint32_t (&j)[2], float2 (&dy)[2][2], float (&w)[2], float (&winv)[2]) {
            float4 yj[2];
#pragma unroll
            for (int m = 0; m < 2; ++m)
                yj[m] = j[m] != kNoRow ? __ldg(reinterpret_cast<const float4*>(Y + static_cast<int64_t>(j[m]) * DP + co))
                                       : yi;
            float r2[2];
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                dy[m][0] = sub2(make_float2(yi.x, yi.y), make_float2(yj[m].x, yj[m].y));
                dy[m][1] = sub2(make_float2(yi.z, yi.w), make_float2(yj[m].z, yj[m].w));
                r2[m] = hsum2(fma2(dy[m][1], dy[m][1], mul2(dy[m][0], dy[m][0])));
            }
#pragma unroll
            for (int q = 1; q < G; q <<= 1) {
                r2[0] += __shfl_xor_sync(kFull, r2[0], q);
                r2[1] += __shfl_xor_sync(kFull, r2[1], q);
            }
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const bool on = j[m] != kNoRow;
                winv[m] = on ? __fdividef(1.f, __fmaf_rn(r2[m], inv_alpha, 1.f)) : 0.f;
                w[m] = (alpha == 1.f || !on) ? winv[m] : exp2f(alpha * __log2f(winv[m]));
            }
        };
        // HD neighbours: attraction (both directions of p_ij) and repulsion
        for (int b = 0; b < k_hd; b += R) {
            uint32_t j[2];
            float pe[2];
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const int e = b + m * R1 + gq;
                const uint32_t jj = warp_get<RH>(nh, static_cast<uint32_t>(e));
                pe[m] = warp_get<RH>(pv, static_cast<uint32_t>(e));
                j[m] = e < k_hd ? jj : kNoRow;
            }
            float2 dy[2][2];
            float w[2], winv[2];
            interact2(j, dy, w, winv);
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const float fa = 4.f * pe[m] * p.inv2N * winv[m];
                const float fr = 4.f * w[m] * invZ * winv[m];
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    att[c] = fma2(bcast2(fa), dy[m][c], att[c]);
                    rep[c] = fma2(bcast2(fr), dy[m][c], rep[c]);
                }
                if (leader) z += w[m];
                if (j[m] != kNoRow) {
                    const float2 a = mul2(bcast2(-fa), dy[m][0]), b = mul2(bcast2(-fa), dy[m][1]);
                    atomicAdd(reinterpret_cast<float4*>(p.A + static_cast<int64_t>(j[m]) * DP + co),
                              make_float4(a.x, a.y, b.x, b.y));
                }
            }
        }
        // repulsion-only rows through the queue: positions [head, tail) of
        // the stream (LD rows outside the HD list first, nld of them, then
        // the negatives outside S_i scaled by (N-1)/n_neg)
        int head = 0, tail = 0, nld = 0;
        auto consume = [&](bool last) {
            while (tail - head >= R || (last && tail > head)) {
                __syncwarp();
                uint32_t j[2];
                float scl[2];
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    const int pos = head + m * R1 + gq;
                    j[m] = pos < tail ? ring[pos & (kRepRing - 1)] : kNoRow;
                    scl[m] = pos < nld ? 1.f : p.neg_scale;
                }
                float2 dy[2][2];
                float w[2], winv[2];
                interact2(j, dy, w, winv);
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    const float fr = scl[m] * 4.f * w[m] * invZ * winv[m];
#pragma unroll
                    for (int c = 0; c < 2; ++c) rep[c] = fma2(bcast2(fr), dy[m][c], rep[c]);
                    if (leader) z = __fmaf_rn(scl[m], w[m], z);
                }
                head = min(head + R, tail);
            }
        };
        {
            const bool keep = lane < k_ld && !ld_in_hd;
            const unsigned mk = __ballot_sync(kFull, keep);
            if (keep) ring[(tail + __popc(mk & lt_mask)) & (kRepRing - 1)] = nl;
            tail += __popc(mk);
            nld = tail;
        }
        __syncwarp();
        for (int s0 = 0; s0 < p.n_neg; s0 += 32) {
            consume(false);
            const int sidx = s0 + lane;
            const uint32_t j = map_other(negative_word(wq.y, wq.w, static_cast<uint32_t>(s0 >> 5)), N, i);
            const bool on = sidx < p.n_neg && !hset_has<kForceHashSlots>(tab, j);
            const unsigned mk = __ballot_sync(kFull, on);
            if (on) ring[(tail + __popc(mk & lt_mask)) & (kRepRing - 1)] = j;
            tail += __popc(mk);
        }
        consume(true);
        // sum over the row groups, scattered over the lanes that share lane
        // mod G: each lane ends with elements of (A_i, R_i) restricted to its
        // components, which it adds to A_i or stores into R_i
        float v[8] = {att[0].x, att[0].y, att[1].x, att[1].y, rep[0].x, rep[0].y, rep[1].x, rep[1].y};
        int base = 0;
        bool owner = true;
        reduce_scatter_stages<8, 8, 16, G>(v, lane, base, owner);
        if (owner) {
#pragma unroll
            for (int q = 0; q < scatter_count<8, G>(); ++q) {
                const int e = base + q;
                if (e < 4)
                    atomicAdd(p.A + gi * DP + co + e, v[q]);
                else
                    p.R[gi * DP + co + e - 4] = v[q];
            }
        }
        z = warp_sum(z);
        z_acc += static_cast<double>(z);
        __syncwarp();
    }
    if (lane == 0) s_z[wib] = z_acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double zb = 0.0;
        for (int v = 0; v < kWarpsPerBlock; ++v) zb += s_z[v];
        p.zpart[blockIdx.x] = zb;
    }
}

}  // namespace fsne
