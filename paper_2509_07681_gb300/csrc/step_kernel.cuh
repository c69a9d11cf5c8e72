// The fused FUnc-SNE iteration kernel (one warp per point) and the update
// kernel. Included by one translation unit per HD storage precision.
//
// One iteration t, every point i in parallel (Jacobi: all reads see state t,
// all writes go to state t+1 buffers or accumulators):
//   HD refinement (Section 3) when the iteration's coin fires: 32 candidates
//     (see params.h), dedup against the list and self, FP32 distances (or
//     dequantised distances with an error band and an exact FP32 re-rank of
//     every candidate that can enter), warp bitonic top-k merge on
//     (d2, idx), new-neighbour flag, warm-restart bisection of beta_i (Eq. 1);
//   LD refinement (every iteration): 32 candidates, distances at Y_t of the
//     old list and the candidates, top-k_ld by (d2, idx);
//   forces (Eq. 5 split as Eq. 6) over the new lists at Y_t:
//     attraction 4 (p_{j|i}/2N) w^{1/alpha} (y_i - y_j) added to A_i and
//     subtracted from A_j; repulsion 4 (w_ij / Zhat_t) w^{1/alpha} (y_i - y_j)
//     over S_i = HD u LD and over n_neg Philox negatives outside S_i scaled
//     by (N-1)/n_neg; per-point Z_t terms summed per block in FP64.
// The update kernel (update_kernel.cu) then applies the forces.
#pragma once

#include "device_common.cuh"

namespace fsne {

constexpr int kWarpsPerBlock = 8;

// Resident blocks per SM the register budget is sized for (8 warps each).
template <int DP>
constexpr int step_min_blocks() { return DP >= 32 ? 2 : 3; }

template <int DP, int RH, int XM>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, step_min_blocks<DP>())
step_kernel(const StepParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    float* xs = reinterpret_cast<float*>(smem + wib * p.smem_per_warp);
    uint32_t* tab = reinterpret_cast<uint32_t*>(xs + p.xs_floats);  // warp hash set
    __shared__ double s_z[kWarpsPerBlock];
    __shared__ unsigned long long s_cnt[kWarpsPerBlock][3];

    const DevScalars* sc = p.sc;
    const uint32_t t = sc->t;
    const bool fire = hd_coin(t, sc->E, p.seed, p.hd_mode);
    const int hc = sc->hd_cur, lc = sc->ld_cur;
    const int32_t* __restrict__ hd_idx_c = hc ? p.hd_idx1 : p.hd_idx0;
    const float* __restrict__ hd_d2_c = hc ? p.hd_d21 : p.hd_d20;
    int32_t* __restrict__ hd_idx_n = hc ? p.hd_idx0 : p.hd_idx1;
    float* __restrict__ hd_d2_n = hc ? p.hd_d20 : p.hd_d21;
    const int32_t* __restrict__ ld_idx_c = lc ? p.ld_idx1 : p.ld_idx0;
    int32_t* __restrict__ ld_idx_n = lc ? p.ld_idx0 : p.ld_idx1;
    const float invZ = static_cast<float>(1.0 / sc->Zhat);
    const uint32_t N = static_cast<uint32_t>(p.N);
    const int k_hd = p.k_hd, k_ld = p.k_ld;
    const float* __restrict__ Y = p.Y;

    // own-row staging area beyond the FP32 row is read as zeros by the
    // BF16 / FP8 distance loops
    for (int f = p.xpitch + lane; f < p.xs_floats; f += 32) xs[f] = 0.f;
    __syncwarp();

    double z_acc = 0.0;
    unsigned long long c_new = 0, c_scored = 0, c_rerank = 0;

    const int64_t tw = static_cast<int64_t>(gridDim.x) * kWarpsPerBlock;
    for (int64_t gi = static_cast<int64_t>(blockIdx.x) * kWarpsPerBlock + wib; gi < p.N; gi += tw) {
        const uint32_t i = static_cast<uint32_t>(gi);
        // ---------------- state of iteration t
        uint32_t hidx[RH];
        float hd2[RH];
#pragma unroll
        for (int r = 0; r < RH; ++r) {
            const int e = r * 32 + lane;
            if (e < k_hd) {
                hidx[r] = static_cast<uint32_t>(__ldg(hd_idx_c + gi * k_hd + e));
                hd2[r] = __ldg(hd_d2_c + gi * k_hd + e);
            } else {
                hidx[r] = 0xffffffffu;
                hd2[r] = __uint_as_float(0x7f800000u);
            }
        }
        const uint32_t lidx = lane < k_ld ? static_cast<uint32_t>(__ldg(ld_idx_c + gi * k_ld + lane)) : 0xffffffffu;
        float yi[DP];
        load_row<DP>(Y + gi * DP, yi);

        // one Philox block per slot: words 0-1 drive the HD candidate, 2-3 the LD one
        const uint4 w = philox(t, i, kStreamRefine, static_cast<uint32_t>(lane), p.seed);

        // ---------------- HD refinement
        uint32_t nh_idx[RH];
        float nh_d2[RH];
        float pv[RH];
#pragma unroll
        for (int r = 0; r < RH; ++r) {
            nh_idx[r] = hidx[r];
            nh_d2[r] = hd2[r];
        }
        bool changed = false;
        if (fire) {
            const float* xrow = p.X32 + gi * p.xpitch;
            for (int f = lane * 4; f < p.xpitch; f += 128)
                *reinterpret_cast<float4*>(xs + f) = __ldg(reinterpret_cast<const float4*>(xrow + f));
            hset_clear(tab, lane);
            __syncwarp();
#pragma unroll
            for (int r = 0; r < RH; ++r)
                if (r * 32 + lane < k_hd) hset_insert(tab, hidx[r]);
            const uint32_t e0 = lane < kHdNnEnd ? map_index(w.x, k_hd) : map_index(w.x, k_ld);
            const uint32_t hv = warp_get<RH>(hidx, e0);
            const uint32_t lv = __shfl_sync(kFull, lidx, static_cast<int>(e0 & 31u));
            uint32_t c;
            if (lane < kHdNnEnd)
                c = static_cast<uint32_t>(__ldg(hd_idx_c + static_cast<int64_t>(hv) * k_hd + map_index(w.y, k_hd)));
            else if (lane < kHdLdNbEnd)
                c = lv;
            else if (lane < kHdLdNnEnd)
                c = static_cast<uint32_t>(__ldg(ld_idx_c + static_cast<int64_t>(lv) * k_ld + map_index(w.y, k_ld)));
            else
                c = map_other(w.x, N, i);
            __syncwarp();
            bool valid = (c != i) && (c < N) && !hset_has(tab, c);
            const unsigned same = __match_any_sync(kFull, c);
            valid &= (same & ((1u << lane) - 1u)) == 0u;

            uint64_t ck = kSentinel;
            if constexpr (XM == 0) {
                if (valid) ck = make_key(dist_f32(xs, p.X32 + static_cast<int64_t>(c) * p.xpitch, p.n4), c);
            } else {
                const int kl1 = k_hd - 1;
                const float thr = warp_get<RH>(hd2, static_cast<uint32_t>(kl1));
                bool need = false;
                if (valid) {
                    ApproxDist a;
                    if constexpr (XM == 1)
                        a = dist_bf16(xs, reinterpret_cast<const uint16_t*>(p.Xq + static_cast<int64_t>(c) * p.qpitch),
                                      p.nq, p.q_u, p.q_gamma);
                    else
                        a = dist_fp8(xs, p.Xq + static_cast<int64_t>(c) * p.qpitch, p.nq, p.qscale_off, p.q_u,
                                     p.q_a, p.q_gamma);  // nq = code words for FP8
                    need = __fsub_rd(a.d2, a.band) <= thr;
                    ++c_scored;
                }
                if (need) {
                    ++c_rerank;
                    ck = make_key(dist_f32(xs, p.X32 + static_cast<int64_t>(c) * p.xpitch, p.n4), c);
                }
            }
            // flag: some candidate precedes the old k-th entry
            uint64_t okeys[RH];
#pragma unroll
            for (int r = 0; r < RH; ++r)
                okeys[r] = (r * 32 + lane < k_hd) ? make_key(hd2[r], hidx[r]) : kSentinel;
            const uint64_t okth = [&] {
                const uint32_t e = static_cast<uint32_t>(k_hd - 1);
                uint64_t out = okeys[0];
#pragma unroll
                for (int r = 0; r < RH; ++r) {
                    const uint64_t x = shfl64(okeys[r], static_cast<int>(e & 31u));
                    if (static_cast<uint32_t>(r) == (e >> 5)) out = x;
                }
                return out;
            }();
            changed = __any_sync(kFull, ck < okth);
            if (changed) {
                merge_candidates<RH>(okeys, ck, lane);
#pragma unroll
                for (int r = 0; r < RH; ++r) {
                    nh_idx[r] = key_idx(okeys[r]);
                    nh_d2[r] = key_d2(okeys[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < RH; ++r) {
                const int e = r * 32 + lane;
                if (e < k_hd) {
                    hd_idx_n[gi * k_hd + e] = static_cast<int32_t>(nh_idx[r]);
                    hd_d2_n[gi * k_hd + e] = nh_d2[r];
                }
            }
            if (changed) {
                const float b = warp_bisect<RH>(nh_d2, k_hd, p.log_perp, p.beta[gi], pv, lane);
#pragma unroll
                for (int r = 0; r < RH; ++r) {
                    const int e = r * 32 + lane;
                    if (e < k_hd) p.P[gi * k_hd + e] = pv[r];
                }
                if (lane == 0) p.beta[gi] = b;
                ++c_new;
            }
        }
        if (!changed) {
#pragma unroll
            for (int r = 0; r < RH; ++r) {
                const int e = r * 32 + lane;
                pv[r] = e < k_hd ? p.P[gi * k_hd + e] : 0.f;
            }
        }

        // ---------------- LD refinement (candidates from the lists of iteration t)
        uint32_t nl;
        {
            __syncwarp();
            hset_clear(tab, lane);
            __syncwarp();
            if (lane < k_ld) hset_insert(tab, lidx);
            const uint32_t e0 = lane < kLdNnEnd ? map_index(w.z, k_ld) : map_index(w.z, k_hd);
            const uint32_t lv = __shfl_sync(kFull, lidx, static_cast<int>(e0 & 31u));
            const uint32_t hv = warp_get<RH>(hidx, e0);
            uint32_t c;
            if (lane < kLdNnEnd)
                c = static_cast<uint32_t>(__ldg(ld_idx_c + static_cast<int64_t>(lv) * k_ld + map_index(w.w, k_ld)));
            else if (lane < kLdHdNbEnd)
                c = hv;
            else
                c = map_other(w.z, N, i);
            __syncwarp();
            bool valid = (c != i) && (c < N) && !hset_has(tab, c);
            const unsigned same = __match_any_sync(kFull, c);
            valid &= (same & ((1u << lane) - 1u)) == 0u;
            uint64_t k2[2] = {kSentinel, kSentinel};
            if (lane < k_ld) {
                float yo[DP];
                load_row<DP>(Y + static_cast<int64_t>(lidx) * DP, yo);
                k2[0] = make_key(sqdist_ld<DP>(yi, yo), lidx);
            }
            if (valid) {
                float yc[DP];
                load_row<DP>(Y + static_cast<int64_t>(c) * DP, yc);
                k2[1] = make_key(sqdist_ld<DP>(yi, yc), c);
            }
            warp_sort<2>(k2, lane);
            nl = key_idx(k2[0]);
            if (lane < k_ld) ld_idx_n[gi * k_ld + lane] = static_cast<int32_t>(nl);
        }

        // ---------------- forces over the new lists at Y_t
        // S_i = HD u LD lists of iteration t+1, as a warp hash set
        __syncwarp();
        hset_clear(tab, lane);
        __syncwarp();
#pragma unroll
        for (int r = 0; r < RH; ++r)
            if (r * 32 + lane < k_hd) hset_insert(tab, nh_idx[r]);
        __syncwarp();
        const bool ld_in_hd = lane < k_ld && hset_has(tab, nl);
        __syncwarp();
        if (lane < k_ld) hset_insert(tab, nl);
        __syncwarp();

        // attraction components in acc[0..DP), repulsion in acc[RO..RO+DP)
        constexpr int RO = DP <= 16 ? 16 : DP;
        constexpr int NACC = DP <= 4 ? RO + DP : 2 * RO;
        float acc[NACC];
#pragma unroll
        for (int c = 0; c < NACC; ++c) acc[c] = 0.f;
        float z = 0.f;
        const float alpha = p.alpha, inv_alpha = p.inv_alpha;
        auto interact = [&](const float (&yj)[DP], float& w_out, float& winv_out, float (&dy)[DP]) {
            float r2 = 0.f;
#pragma unroll
            for (int c = 0; c < DP; ++c) {
                dy[c] = __fsub_rn(yi[c], yj[c]);
                r2 = __fmaf_rn(dy[c], dy[c], r2);
            }
            const float winv = 1.f / __fmaf_rn(r2, inv_alpha, 1.f);
            winv_out = winv;
            w_out = alpha == 1.f ? winv : powf(winv, alpha);
        };
#pragma unroll
        for (int r = 0; r < RH; ++r) {
            const int e = r * 32 + lane;
            if (e < k_hd) {
                const uint32_t j = nh_idx[r];
                float yj[DP], dy[DP], w, winv;
                load_row<DP>(Y + static_cast<int64_t>(j) * DP, yj);
                interact(yj, w, winv, dy);
                const float fa = 4.f * pv[r] * p.inv2N * winv;
                const float fr = 4.f * w * invZ * winv;
#pragma unroll
                for (int c = 0; c < DP; ++c) {
                    acc[c] = __fmaf_rn(fa, dy[c], acc[c]);
                    acc[RO + c] = __fmaf_rn(fr, dy[c], acc[RO + c]);
                }
                z += w;
                atomic_add_row<DP>(p.A + static_cast<int64_t>(j) * DP, dy, -fa);
            }
        }
        if (lane < k_ld) {
            if (!ld_in_hd) {
                float yj[DP], dy[DP], w, winv;
                load_row<DP>(Y + static_cast<int64_t>(nl) * DP, yj);
                interact(yj, w, winv, dy);
                const float fr = 4.f * w * invZ * winv;
#pragma unroll
                for (int c = 0; c < DP; ++c) acc[RO + c] = __fmaf_rn(fr, dy[c], acc[RO + c]);
                z += w;
            }
        }
        for (int s = lane; s < p.n_neg; s += 32) {
            const uint4 w4 = philox(t, i, kStreamNeg, static_cast<uint32_t>(s), p.seed);
            const uint32_t j = map_other(w4.x, N, i);
            if (!hset_has(tab, j)) {
                float yj[DP], dy[DP], w, winv;
                load_row<DP>(Y + static_cast<int64_t>(j) * DP, yj);
                interact(yj, w, winv, dy);
                const float fr = p.neg_scale * 4.f * w * invZ * winv;
#pragma unroll
                for (int c = 0; c < DP; ++c) acc[RO + c] = __fmaf_rn(fr, dy[c], acc[RO + c]);
                z = __fmaf_rn(p.neg_scale, w, z);
            }
        }
        // warp reductions: the lane owning component c adds A_i[c] and stores R_i[c]
        if constexpr (DP <= 4) {
#pragma unroll
            for (int c = 0; c < NACC; ++c) acc[c] = warp_sum(acc[c]);
            if (lane < DP) {
                float a = acc[0], b = acc[RO];
#pragma unroll
                for (int c = 1; c < DP; ++c)
                    if (lane == c) {
                        a = acc[c];
                        b = acc[RO + c];
                    }
                atomicAdd(p.A + gi * DP + lane, a);
                p.R[gi * DP + lane] = b;
            }
        } else if constexpr (DP == 32) {
            const float a = warp_reduce_scatter32<0>(acc, lane);
            const float b = warp_reduce_scatter32<32>(acc, lane);
            atomicAdd(p.A + gi * DP + lane, a);
            p.R[gi * DP + lane] = b;
        } else {
            const float v = warp_reduce_scatter32(acc, lane);
            const int c = lane & 15;
            if (c < DP) {
                if (lane < 16)
                    atomicAdd(p.A + gi * DP + c, v);
                else
                    p.R[gi * DP + c] = v;
            }
        }
        z = warp_sum(z);
        z_acc += static_cast<double>(z);
        __syncwarp();
    }

    if (lane == 0) {
        s_z[wib] = z_acc;
        s_cnt[wib][0] = c_new;
    }
    // candidate counters are per lane
    unsigned long long cs = c_scored, cr = c_rerank;
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
        cs += __shfl_xor_sync(kFull, cs, m);
        cr += __shfl_xor_sync(kFull, cr, m);
    }
    if (lane == 0) {
        s_cnt[wib][1] = cs;
        s_cnt[wib][2] = cr;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double zb = 0.0;
        unsigned long long a = 0, b = 0, c = 0;
        for (int w = 0; w < kWarpsPerBlock; ++w) {
            zb += s_z[w];
            a += s_cnt[w][0];
            b += s_cnt[w][1];
            c += s_cnt[w][2];
        }
        p.zpart[blockIdx.x] = zb;
        p.cnt[3 * blockIdx.x + 0] = a;
        p.cnt[3 * blockIdx.x + 1] = b;
        p.cnt[3 * blockIdx.x + 2] = c;
    }
}

}  // namespace fsne
