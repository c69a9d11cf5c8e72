// Update kernel of the FUnc-SNE iteration: applies the forces gathered by
// the step kernel and advances the device-resident scalars.
#include "device_common.cuh"
#include "launch.h"

namespace fsne {

// g = att * exag * A - rep * R; V = momentum V - lr g; Y += V; A = 0.
// The last block to finish advances the scalars of the iteration.
__global__ void __launch_bounds__(256) update_kernel(const UpdateParams u) {
    const DevScalars* sc = u.sc;
    const uint32_t t = sc->t;
    const float exag = (static_cast<int64_t>(t) < u.exag_iters) ? u.exaggeration : 1.f;
    const float ca = u.att * exag, cr = u.rep;
    const int64_t n4 = u.n_elem / 4;
    float4* Y = reinterpret_cast<float4*>(u.Y);
    float4* V = reinterpret_cast<float4*>(u.V);
    float4* A = reinterpret_cast<float4*>(u.A);
    const float4* R = reinterpret_cast<const float4*>(u.R);
    bool bad = false;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < n4;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float4 a = A[e], r = R[e];
        float4 v = V[e], y = Y[e];
        if (u.dbg_att) {
            reinterpret_cast<float4*>(u.dbg_att)[e] = a;
            reinterpret_cast<float4*>(u.dbg_rep)[e] = r;
        }
        v.x = u.momentum * v.x - u.lr * (ca * a.x - cr * r.x);
        v.y = u.momentum * v.y - u.lr * (ca * a.y - cr * r.y);
        v.z = u.momentum * v.z - u.lr * (ca * a.z - cr * r.z);
        v.w = u.momentum * v.w - u.lr * (ca * a.w - cr * r.w);
        y.x += v.x;
        y.y += v.y;
        y.z += v.z;
        y.w += v.w;
        bad |= !(isfinite(y.x) && isfinite(y.y) && isfinite(y.z) && isfinite(y.w));
        V[e] = v;
        Y[e] = y;
        A[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&u.sc->err, kErrNonFinite);
    // last-block detection (no waiting): the block taking the final ticket
    // sees every other block's reads of t done.
    __shared__ bool last;
    __threadfence();
    if (threadIdx.x == 0) last = (atomicAdd(&u.sc->ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    if (threadIdx.x < 32) {
        double z = 0.0;
        unsigned long long nn = 0, ns = 0, nr = 0;
        const DevScalars* s0 = u.sc;
        const bool fired = hd_coin(t, s0->E, u.seed, u.hd_mode, u.coin_p0, u.coin_p1);
        for (int b = threadIdx.x; b < u.n_zpart; b += 32) z += u.zpart[b];
        // the refinement kernel ran (and wrote its counters) when the coin
        // fired or the insertion window was refined alone
        if (fired || fresh_only(s0, t, fired, u.N))
            for (int b = threadIdx.x; b < u.n_cnt; b += 32) {
                nn += u.cnt[3 * b];
                ns += u.cnt[3 * b + 1];
                nr += u.cnt[3 * b + 2];
            }
        z = warp_sum_d(z);
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) {
            nn += __shfl_xor_sync(kFull, nn, m);
            ns += __shfl_xor_sync(kFull, ns, m);
            nr += __shfl_xor_sync(kFull, nr, m);
        }
        if (threadIdx.x == 0) {
            DevScalars* s = u.sc;
            const bool fire = hd_coin(t, s->E, u.seed, u.hd_mode, u.coin_p0, u.coin_p1);
            s->last_Z = z;
            s->Zhat = __dadd_rn(__dmul_rn(__dsub_rn(1.0, u.gamma_z), s->Zhat), __dmul_rn(u.gamma_z, z));
            if (fire) {
                const double frac = __ddiv_rn(static_cast<double>(nn), static_cast<double>(u.N));
                s->E = __dadd_rn(__dmul_rn(__dsub_rn(1.0, u.gamma_e), s->E), __dmul_rn(u.gamma_e, frac));
                s->hd_cur ^= 1;
                s->n_refined += 1;
            }
            s->ld_cur ^= 1;
            s->last_coin = fire ? 1 : 0;
            s->last_n_new = nn;
            s->cand_scored += ns;
            s->cand_reranked += nr;
            s->t = t + 1;
            s->ticket = 0;
        }
    }
}

cudaError_t update_launch(const UpdateParams& u, int blocks, cudaStream_t s) {
    update_kernel<<<blocks, 256, 0, s>>>(u);
    return cudaGetLastError();
}

}  // namespace fsne
