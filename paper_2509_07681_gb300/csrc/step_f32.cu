// Phase kernels: HD refinement with FP32 rows, LD refinement and forces for
// every LD row width, and the LD distance read-out.
#include "phase_instances.cuh"

namespace fsne {

cudaError_t hd_refine_launch_f32(const StepParams& p, int RH, int G, int blocks, size_t smem, cudaStream_t s) {
    return hd_refine_launch_xm<0>(p, RH, G, blocks, smem, s);
}
int hd_refine_occupancy_f32(int RH, int G, bool pf, size_t smem) { return hd_refine_occupancy_xm<0>(RH, G, pf, smem); }

#define FSNE_DP_RH(X)                                                                           \
    X(2, 1) X(4, 1) X(8, 1) X(16, 1) X(32, 1) X(2, 2) X(4, 2) X(8, 2) X(16, 2) X(32, 2)

// The row-pair layout of the LD distances (rows of 8, 16 or 32 floats).
#define FSNE_PAIR_DP_RH(X) X(8, 1) X(16, 1) X(32, 1) X(8, 2) X(16, 2) X(32, 2)

cudaError_t ld_refine_launch(const StepParams& p, int DP, int RH, bool pair, int blocks, size_t smem, cudaStream_t s) {
#define FSNE_CASE2(dp, rh, pr)                                                                  \
    if (DP == dp && RH == rh && pair == pr) {                                                   \
        FSNE_SET_SMEM((ld_refine_kernel<dp, rh, pr>), smem);                                    \
        ld_refine_kernel<dp, rh, pr><<<blocks, kWarpsPerBlock * 32, smem, s>>>(p);              \
        return cudaGetLastError();                                                              \
    }
#define FSNE_CASE(dp, rh) FSNE_CASE2(dp, rh, false)
#define FSNE_CASE_P(dp, rh) FSNE_CASE2(dp, rh, true)
    FSNE_DP_RH(FSNE_CASE)
    FSNE_PAIR_DP_RH(FSNE_CASE_P)
#undef FSNE_CASE_P
#undef FSNE_CASE
#undef FSNE_CASE2
    return cudaErrorInvalidValue;
}

// Lanes per LD row in the forces kernel: cw floats per lane (4, 8 or 16).
#define FSNE_FORCES_CW(X, dp, rh) X(dp, rh, 4) X(dp, rh, 8) X(dp, rh, 16)

cudaError_t forces_launch(const StepParams& p, int DP, int RH, int CW, int blocks, size_t smem, cudaStream_t s) {
#define FSNE_CASE3(dp, rh, cw)                                                                  \
    if (DP == dp && RH == rh && (CW == cw || (cw == 4 && dp < CW))) {                           \
        FSNE_SET_SMEM((forces_kernel<dp, rh, cw>), smem);                                       \
        forces_kernel<dp, rh, cw><<<blocks, kWarpsPerBlock * 32, smem, s>>>(p);                 \
        return cudaGetLastError();                                                              \
    }
#define FSNE_CASE(dp, rh) FSNE_FORCES_CW(FSNE_CASE3, dp, rh)
    FSNE_DP_RH(FSNE_CASE)
#undef FSNE_CASE
#undef FSNE_CASE3
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ insertion window
// In an iteration whose coin did not fire but an insertion window is open,
// hd_refine_kernel wrote the window's new HD lists (rows fresh_lo .. N-1) to
// the other buffer. Once the LD refinement (which reads the lists of t) is
// done, this copies them into the current buffer, where the forces and the
// next iteration read them. Any other iteration: returns at once.
__global__ void __launch_bounds__(256) fresh_lists_kernel(const StepParams p) {
    const DevScalars* sc = p.sc;
    const uint32_t t = sc->t;
    const bool fire = hd_coin(t, sc->E, p.seed, p.hd_mode, p.coin_p0, p.coin_p1);
    if (!fresh_only(sc, t, fire, p.N)) return;
    const int cur = sc->hd_cur;
    int32_t* __restrict__ idx_c = cur ? p.hd_idx1 : p.hd_idx0;
    const int32_t* __restrict__ idx_o = cur ? p.hd_idx0 : p.hd_idx1;
    float* __restrict__ d2_c = cur ? p.hd_d21 : p.hd_d20;
    const float* __restrict__ d2_o = cur ? p.hd_d20 : p.hd_d21;
    const int64_t hi = p.N * p.k_hd;
    for (int64_t e = sc->fresh_lo * p.k_hd + static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < hi;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        idx_c[e] = idx_o[e];
        d2_c[e] = d2_o[e];
    }
}

cudaError_t fresh_lists_launch(const StepParams& p, int blocks, cudaStream_t s) {
    fresh_lists_kernel<<<blocks, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t forces_pair_launch(const StepParams& p, int DP, int RH, int blocks, size_t smem, cudaStream_t s) {
#define FSNE_CASE(dp, rh)                                                                       \
    if (DP == dp && RH == rh) {                                                                 \
        FSNE_SET_SMEM((forces_pair_kernel<dp, rh>), smem);                                      \
        forces_pair_kernel<dp, rh><<<blocks, kWarpsPerBlock * 32, smem, s>>>(p);                \
        return cudaGetLastError();                                                              \
    }
    FSNE_PAIR_DP_RH(FSNE_CASE)
#undef FSNE_CASE
    return cudaErrorInvalidValue;
}

int forces_pair_occupancy(int DP, int RH, size_t smem) {
    int n = 0;
#define FSNE_CASE(dp, rh)                                                                       \
    if (DP == dp && RH == rh) {                                                                 \
        FSNE_SET_SMEM((forces_pair_kernel<dp, rh>), smem);                                      \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, forces_pair_kernel<dp, rh>, kWarpsPerBlock * 32, smem); \
    }
    FSNE_PAIR_DP_RH(FSNE_CASE)
#undef FSNE_CASE
    return n;
}

int ld_refine_occupancy(int DP, int RH, bool pair, size_t smem) {
    int n = 0;
#define FSNE_CASE2(dp, rh, pr)                                                                  \
    if (DP == dp && RH == rh && pair == pr) {                                                   \
        FSNE_SET_SMEM((ld_refine_kernel<dp, rh, pr>), smem);                                    \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, ld_refine_kernel<dp, rh, pr>, kWarpsPerBlock * 32, smem); \
    }
#define FSNE_CASE(dp, rh) FSNE_CASE2(dp, rh, false)
#define FSNE_CASE_P(dp, rh) FSNE_CASE2(dp, rh, true)
    FSNE_DP_RH(FSNE_CASE)
    FSNE_PAIR_DP_RH(FSNE_CASE_P)
#undef FSNE_CASE_P
#undef FSNE_CASE
#undef FSNE_CASE2
    return n;
}

int forces_occupancy(int DP, int RH, int CW, size_t smem) {
    int n = 0;
#define FSNE_CASE3(dp, rh, cw)                                                                  \
    if (DP == dp && RH == rh && (CW == cw || (cw == 4 && dp < CW))) {                           \
        FSNE_SET_SMEM((forces_kernel<dp, rh, cw>), smem);                                       \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, forces_kernel<dp, rh, cw>, kWarpsPerBlock * 32, smem); \
        return n;                                                                               \
    }
#define FSNE_CASE(dp, rh) FSNE_FORCES_CW(FSNE_CASE3, dp, rh)
    FSNE_DP_RH(FSNE_CASE)
#undef FSNE_CASE
#undef FSNE_CASE3
    return n;
}

// LD distances of the current LD lists (read-out only).
__global__ void ld_distances_kernel(const float* __restrict__ Y, const int32_t* __restrict__ idx, int64_t N,
                                    int k, int DP, float* d2) {
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= N * k) return;
    const int64_t i = e / k;
    const int64_t j = idx[e];
    float acc = 0.f;
    for (int c = 0; c < DP; ++c) {
        const float d = __fsub_rn(Y[i * DP + c], Y[j * DP + c]);
        acc = __fmaf_rn(d, d, acc);
    }
    d2[e] = acc;
}

cudaError_t launch_ld_distances(const float* Y, const int32_t* idx, int64_t N, int k, int DP, float* d2,
                                cudaStream_t s) {
    const int64_t n = N * k;
    ld_distances_kernel<<<static_cast<int>((n + 255) / 256), 256, 0, s>>>(Y, idx, N, k, DP, d2);
    return cudaGetLastError();
}

}  // namespace fsne
