// Dispatch of the phase kernels over the LD row width DP, the HD list width
// (RH registers of 32 entries) and the HD storage precision XM.
#pragma once

#include "launch.h"
#include "phase_kernels.cuh"

namespace fsne {

#define FSNE_SET_SMEM(kern, smem) \
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem))

// RH in {1, 2} (k_hd up to 32 or 64), G in {1, 2, 4, 8} lanes per gathered row.
#define FSNE_HD_CASES(X) X(1, 1) X(1, 2) X(1, 4) X(1, 8) X(2, 1) X(2, 2) X(2, 4) X(2, 8)

template <int XM>
cudaError_t hd_refine_launch_xm(const StepParams& p, int RH, int G, int blocks, size_t smem, cudaStream_t s) {
#define FSNE_CASE2(rh, g, pf)                                                           \
    if (RH == rh && G == g && (p.hd_prefetch != 0) == pf) {                             \
        FSNE_SET_SMEM((hd_refine_kernel<rh, XM, g, pf>), smem);                         \
        hd_refine_kernel<rh, XM, g, pf><<<blocks, kWarpsPerBlock * 32, smem, s>>>(p);   \
        return cudaGetLastError();                                                      \
    }
#define FSNE_CASE(rh, g) FSNE_CASE2(rh, g, false) FSNE_CASE2(rh, g, true)
    FSNE_HD_CASES(FSNE_CASE)
#undef FSNE_CASE
#undef FSNE_CASE2
    return cudaErrorInvalidValue;
}

template <int XM>
int hd_refine_occupancy_xm(int RH, int G, bool pf, size_t smem) {
    int n = 0;
#define FSNE_CASE2(rh, g, PF)                                                                      \
    if (RH == rh && G == g && pf == PF) {                                                          \
        FSNE_SET_SMEM((hd_refine_kernel<rh, XM, g, PF>), smem);                                    \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, hd_refine_kernel<rh, XM, g, PF>, kWarpsPerBlock * 32, smem); \
        return n;                                                                                  \
    }
#define FSNE_CASE(rh, g) FSNE_CASE2(rh, g, false) FSNE_CASE2(rh, g, true)
    FSNE_HD_CASES(FSNE_CASE)
#undef FSNE_CASE
#undef FSNE_CASE2
    return 0;
}

}  // namespace fsne
