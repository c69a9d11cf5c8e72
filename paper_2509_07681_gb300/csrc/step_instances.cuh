// Dispatch of the fused step kernel over the LD row width DP and the HD
// list width (RH registers of 32 entries) for one storage precision XM.
#pragma once

#include "launch.h"
#include "step_kernel.cuh"

namespace fsne {

template <int XM>
cudaError_t step_launch_xm(const StepParams& p, int DP, int RH, int blocks, size_t smem, cudaStream_t s) {
#define FSNE_CASE(dp, rh)                                                                              \
    if (DP == dp && RH == rh) {                                                                        \
        cudaFuncSetAttribute(step_kernel<dp, rh, XM>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                             static_cast<int>(smem));                                                  \
        step_kernel<dp, rh, XM><<<blocks, kWarpsPerBlock * 32, smem, s>>>(p);                          \
        return cudaGetLastError();                                                                     \
    }
    FSNE_CASE(2, 1) FSNE_CASE(4, 1) FSNE_CASE(8, 1) FSNE_CASE(16, 1) FSNE_CASE(32, 1)
    FSNE_CASE(2, 2) FSNE_CASE(4, 2) FSNE_CASE(8, 2) FSNE_CASE(16, 2) FSNE_CASE(32, 2)
#undef FSNE_CASE
    return cudaErrorInvalidValue;
}

template <int XM>
int step_occupancy_xm(int DP, int RH, size_t smem) {
    int n = 0;
#define FSNE_CASE(dp, rh)                                                                              \
    if (DP == dp && RH == rh) {                                                                        \
        cudaFuncSetAttribute(step_kernel<dp, rh, XM>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                             static_cast<int>(smem));                                                  \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<dp, rh, XM>, kWarpsPerBlock * 32, \
                                                      smem);                                           \
    }
    FSNE_CASE(2, 1) FSNE_CASE(4, 1) FSNE_CASE(8, 1) FSNE_CASE(16, 1) FSNE_CASE(32, 1)
    FSNE_CASE(2, 2) FSNE_CASE(4, 2) FSNE_CASE(8, 2) FSNE_CASE(16, 2) FSNE_CASE(32, 2)
#undef FSNE_CASE
    return n;
}

}  // namespace fsne
