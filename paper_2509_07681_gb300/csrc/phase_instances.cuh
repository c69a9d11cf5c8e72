// Dispatch of the phase kernels over the LD row width DP, the HD list width
// (RH registers of 32 entries) and the HD storage precision XM.
#pragma once

#include "launch.h"
#include "phase_kernels.cuh"

namespace fsne {

#define FSNE_SET_SMEM(kern, smem) \
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem))

template <int XM>
cudaError_t hd_refine_launch_xm(const StepParams& p, int RH, int blocks, size_t smem, cudaStream_t s) {
    if (RH == 1) {
        FSNE_SET_SMEM((hd_refine_kernel<1, XM>), smem);
        hd_refine_kernel<1, XM><<<blocks, kWarpsPerBlock * 32, smem, s>>>(p);
    } else {
        FSNE_SET_SMEM((hd_refine_kernel<2, XM>), smem);
        hd_refine_kernel<2, XM><<<blocks, kWarpsPerBlock * 32, smem, s>>>(p);
    }
    return cudaGetLastError();
}

template <int XM>
int hd_refine_occupancy_xm(int RH, size_t smem) {
    int n = 0;
    if (RH == 1) {
        FSNE_SET_SMEM((hd_refine_kernel<1, XM>), smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, hd_refine_kernel<1, XM>, kWarpsPerBlock * 32, smem);
    } else {
        FSNE_SET_SMEM((hd_refine_kernel<2, XM>), smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, hd_refine_kernel<2, XM>, kWarpsPerBlock * 32, smem);
    }
    return n;
}

}  // namespace fsne
