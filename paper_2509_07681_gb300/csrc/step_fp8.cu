// Fused step kernels with FP8-E4M3 row-scaled HD rows (FP32 re-rank at the
// list boundary).
#include "step_instances.cuh"

namespace fsne {

cudaError_t step_launch_fp8(const StepParams& p, int DP, int RH, int blocks, size_t smem, cudaStream_t s) {
    return step_launch_xm<2>(p, DP, RH, blocks, smem, s);
}
int step_occupancy_fp8(int DP, int RH, size_t smem) { return step_occupancy_xm<2>(DP, RH, smem); }

}  // namespace fsne
