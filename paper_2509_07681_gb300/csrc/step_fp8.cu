// HD refinement with FP8-E4M3 row-scaled rows (FP32 re-rank at the list
// boundary).
#include "phase_instances.cuh"

namespace fsne {

cudaError_t hd_refine_launch_fp8(const StepParams& p, int RH, int G, int blocks, size_t smem, cudaStream_t s) {
    return hd_refine_launch_xm<2>(p, RH, G, blocks, smem, s);
}
int hd_refine_occupancy_fp8(int RH, int G, bool pf, size_t smem) { return hd_refine_occupancy_xm<2>(RH, G, pf, smem); }

}  // namespace fsne
