// Fused step kernels with FP32 HD rows, and the LD distance read-out.
#include "step_instances.cuh"

namespace fsne {

cudaError_t step_launch_f32(const StepParams& p, int DP, int RH, int blocks, size_t smem, cudaStream_t s) {
    return step_launch_xm<0>(p, DP, RH, blocks, smem, s);
}
int step_occupancy_f32(int DP, int RH, size_t smem) { return step_occupancy_xm<0>(DP, RH, smem); }

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
