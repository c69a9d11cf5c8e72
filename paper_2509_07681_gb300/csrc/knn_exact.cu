// Exact k nearest neighbours by brute force (evaluation of neighbour recall,
// not part of the iteration). FP32 distances summed as in dist_f32, ties by index.
// Pass 1: block = 8 queries (one warp each) x one slice of the points; each
// warp keeps a sorted top-(32*RK) list and merges 32 scanned rows at a time.
// Pass 2: one warp per query merges the slices' lists.
#include "device_common.cuh"
#include "launch.h"

namespace fsne {

template <int RK>
__global__ void __launch_bounds__(256) knn_scan_kernel(const KnnParams kp) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float* xs = reinterpret_cast<float*>(smem) + wib * kp.xpitch;
    const int64_t qn = static_cast<int64_t>(blockIdx.x) * 8 + wib;
    if (qn >= kp.n_q) return;
    const int64_t q = kp.queries[qn];
    for (int f = lane * 4; f < kp.xpitch; f += 128)
        *reinterpret_cast<float4*>(xs + f) = __ldg(reinterpret_cast<const float4*>(kp.X32 + q * kp.xpitch + f));
    __syncwarp();
    const int64_t per = (kp.N + kp.n_split - 1) / kp.n_split;
    const int64_t j0 = static_cast<int64_t>(blockIdx.y) * per;
    const int64_t j1 = min(kp.N, j0 + per);
    uint64_t top[RK];
#pragma unroll
    for (int r = 0; r < RK; ++r) top[r] = kSentinel;
    const int last = 32 * RK - 1;
    for (int64_t base = j0; base < j1; base += 32) {
        const int64_t j = base + lane;
        uint64_t ck = kSentinel;
        if (j < j1 && j != q)
            ck = make_key(dist_f32(xs, kp.X32 + j * kp.xpitch, kp.n4), static_cast<uint32_t>(j));
        const uint64_t kth = shfl64(top[last >> 5], last & 31);
        if (__any_sync(kFull, ck < kth)) merge_candidates<RK>(top, ck, lane);
    }
    unsigned long long* out = kp.part + (qn * kp.n_split + blockIdx.y) * (32 * RK);
#pragma unroll
    for (int r = 0; r < RK; ++r) out[r * 32 + lane] = top[r];
}

template <int RK>
__global__ void __launch_bounds__(256) knn_merge_kernel(const KnnParams kp) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t qn = static_cast<int64_t>(blockIdx.x) * 8 + wib;
    if (qn >= kp.n_q) return;
    const unsigned long long* in = kp.part + qn * kp.n_split * (32 * RK);
    uint64_t top[RK];
#pragma unroll
    for (int r = 0; r < RK; ++r) top[r] = in[r * 32 + lane];
    const int last = 32 * RK - 1;
    for (int s = 1; s < kp.n_split; ++s)
        for (int r = 0; r < RK; ++r) {
            const uint64_t ck = in[(s * RK + r) * 32 + lane];
            const uint64_t kth = shfl64(top[last >> 5], last & 31);
            if (__any_sync(kFull, ck < kth)) merge_candidates<RK>(top, ck, lane);
        }
#pragma unroll
    for (int r = 0; r < RK; ++r) {
        const int e = r * 32 + lane;
        if (e < kp.k) {
            kp.idx[qn * kp.k + e] = static_cast<int32_t>(key_idx(top[r]));
            if (kp.d2) kp.d2[qn * kp.k + e] = key_d2(top[r]);
        }
    }
}

cudaError_t launch_exact_knn(const KnnParams& kp, cudaStream_t s) {
    const int qb = static_cast<int>((kp.n_q + 7) / 8);
    const dim3 grid(qb, kp.n_split);
    const size_t smem = static_cast<size_t>(8) * kp.xpitch * sizeof(float);
    if (kp.RK == 1) {
        cudaFuncSetAttribute(knn_scan_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        knn_scan_kernel<1><<<grid, 256, smem, s>>>(kp);
        knn_merge_kernel<1><<<qb, 256, 0, s>>>(kp);
    } else {
        cudaFuncSetAttribute(knn_scan_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        knn_scan_kernel<2><<<grid, 256, smem, s>>>(kp);
        knn_merge_kernel<2><<<qb, 256, 0, s>>>(kp);
    }
    return cudaGetLastError();
}

}  // namespace fsne
