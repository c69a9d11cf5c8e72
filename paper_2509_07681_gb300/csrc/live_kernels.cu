// Live changes of the point set: rows of X replaced (drift) and points
// removed. The paper lets points be added or removed while the iteration
// runs (Section 3); how a removal repairs the lists is this library's
// reading: the kept points keep their order and are renumbered, and every
// list entry that pointed to a removed point is replaced by a random other
// kept point not yet in the list.
#include "device_common.cuh"
#include "launch.h"

namespace fsne {

// dst[n, 0..pitch) = src[old[n], 0..pitch) for n < n_rows (4-byte words).
__global__ void gather_rows_kernel(uint32_t* __restrict__ dst, const uint32_t* __restrict__ src, int64_t pitch,
                                   const int32_t* __restrict__ old, int64_t n_rows) {
    const int64_t total = n_rows * pitch;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t n = e / pitch, c = e - n * pitch;
        dst[e] = src[static_cast<int64_t>(old[n]) * pitch + c];
    }
}

// dst[r, 0..cols) = src[r, 0..cols) (4-byte words): one warp per row, the
// lanes over the columns; the padding columns of dst are not touched.
__global__ void repack_rows_kernel(uint32_t* __restrict__ dst, int64_t dpitch, const uint32_t* __restrict__ src,
                                   int64_t spitch, int64_t rows, int64_t cols) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    for (int64_t r = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows;
         r += warps)
        for (int64_t c = lane; c < cols; c += 32) dst[r * dpitch + c] = src[r * spitch + c];
}

// X32[ids[r], 0..D) = rows[r, 0..D) (the padding columns stay zero).
__global__ void scatter_rows_kernel(float* __restrict__ X32, int xpitch, const int64_t* __restrict__ ids,
                                    const float* __restrict__ rows, int64_t n, int D) {
    const int64_t total = n * D;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = e / D, c = e - r * D;
        X32[ids[r] * xpitch + c] = rows[e];
    }
}

// One warp per list row of a kept point n (k <= 64 entries, two per lane at
// most): entries are renumbered through new_of (-1: the neighbour was
// removed); removed entries are replaced in slot order, slot e drawing
// j = map_other(w0, N, n) from counter (t, n, REMOVE, salt + e) and stepping
// to j + 1 (mod N, skipping n) while j is already in the row.
__global__ void remap_lists_kernel(int32_t* __restrict__ list, int k, const int32_t* __restrict__ new_of,
                                   int64_t N, uint32_t t, uint64_t seed, uint32_t salt) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    for (int64_t n = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); n < N;
         n += warps) {
        int32_t v[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int e = r * 32 + lane;
            v[r] = e < k ? new_of[list[n * k + e]] : INT32_MAX;
        }
        for (int r = 0; r < 2; ++r) {
            unsigned todo = __ballot_sync(kFull, v[r] < 0);
            while (todo) {
                const int src = __ffs(static_cast<int>(todo)) - 1;
                todo &= todo - 1u;
                const uint32_t e = static_cast<uint32_t>(r * 32 + src);
                const uint4 w = philox(t, static_cast<uint32_t>(n), kStreamRemove, salt + e, seed);
                uint32_t j = map_other(w.x, static_cast<uint32_t>(N), static_cast<uint32_t>(n));
                // at most k + 1 steps: the row holds fewer than k other points
                for (int step = 0; step <= k + 1; ++step) {
                    const bool taken = __any_sync(kFull, v[0] == static_cast<int32_t>(j) ||
                                                             v[1] == static_cast<int32_t>(j));
                    if (!taken) break;
                    j = static_cast<uint32_t>((static_cast<int64_t>(j) + 1) % N);
                    if (j == static_cast<uint32_t>(n)) j = static_cast<uint32_t>((static_cast<int64_t>(j) + 1) % N);
                }
                if (lane == src) v[r] = static_cast<int32_t>(j);
            }
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int e = r * 32 + lane;
            if (e < k) list[n * k + e] = v[r];
        }
    }
}

// Y and V scaled by one factor (the embedding's padding columns stay 0).
__global__ void scale_rows_kernel(float* __restrict__ Y, float* __restrict__ V, int64_t n, float f) {
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < n;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        Y[e] *= f;
        V[e] *= f;
    }
}

static int grid_for(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    if (b > 8192) b = 8192;
    if (b < 1) b = 1;
    return static_cast<int>(b);
}

cudaError_t launch_gather_rows(uint32_t* dst, const uint32_t* src, int64_t pitch, const int32_t* old,
                               int64_t n_rows, cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    gather_rows_kernel<<<grid_for(n_rows * pitch, 256), 256, 0, s>>>(dst, src, pitch, old, n_rows);
    return cudaGetLastError();
}

cudaError_t launch_repack_rows(void* dst, int64_t dpitch, const void* src, int64_t spitch, int64_t rows,
                               int64_t cols, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    repack_rows_kernel<<<grid_for(rows * 32, 256), 256, 0, s>>>(static_cast<uint32_t*>(dst), dpitch,
                                                                static_cast<const uint32_t*>(src), spitch, rows,
                                                                cols);
    return cudaGetLastError();
}

cudaError_t launch_scatter_rows(float* X32, int xpitch, const int64_t* ids, const float* rows, int64_t n, int D,
                                cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    scatter_rows_kernel<<<grid_for(n * D, 256), 256, 0, s>>>(X32, xpitch, ids, rows, n, D);
    return cudaGetLastError();
}

cudaError_t launch_remap_lists(int32_t* list, int k, const int32_t* new_of, int64_t N, uint32_t t, uint64_t seed,
                               uint32_t salt, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    remap_lists_kernel<<<grid_for(N * 32, 256), 256, 0, s>>>(list, k, new_of, N, t, seed, salt);
    return cudaGetLastError();
}

}  // namespace fsne

namespace fsne {
cudaError_t launch_scale_rows(float* Y, float* V, int64_t n_elem, float factor, cudaStream_t s) {
    if (n_elem <= 0) return cudaSuccess;
    scale_rows_kernel<<<grid_for(n_elem, 256), 256, 0, s>>>(Y, V, n_elem, factor);
    return cudaGetLastError();
}
}  // namespace fsne
