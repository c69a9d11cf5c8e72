// Brute-force exact KNN that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the moment they need neighbours:
// code that runs inside another framework whose caching allocator owns the
// device memory pool, real-time paths that must not trigger the implicit
// synchronisation of an allocation, or processes that pre-plan every byte
// of a fixed memory budget. For them this file keeps the scratch of the KNN
// kernels (the query indices and the per-query, per-slice partial top-k
// lists) in one file-scope device array of fixed size. Every GPU that loads
// the library holds that array until the process exits.
#include <cstdio>
#include <mutex>

#include "../../include/funcsne.h"
#include "launch.h"

namespace fsne {
void set_global_error(const char* msg);
}

namespace {

// 4 MiB of scratch per device.
constexpr size_t kScratchBytes = size_t(4) << 20;
static __device__ __align__(256) unsigned char g_knn_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};

int reject(int code, const char* fmt, long long a = 0, long long b = 0) {
    char buf[256];
    snprintf(buf, sizeof(buf), fmt, a, b);
    fsne::set_global_error(buf);
    return code;
}

}  // namespace

extern "C" int funcsne_exact_knn_noalloc(const float* X, int64_t N, int32_t D, int32_t ldx,
                                         const int32_t* queries, int64_t n_q, int32_t k, int32_t* idx,
                                         float* d2, void* stream) {
    if (!X || !queries || !idx) return reject(FUNCSNE_E_ARG, "exact_knn_noalloc: NULL argument");
    if (N < 2 || N >= (int64_t(1) << 31) - 1) return reject(FUNCSNE_E_ARG, "exact_knn_noalloc: N out of range (%lld)", N);
    if (D < 1 || ldx % 4 != 0 || ldx < (D + 3) / 4 * 4 || ldx > 4096)
        return reject(FUNCSNE_E_ARG, "exact_knn_noalloc: need ldx %% 4 == 0, ldx >= D rounded up to 4, ldx <= 4096 "
                      "(D=%lld, ldx=%lld)", D, ldx);
    if (reinterpret_cast<uintptr_t>(X) % 16 != 0) return reject(FUNCSNE_E_ARG, "exact_knn_noalloc: X must be 16-byte aligned");
    if (k < 1 || k > 64 || k >= N) return reject(FUNCSNE_E_ARG, "exact_knn_noalloc: k must be in [1, min(64, N-1)] (k=%lld)", k);
    if (n_q < 0) return reject(FUNCSNE_E_ARG, "exact_knn_noalloc: n_q must be >= 0");
    if (n_q == 0) return FUNCSNE_OK;
    // bounded first, so that the byte counts below cannot wrap around
    if (n_q > static_cast<int64_t>(kScratchBytes / 4))
        return reject(FUNCSNE_E_ARG, "exact_knn_noalloc: n_q=%lld exceeds the 4 MiB static scratch", n_q);
    const int RK = k <= 32 ? 1 : 2;
    const size_t q_bytes = (static_cast<size_t>(n_q) * 4 + 255) / 256 * 256;
    const size_t per_slice = static_cast<size_t>(n_q) * 32 * RK * sizeof(unsigned long long);
    if (q_bytes + per_slice > kScratchBytes) {
        const long long max_q = static_cast<long long>(kScratchBytes / (4 + 32 * RK * 8)) - 64;
        return reject(FUNCSNE_E_ARG, "exact_knn_noalloc: n_q=%lld exceeds the 4 MiB static scratch "
                      "(at most about %lld queries at this k)", n_q, max_q);
    }
    for (int64_t a = 0; a < n_q; ++a)
        if (queries[a] < 0 || queries[a] >= N)
            return reject(FUNCSNE_E_ARG, "exact_knn_noalloc: query %lld out of range (%lld)", a, queries[a]);

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return reject(FUNCSNE_E_CUDA, "exact_knn_noalloc: no usable current device");
    unsigned char* base = nullptr;
    int sms = 0;
    {
        // once per device, with that device current: the host-side name of
        // the array is not a device address, so look the address up.
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_knn_scratch);
            if (e != cudaSuccess)
                return reject(FUNCSNE_E_CUDA, "exact_knn_noalloc: cudaGetSymbolAddress failed (error %lld)", e);
            int s = 0;
            e = cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return reject(FUNCSNE_E_CUDA, "exact_knn_noalloc: device query failed (error %lld)", e);
            g_scratch_addr[dev] = static_cast<unsigned char*>(p);
            g_num_sms[dev] = s;
        }
        base = g_scratch_addr[dev];
        sms = g_num_sms[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t* dq = reinterpret_cast<int32_t*>(base);
    unsigned long long* part = reinterpret_cast<unsigned long long*>(base + q_bytes);

    fsne::KnnParams kp{};
    kp.N = N;
    kp.n4 = (D + 3) / 4;
    kp.xpitch = ldx;
    kp.k = k;
    kp.RK = RK;
    kp.n_q = n_q;
    const int64_t qb = (n_q + 7) / 8;
    int64_t ns = (8LL * sms + qb - 1) / qb;
    if (ns < 1) ns = 1;
    if (ns > 256) ns = 256;
    if (ns > N / 64 + 1) ns = N / 64 + 1;
    const int64_t fit = static_cast<int64_t>((kScratchBytes - q_bytes) / per_slice);
    if (ns > fit) ns = fit;
    kp.n_split = static_cast<int32_t>(ns);
    kp.X32 = X;
    kp.queries = dq;
    kp.part = part;
    kp.idx = idx;
    kp.d2 = d2;
    // every scratch entry the kernels read is written first in the same call,
    // so nothing needs clearing
    cudaError_t e = cudaMemcpyAsync(dq, queries, static_cast<size_t>(n_q) * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = fsne::launch_exact_knn(kp, s);
    if (e != cudaSuccess) return reject(FUNCSNE_E_CUDA, "exact_knn_noalloc: launch failed (error %lld)", e);
    return FUNCSNE_OK;
}
