// Online MLP surrogate of the embedding map x -> y (an addition to the
// method: it places inserted points before the iteration refines them).
//
// Network D-H-H-d, ReLU, bfloat16 operands with FP32 accumulation:
//   X^ = bf16((x - mu) / sigma),  H1 = bf16(relu(X^ W1^T + b1)),
//   H2 = bf16(relu(H1 W2^T + b2)),  O = H2 W3^T + b3,
//   target T = y / s with s = RMS of the batch's y,  L = mean (O - T)^2,
//   G3 = bf16(2 (O - T) / (B d)),  G2 = bf16((G3 W3) [H2 > 0]),
//   G1 = bf16((G2 W2) [H1 > 0]),  dW3 = G3^T H2,  dW2 = G2^T H1,
//   dW1 = G1^T X^,  db = column sums of G;  Adam with bias correction on
//   FP32 master parameters, then the bfloat16 copy is refreshed.
// Parameters are one flat array: W1 (H x D) b1 (H) W2 (H x H) b2 (H)
// W3 (d x H) b3 (d). The GEMMs run on the tensor cores (tcgen05.mma with
// TMEM accumulators, tc_gemm.cuh); the weight gradients (K = B) are split
// over K so that they fill the GPU, and their kernels also sum the bias
// gradients.
#include "device_common.cuh"
#include "launch.h"
#include "tc_gemm.cuh"

namespace fsne {

// ------------------------------------------------------------------ GEMM
// C[m][n] = sum_k A(m, k) B(n, k) on the tensor cores (tcgen05.mma,
// kind::f16: BF16 operands, FP32 accumulation in TMEM). Operand element
// (r, k) is p[r rs + k ks]. A CTA of 256 threads computes a 128 x 64 tile of
// C over the K values [z kc, (z + 1) kc) of its slice z (blockIdx.z),
// staging 64 K values of A and B at a time into shared memory in the layout
// of tc_gemm.cuh: two threads stage a row of A and four a row of B (16-byte
// vectors when a row is contiguous in K and aligned, single values
// otherwise, with consecutive threads on consecutive rows). Rows and K
// values outside the matrices are staged as zeros. Thread 0 issues the four
// MMAs of a chunk and commits them to an mbarrier that every thread waits on
// (a bounded wait: on time-out the kernel records kErrTimeout and stops)
// before the next chunk overwrites the operands. The accumulator tile goes
// from TMEM through shared memory to coalesced global writes.
// kEpiSplitF32 stores the partial tile of slice z at Cf + z M N (dense
// M x N) and, from the first column of tiles, the partial row sums of A at
// wsb + z M; gemm_reduce_kernel adds the slices in order.
enum { kEpiBiasReluBf16 = 0, kEpiBiasF32 = 1, kEpiMaskBf16 = 2, kEpiSplitF32 = 3 };

struct TcOperand {
    const __nv_bfloat16* p;
    int64_t rs, ks;   // strides of a row and of a K step, in elements
    int vec;          // rows contiguous in K and 16-byte aligned: 8-value loads
};

struct GemmArgs {
    int M, N, K, kc;  // kc: K values per CTA (a multiple of 64)
    TcOperand a, b;
    int ldc;
    const float* bias;          // N (bias epilogues)
    const __nv_bfloat16* mask;  // M x N, ldc (mask epilogue): keep where mask > 0
    __nv_bfloat16* Cb;          // bfloat16 output
    float* Cf;                  // FP32 output; the slices for kEpiSplitF32
    float* wsb;                 // row-sum slices (kEpiSplitF32)
    uint32_t* err;              // device error word
};

// Operand regions of the dynamic shared memory: A (128 rows) and B (64
// rows). A chunk takes 16 KB / 8 KB; each region is sized so that every
// address the descriptors can reach stays inside it. After the last MMA the
// A region holds the FP32 tile for the coalesced epilogue.
constexpr int kTcRegionA = 48 * 1024;
constexpr int kTcRegionB = 16 * 1024;
constexpr int kTcSmem = kTcRegionA + kTcRegionB;
constexpr int kTcThreads = 256;
constexpr int kTcTileLd = kTcBN + 1;  // padded row of the FP32 tile (floats)
constexpr uint32_t kTcWaitLimit = 1u << 24;

// Stage K values [k0 + kq, k0 + kq + nk) of operand row `row` (R rows in
// all) as row r of an Rt-row chunk at `dst` (zeros outside the matrix);
// returns the sum of the staged values (row sums of A for the bias
// gradients).
__device__ __forceinline__ float tc_stage(unsigned char* dst, const TcOperand& o, int r, int Rt, int row, int R,
                                          int k0, int kq, int nk, int kend) {
    float sum = 0.f;
    const bool in = row < R;
    const __nv_bfloat16* src = o.p + static_cast<int64_t>(in ? row : 0) * o.rs;
    if (o.vec) {
        for (int q = kq; q < kq + nk; q += 8) {
            const int k = k0 + q;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (in && k + 8 <= kend) {
                v = __ldg(reinterpret_cast<const uint4*>(src + k));
            } else if (in && k < kend) {
                __nv_bfloat16 t[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) t[e] = k + e < kend ? src[k + e] : __float2bfloat16_rn(0.f);
                v = *reinterpret_cast<const uint4*>(t);
            }
            *reinterpret_cast<uint4*>(dst + tc_offset(r, q, Rt)) = v;
            const __nv_bfloat16* t = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
            for (int e = 0; e < 8; ++e) sum += __bfloat162float(t[e]);
        }
    } else {
#pragma unroll 8
        for (int q = kq; q < kq + nk; ++q) {
            const int k = k0 + q;
            const __nv_bfloat16 v = (in && k < kend) ? src[static_cast<int64_t>(k) * o.ks] : __float2bfloat16_rn(0.f);
            *reinterpret_cast<__nv_bfloat16*>(dst + tc_offset(r, q, Rt)) = v;
            sum += __bfloat162float(v);
        }
    }
    return sum;
}

template <int EPI>
__global__ void __launch_bounds__(kTcThreads, 1) tc_gemm_kernel(const GemmArgs g) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ float s_rows[2][kTcBM];
    const int tid = threadIdx.x, warp = tid >> 5;
    unsigned char* As = tc_smem;
    unsigned char* Bs = tc_smem + kTcRegionA;
    if (warp == 0) tc_alloc(&tmem_base, kTcBN);
    if (tid == 0) mbar_init(&bar, 1);
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t taddr = tmem_base;

    const int m0 = blockIdx.y * kTcBM, n0 = blockIdx.x * kTcBN;
    const int kbeg = blockIdx.z * g.kc;
    const int kend = min(g.K, kbeg + g.kc);
    constexpr uint32_t lbo_a = (kTcBM / 8) * 128, lbo_b = (kTcBN / 8) * 128;
    constexpr uint32_t idesc = tc_idesc_bf16(kTcBM, kTcBN);
    const uint32_t a_addr = smem_u32(As), b_addr = smem_u32(Bs);
    // A: two threads a row (32 K values each); B: four threads a row (16 each)
    const int ar = tid & (kTcBM - 1), aq = (tid >> 7) * (kTcBK / 2);
    const int br = tid & (kTcBN - 1), bq = (tid >> 6) * (kTcBK / 4);
    float rsum = 0.f;
    uint32_t phase = 0;
    bool issued = false, timed_out = false;
    for (int k0 = kbeg; k0 < kend; k0 += kTcBK) {
        rsum += tc_stage(As, g.a, ar, kTcBM, m0 + ar, g.M, k0, aq, kTcBK / 2, kend);
        tc_stage(Bs, g.b, br, kTcBN, n0 + br, g.N, k0, bq, kTcBK / 4, kend);
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after_sync();
#pragma unroll
            for (int j = 0; j < kTcBK / 16; ++j) {
                const uint64_t ad = tc_smem_desc(a_addr + 2 * j * lbo_a, lbo_a, 128);
                const uint64_t bd = tc_smem_desc(b_addr + 2 * j * lbo_b, lbo_b, 128);
                tc_mma_bf16(taddr, ad, bd, idesc, issued || j > 0);
            }
            tc_commit(&bar);
        }
        issued = true;
        const bool ok = mbar_wait(&bar, phase, kTcWaitLimit);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
    }
    if (timed_out) {
        if (tid == 0) atomicOr(g.err, kErrTimeout);
        // the MMAs of the last chunk may still run: one more bounded wait
        mbar_wait(&bar, phase ^ 1u, kTcWaitLimit);
    } else {
        // TMEM -> the FP32 tile in shared memory: warp w reads lanes
        // 32 (w mod 4) + l (tile rows) and columns 32 (w / 4) .. + 31
        tc_fence_after_sync();
        float* Cs = reinterpret_cast<float*>(tc_smem);
        const int row = 32 * (warp & 3) + (tid & 31);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c0 = 32 * (warp >> 2) + 16 * h;
            float v[16];
            if (issued) {
                tc_ld16(taddr + (static_cast<uint32_t>(32 * (warp & 3)) << 16) + static_cast<uint32_t>(c0), v);
            } else {
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = 0.f;
            }
#pragma unroll
            for (int q = 0; q < 16; ++q) Cs[row * kTcTileLd + c0 + q] = v[q];
        }
        if (EPI == kEpiSplitF32) s_rows[tid >> 7][ar] = rsum;
        __syncthreads();
        // coalesced writes: consecutive threads take consecutive columns
        const int z = blockIdx.z;
        if (EPI == kEpiSplitF32 && blockIdx.x == 0 && tid < kTcBM && m0 + tid < g.M)
            g.wsb[static_cast<int64_t>(z) * g.M + m0 + tid] = s_rows[0][tid] + s_rows[1][tid];
        for (int e = tid; e < kTcBM * kTcBN; e += kTcThreads) {
            const int r = e / kTcBN, c = e % kTcBN;
            const int m = m0 + r, n = n0 + c;
            if (m >= g.M || n >= g.N) continue;
            const float v = Cs[r * kTcTileLd + c];
            if constexpr (EPI == kEpiSplitF32) {
                g.Cf[(static_cast<int64_t>(z) * g.M + m) * g.N + n] = v;
            } else {
                const int64_t o = static_cast<int64_t>(m) * g.ldc + n;
                if constexpr (EPI == kEpiBiasReluBf16) {
                    const float t = v + g.bias[n];
                    g.Cb[o] = __float2bfloat16_rn(t > 0.f ? t : 0.f);
                } else if constexpr (EPI == kEpiBiasF32) {
                    g.Cf[o] = v + g.bias[n];
                } else {
                    g.Cb[o] = __bfloat162float(g.mask[o]) > 0.f ? __float2bfloat16_rn(v) : __float2bfloat16_rn(0.f);
                }
            }
        }
    }
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after_sync();
        tc_dealloc(taddr, kTcBN);
    }
}

// A bounded wait that runs out: one thread polls an mbarrier that expects an
// arrival nothing makes, `polls` times, then records kErrTimeout.
__global__ void bounded_wait_kernel(uint32_t* err, uint32_t polls) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    if (!mbar_wait(&bar, 0u, polls)) atomicOr(err, kErrTimeout);
}

cudaError_t launch_bounded_wait(uint32_t* err, uint32_t polls, cudaStream_t s) {
    bounded_wait_kernel<<<1, 32, 0, s>>>(err, polls);
    return cudaGetLastError();
}

// C[e] = sum over z = 0 .. S-1 of ws[z M N + e] (e < M N) and
// rows[m] = sum over z of wsb[z M + m] (m < M), both in slice order.
__global__ void gemm_reduce_kernel(const float* __restrict__ ws, const float* __restrict__ wsb, int S, int M, int N,
                                   float* __restrict__ C, float* __restrict__ rows) {
    const int64_t MN = static_cast<int64_t>(M) * N;
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e < MN) {
        float s = 0.f;
        for (int z = 0; z < S; ++z) s += ws[z * MN + e];
        C[e] = s;
    }
    if (e < M) {
        float s = 0.f;
        for (int z = 0; z < S; ++z) s += wsb[static_cast<int64_t>(z) * M + e];
        rows[e] = s;
    }
}

static TcOperand operand(const __nv_bfloat16* p, int64_t rs, int64_t ks) {
    TcOperand o;
    o.p = p;
    o.rs = rs;
    o.ks = ks;
    o.vec = ks == 1 && rs % 8 == 0 && reinterpret_cast<uintptr_t>(p) % 16 == 0;
    return o;
}

template <int EPI>
static void tc_launch(const GemmArgs& g, int slices, cudaStream_t s) {
    cudaFuncSetAttribute(tc_gemm_kernel<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    const dim3 grid((g.N + kTcBN - 1) / kTcBN, (g.M + kTcBM - 1) / kTcBM, slices);
    tc_gemm_kernel<EPI><<<grid, kTcThreads, kTcSmem, s>>>(g);
}

template <int EPI>
static void gemm(GemmArgs g, cudaStream_t s) {
    g.kc = (g.K + kTcBK - 1) / kTcBK * kTcBK;
    tc_launch<EPI>(g, 1, s);
}

// Weight gradient C (dense M x N) = sum over the K = B batch rows of
// A(m, k) B(n, k), and rows[m] = sum_k A(m, k) (the bias gradient). Split
// over K into slices of at least 128 rows (at most 32 slices, and no more
// than the workspace of ws_floats holds).
static void gemm_weight_grad(GemmArgs g, float* ws, int64_t ws_floats, float* C, float* rows, cudaStream_t s) {
    const int64_t per = static_cast<int64_t>(g.M) * g.N + g.M;
    int S = (g.K + 127) / 128;
    if (S > 32) S = 32;
    while (S > 1 && S * per > ws_floats) --S;
    g.kc = ((g.K + S - 1) / S + kTcBK - 1) / kTcBK * kTcBK;
    S = (g.K + g.kc - 1) / g.kc;
    g.Cf = ws;
    g.wsb = ws + static_cast<int64_t>(S) * g.M * g.N;
    tc_launch<kEpiSplitF32>(g, S, s);
    const int64_t n = static_cast<int64_t>(g.M) * g.N > g.M ? static_cast<int64_t>(g.M) * g.N : g.M;
    gemm_reduce_kernel<<<static_cast<int>((n + 255) / 256), 256, 0, s>>>(g.Cf, g.wsb, S, g.M, g.N, C, rows);
}

// ------------------------------------------------------------------ data
// Per-feature mean and standard deviation of the first N rows (FP64 sums).
__global__ void mlp_stats_kernel(const float* __restrict__ X, int64_t N, int xpitch, float* mu, float* sigma) {
    const int f = blockIdx.x;
    double s = 0.0, s2 = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const double v = X[i * xpitch + f];
        s += v;
        s2 += v * v;
    }
    __shared__ double ps[256], ps2[256];
    ps[threadIdx.x] = s;
    ps2[threadIdx.x] = s2;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            ps[threadIdx.x] += ps[threadIdx.x + w];
            ps2[threadIdx.x] += ps2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double m = ps[0] / static_cast<double>(N);
        const double var = ps2[0] / static_cast<double>(N) - m * m;
        mu[f] = static_cast<float>(m);
        sigma[f] = var > 0.0 ? static_cast<float>(sqrt(var)) : 1.f;
    }
}

// Normalised bfloat16 input rows X^ of the given point indices.
__global__ void mlp_inputs_kernel(const float* __restrict__ X, int xpitch, int D, const int32_t* __restrict__ idx,
                                  int64_t first, int rows, const float* __restrict__ mu,
                                  const float* __restrict__ sigma, __nv_bfloat16* Xb) {
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= static_cast<int64_t>(rows) * D) return;
    const int r = static_cast<int>(e / D), f = static_cast<int>(e % D);
    const int64_t i = idx ? idx[r] : first + r;
    Xb[e] = __float2bfloat16_rn((X[i * xpitch + f] - mu[f]) / sigma[f]);
}

// Batch of the training step `step`: row b is point map(w0, N) of the
// Philox block at counter (step, b, MLP, 0); targets y (scaled later).
__global__ void mlp_batch_kernel(MlpParams q) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t step = *q.step;
    __shared__ double red[256];
    double acc = 0.0;
    if (b < q.B) {
        const uint4 w = philox(step, static_cast<uint32_t>(b), kStreamMlp, 0u, q.seed);
        const uint32_t i = map_index(w.x, static_cast<uint32_t>(q.N));
        q.idx[b] = static_cast<int32_t>(i);
        for (int c = 0; c < q.d; ++c) {
            const float y = q.Y[static_cast<int64_t>(i) * q.DP + c];
            q.T[b * q.d + c] = y;
            acc += static_cast<double>(y) * y;
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) q.part[blockIdx.x] = red[0];
}

// s = RMS of the batch targets (1 when zero); targets divided by s. Every
// block sums the partials in the same order, so all use the same s.
__global__ void mlp_scale_kernel(MlpParams q, int nparts) {
    __shared__ float s_scale;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < nparts; ++b) t += q.part[b];
        const double ms = t / (static_cast<double>(q.B) * q.d);
        const float s = ms > 0.0 ? static_cast<float>(sqrt(ms)) : 1.f;
        s_scale = s;
        if (blockIdx.x == 0) *q.scale = s;
    }
    __syncthreads();
    const float inv = 1.f / s_scale;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < q.B * q.d) q.T[e] *= inv;
}

// G3 = bf16(2 (O - T) / (B d)); loss partials.
__global__ void mlp_loss_kernel(MlpParams q) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    __shared__ double red[256];
    double l = 0.0;
    if (e < q.B * q.d) {
        const float r = q.O[e] - q.T[e];
        l = static_cast<double>(r) * r;
        q.G3[e] = __float2bfloat16_rn(2.f * r / static_cast<float>(q.B * q.d));
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) q.part[blockIdx.x] = red[0];
}

__global__ void mlp_loss_finish_kernel(MlpParams q, int nparts) {
    if (threadIdx.x != 0) return;
    double t = 0.0;
    for (int b = 0; b < nparts; ++b) t += q.part[b];
    *q.loss = t / (static_cast<double>(q.B) * q.d);
}

// Adam with bias correction; refreshes the bfloat16 copy; step advances in
// mlp_step_kernel.
__global__ void mlp_adam_kernel(MlpParams q) {
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= q.n_params) return;
    const int step = static_cast<int>(*q.step) + 1;
    const float c1 = 1.f - powf(q.beta1, static_cast<float>(step));
    const float c2 = 1.f - powf(q.beta2, static_cast<float>(step));
    const float g = q.grad[e];
    const float m = q.beta1 * q.m[e] + (1.f - q.beta1) * g;
    const float v = q.beta2 * q.v[e] + (1.f - q.beta2) * g * g;
    q.m[e] = m;
    q.v[e] = v;
    const float th = q.theta[e] - q.lr * (m / c1) / (sqrtf(v / c2) + q.eps);
    q.theta[e] = th;
    q.wb[e] = __float2bfloat16_rn(th);
}

__global__ void mlp_step_kernel(MlpParams q) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *q.step += 1u;
}

// Y[first + r][c] = s O[r][c] for the placed rows (LD padding untouched).
__global__ void mlp_place_kernel(const float* __restrict__ O, int rows, int d, int DP, int64_t first,
                                 const float* __restrict__ scale, float* Y) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * d) return;
    const int r = e / d, c = e % d;
    Y[(first + r) * DP + c] = *scale * O[e];
}

// ------------------------------------------------------------------ host side
static int blocks_for(int64_t n, int t) { return static_cast<int>((n + t - 1) / t); }

cudaError_t launch_mlp_stats(const float* X, int64_t N, int D, int xpitch, float* mu, float* sigma, cudaStream_t s) {
    mlp_stats_kernel<<<D, 256, 0, s>>>(X, N, xpitch, mu, sigma);
    return cudaGetLastError();
}

// forward of `rows` input rows already in q.Xb: H1, H2, O.
static void mlp_forward(const MlpParams& q, int rows, cudaStream_t s) {
    const int D = q.D, H = q.H, d = q.d;
    const __nv_bfloat16* W1 = q.wb;
    const __nv_bfloat16* W2 = q.wb + static_cast<int64_t>(H) * D + H;
    const __nv_bfloat16* W3 = W2 + static_cast<int64_t>(H) * H + H;
    const float* b1 = q.theta + static_cast<int64_t>(H) * D;
    const float* b2 = b1 + H + static_cast<int64_t>(H) * H;
    const float* b3 = b2 + H + static_cast<int64_t>(d) * H;
    GemmArgs g{};
    g.err = q.err;
    // H1 = relu(X^ W1^T + b1): A(b, f) = X^[b][f], B(h, f) = W1[h][f]
    g.M = rows; g.N = H; g.K = D; g.ldc = H;
    g.a = operand(q.Xb, D, 1); g.b = operand(W1, D, 1); g.bias = b1; g.Cb = q.H1;
    gemm<kEpiBiasReluBf16>(g, s);
    // H2 = relu(H1 W2^T + b2)
    g.K = H; g.a = operand(q.H1, H, 1); g.b = operand(W2, H, 1); g.bias = b2; g.Cb = q.H2;
    gemm<kEpiBiasReluBf16>(g, s);
    // O = H2 W3^T + b3
    g.N = d; g.ldc = d; g.a = operand(q.H2, H, 1); g.b = operand(W3, H, 1); g.bias = b3; g.Cb = nullptr; g.Cf = q.O;
    gemm<kEpiBiasF32>(g, s);
}

cudaError_t launch_mlp_train_step(const MlpParams& q, cudaStream_t s) {
    const int B = q.B, D = q.D, H = q.H, d = q.d;
    const int nb = blocks_for(B, 256);
    mlp_batch_kernel<<<nb, 256, 0, s>>>(q);
    mlp_scale_kernel<<<blocks_for(static_cast<int64_t>(B) * d, 256), 256, 0, s>>>(q, nb);
    mlp_inputs_kernel<<<blocks_for(static_cast<int64_t>(B) * D, 256), 256, 0, s>>>(q.X32, q.xpitch, D, q.idx, 0, B,
                                                                                   q.mu, q.sigma, q.Xb);
    mlp_forward(q, B, s);
    const int nl = blocks_for(static_cast<int64_t>(B) * d, 256);
    mlp_loss_kernel<<<nl, 256, 0, s>>>(q);
    mlp_loss_finish_kernel<<<1, 32, 0, s>>>(q, nl);
    // backward
    const __nv_bfloat16* W2 = q.wb + static_cast<int64_t>(H) * D + H;
    const __nv_bfloat16* W3 = W2 + static_cast<int64_t>(H) * H + H;
    float* gW1 = q.grad;
    float* gb1 = gW1 + static_cast<int64_t>(H) * D;
    float* gW2 = gb1 + H;
    float* gb2 = gW2 + static_cast<int64_t>(H) * H;
    float* gW3 = gb2 + H;
    float* gb3 = gW3 + static_cast<int64_t>(d) * H;
    GemmArgs g{};
    // dW3 = G3^T H2 (d x H), db3 = column sums of G3
    g.err = q.err;
    g.M = d; g.N = H; g.K = B; g.a = operand(q.G3, 1, d); g.b = operand(q.H2, 1, H);
    gemm_weight_grad(g, q.ws, q.ws_floats, gW3, gb3, s);
    // G2 = (G3 W3) [H2 > 0]  (B x H)
    g = GemmArgs{};
    g.err = q.err;
    g.M = B; g.N = H; g.K = d; g.ldc = H; g.a = operand(q.G3, d, 1); g.b = operand(W3, 1, H); g.mask = q.H2;
    g.Cb = q.G2;
    gemm<kEpiMaskBf16>(g, s);
    // dW2 = G2^T H1 (H x H), db2 = column sums of G2
    g = GemmArgs{};
    g.err = q.err;
    g.M = H; g.N = H; g.K = B; g.a = operand(q.G2, 1, H); g.b = operand(q.H1, 1, H);
    gemm_weight_grad(g, q.ws, q.ws_floats, gW2, gb2, s);
    // G1 = (G2 W2) [H1 > 0]  (B x H)
    g = GemmArgs{};
    g.err = q.err;
    g.M = B; g.N = H; g.K = H; g.ldc = H; g.a = operand(q.G2, H, 1); g.b = operand(W2, 1, H); g.mask = q.H1;
    g.Cb = q.G1;
    gemm<kEpiMaskBf16>(g, s);
    // dW1 = G1^T X^ (H x D), db1 = column sums of G1
    g = GemmArgs{};
    g.err = q.err;
    g.M = H; g.N = D; g.K = B; g.a = operand(q.G1, 1, H); g.b = operand(q.Xb, 1, D);
    gemm_weight_grad(g, q.ws, q.ws_floats, gW1, gb1, s);
    mlp_adam_kernel<<<blocks_for(q.n_params, 256), 256, 0, s>>>(q);
    mlp_step_kernel<<<1, 32, 0, s>>>(q);
    return cudaGetLastError();
}

cudaError_t launch_mlp_place(const MlpParams& q, const float* X, int xpitch, int64_t first, int64_t rows, float* Y,
                             int DP, cudaStream_t s) {
    for (int64_t r0 = 0; r0 < rows; r0 += q.B) {
        const int n = static_cast<int>(rows - r0 < q.B ? rows - r0 : q.B);
        mlp_inputs_kernel<<<blocks_for(static_cast<int64_t>(n) * q.D, 256), 256, 0, s>>>(
            X, xpitch, q.D, nullptr, first + r0, n, q.mu, q.sigma, q.Xb);
        mlp_forward(q, n, s);
        mlp_place_kernel<<<blocks_for(static_cast<int64_t>(n) * q.d, 256), 256, 0, s>>>(q.O, n, q.d, DP, first + r0,
                                                                                        q.scale, Y);
    }
    return cudaGetLastError();
}

// Initial parameters: weights of layer l (0-based) uniform in (-a, a) with
// a = sqrt(6 / fan_in) for l < 2 and sqrt(3 / fan_in) for the output layer;
// entry (r, c) from word c mod 4 of the Philox block at counter
// (l + 1, r, MLP_INIT, c div 4) as a (2 (w + 0.5) 2^-32 - 1) in FP64,
// rounded to binary32; biases 0.
__global__ void mlp_init_kernel(float* theta, __nv_bfloat16* wb, int D, int H, int d, uint64_t seed) {
    const int64_t n1 = static_cast<int64_t>(H) * D, n2 = static_cast<int64_t>(H) * H, n3 = static_cast<int64_t>(d) * H;
    const int64_t total = n1 + H + n2 + H + n3 + d;
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= total) return;
    int layer = -1, cols = 0;
    int64_t off = e;
    if (off < n1) { layer = 0; cols = D; }
    else if ((off -= n1) < H) { layer = -1; }
    else if ((off -= H) < n2) { layer = 1; cols = H; }
    else if ((off -= n2) < H) { layer = -1; }
    else if ((off -= H) < n3) { layer = 2; cols = H; }
    float v = 0.f;
    if (layer >= 0) {
        const int r = static_cast<int>(off / cols), c = static_cast<int>(off % cols);
        const uint4 w = philox(static_cast<uint32_t>(layer + 1), static_cast<uint32_t>(r), kStreamMlpInit,
                               static_cast<uint32_t>(c / 4), seed);
        const uint32_t word = (c & 3) == 0 ? w.x : (c & 3) == 1 ? w.y : (c & 3) == 2 ? w.z : w.w;
        const double a = sqrt((layer < 2 ? 6.0 : 3.0) / static_cast<double>(cols));
        const double u = (static_cast<double>(word) + 0.5) * (1.0 / 4294967296.0);
        v = static_cast<float>(a * (2.0 * u - 1.0));
    }
    theta[e] = v;
    wb[e] = __float2bfloat16_rn(v);
}

cudaError_t launch_mlp_init(float* theta, __nv_bfloat16* wb, int D, int H, int d, uint64_t seed, cudaStream_t s) {
    const int64_t total = static_cast<int64_t>(H) * D + H + static_cast<int64_t>(H) * H + H + static_cast<int64_t>(d) * H + d;
    mlp_init_kernel<<<blocks_for(total, 256), 256, 0, s>>>(theta, wb, D, H, d, seed);
    return cudaGetLastError();
}

__global__ void bf16_to_f32_kernel(const __nv_bfloat16* in, int64_t n, float* out) {
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e < n) out[e] = __bfloat162float(in[e]);
}

cudaError_t launch_bf16_to_f32(const __nv_bfloat16* in, int64_t n, float* out, cudaStream_t s) {
    bf16_to_f32_kernel<<<blocks_for(n, 256), 256, 0, s>>>(in, n, out);
    return cudaGetLastError();
}

}  // namespace fsne
