// Set-up kernels of the FUnc-SNE state: initial neighbour lists, list
// finalisation (FP32 distances, (d2, idx) order, cold or imported P),
// the random linear projection Y0, the first normalisation estimate, the
// BF16 / FP8 row copies, and import checks.
#include "device_common.cuh"
#include "launch.h"

namespace fsne {

// Initial list of point i: slot l draws an offset o_l in [0, N-1) from
// counter (0, i, stream, l); an offset already taken moves to the next free
// one (mod N-1); the neighbour is (i + 1 + o_l) mod N. k <= 64.
__global__ void init_lists_kernel(int64_t N, int k, uint32_t stream, uint64_t seed, int32_t* out) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= N) return;
    uint32_t off[64];
    const uint32_t m = static_cast<uint32_t>(N - 1);
    for (int l = 0; l < k; ++l) {
        const uint4 w = philox(0u, static_cast<uint32_t>(i), stream, static_cast<uint32_t>(l), seed);
        uint32_t o = map_index(w.x, m);
        for (;;) {
            bool taken = false;
            for (int a = 0; a < l; ++a) taken |= (off[a] == o);
            if (!taken) break;
            o = (o + 1u == m) ? 0u : o + 1u;
        }
        off[l] = o;
        out[i * k + l] = static_cast<int32_t>((static_cast<uint64_t>(i) + 1u + o) % static_cast<uint64_t>(N));
    }
}

// Warp per point: FP32 distances of the listed HD neighbours (grouped as in
// the iteration, so stored and freshly scored distances agree bit for bit), order by
// (d2, idx), then either a cold-start bisection (Pin == nullptr) or the
// imported P row permuted along with the entries. Lists must be valid.
template <int RH>
__global__ void __launch_bounds__(256) hd_finalize_kernel(FinalizeParams f) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    float* xs = reinterpret_cast<float*>(smem) + wib * f.xpitch;
    const int k = f.k_hd;
    for (int64_t gi = static_cast<int64_t>(blockIdx.x) * wpb + wib; gi < f.N;
         gi += static_cast<int64_t>(gridDim.x) * wpb) {
        const float* xrow = f.X32 + gi * f.xpitch;
        for (int q = lane * 4; q < f.xpitch; q += 128)
            *reinterpret_cast<float4*>(xs + q) = __ldg(reinterpret_cast<const float4*>(xrow + q));
        __syncwarp();
        uint64_t key[RH];
        float pin[RH];
        uint32_t idx0[RH];
#pragma unroll
        for (int r = 0; r < RH; ++r) {
            const int e = r * 32 + lane;
            key[r] = kSentinel;
            pin[r] = 0.f;
            idx0[r] = 0xffffffffu;
            if (e < k) {
                idx0[r] = static_cast<uint32_t>(f.idx[gi * k + e]);
                if (f.Pin) pin[r] = f.Pin[gi * k + e];
            }
            // the same FP32 grouping as the iteration's distances
            const float d = group_rerank_f32(xs, f.X32, f.xpitch, f.n4, idx0[r], e < k, lane, f.g);
            if (e < k) key[r] = make_key(d, idx0[r]);
        }
        warp_sort<RH>(key, lane);
        float d2[RH], pv[RH];
#pragma unroll
        for (int r = 0; r < RH; ++r) d2[r] = key_d2(key[r]);
        if (f.Pin) {
            // carry the imported p_{j|i} to the entry's new position
#pragma unroll
            for (int r = 0; r < RH; ++r) {
                const uint32_t j = key_idx(key[r]);
                float v = 0.f;
#pragma unroll
                for (int r2 = 0; r2 < RH; ++r2)
                    for (int m = 0; m < 32; ++m) {
                        const uint32_t o = __shfl_sync(kFull, idx0[r2], m);
                        const float pp = __shfl_sync(kFull, pin[r2], m);
                        if (o == j) v = pp;
                    }
                pv[r] = v;
            }
        } else {
            const float b = warp_bisect<RH>(d2, k, f.log_perp, 0.f, pv, lane);
            if (lane == 0) f.beta[gi] = b;
        }
#pragma unroll
        for (int r = 0; r < RH; ++r) {
            const int e = r * 32 + lane;
            if (e < k) {
                f.idx[gi * k + e] = static_cast<int32_t>(key_idx(key[r]));
                f.d2[gi * k + e] = d2[r];
                f.P[gi * k + e] = pv[r];
            }
        }
        __syncwarp();
    }
}

// Gaussian matrix R from counter (ctr, f, INIT_Y, c), Box-Muller in FP64,
// stored as FP32 in D4 rows of DP columns (rows f >= D and columns c >= d
// zero, so the padding of X and of Y contributes nothing).
__global__ void gauss_matrix_kernel(int D, int D4, int d, int DP, uint32_t ctr, uint64_t seed, float* R) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= D4 * DP) return;
    const int fi = e / DP, c = e % DP;
    if (fi >= D || c >= d) {
        R[e] = 0.f;
        return;
    }
    const uint4 w = philox(ctr, static_cast<uint32_t>(fi), kStreamInitY, static_cast<uint32_t>(c), seed);
    const double u1 = (static_cast<double>(w.x) + 0.5) * (1.0 / 4294967296.0);
    const double u2 = (static_cast<double>(w.y) + 0.5) * (1.0 / 4294967296.0);
    R[e] = static_cast<float>(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
}

// Column sums (FP64) of a row-major N x cols FP32 matrix with row pitch
// `pitch` (of squared deviations from `shift` when `square`): block b sums
// rows [b * rows_per_block, ...) into part[b * cols + c]. Up to 128 columns,
// the block's threads form blockDim / cols row lanes per column, whose sums
// are then added in row-lane order; wider matrices take a column per thread.
__global__ void __launch_bounds__(256) col_sums_kernel(const float* __restrict__ M, int64_t N, int cols, int pitch,
                                                       int64_t rows_per_block, const double* __restrict__ shift,
                                                       int square, double* part) {
    __shared__ double s_part[256];
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * rows_per_block;
    const int64_t r1 = min(N, r0 + rows_per_block);
    if (cols <= 128) {
        const int nrl = static_cast<int>(blockDim.x) / cols;
        const int rl = static_cast<int>(threadIdx.x) / cols, c = static_cast<int>(threadIdx.x) % cols;
        double acc = 0.0;
        if (rl < nrl) {
            const double sh = shift ? shift[c] : 0.0;
            for (int64_t r = r0 + rl; r < r1; r += nrl) {
                const double v = static_cast<double>(M[r * pitch + c]) - sh;
                acc += square ? v * v : v;
            }
        }
        s_part[threadIdx.x] = acc;
        __syncthreads();
        if (static_cast<int>(threadIdx.x) < cols) {
            double t = 0.0;
            for (int k = 0; k < nrl; ++k) t += s_part[k * cols + threadIdx.x];
            part[static_cast<int64_t>(blockIdx.x) * cols + threadIdx.x] = t;
        }
        return;
    }
    for (int c = threadIdx.x; c < cols; c += blockDim.x) {
        double acc = 0.0;
        const double sh = shift ? shift[c] : 0.0;
        for (int64_t r = r0; r < r1; ++r) {
            const double v = static_cast<double>(M[r * pitch + c]) - sh;
            acc += square ? v * v : v;
        }
        part[static_cast<int64_t>(blockIdx.x) * cols + c] = acc;
    }
}

// out[c] = (sum_b part[b*cols + c]) * scale, summed in block order.
__global__ void reduce_parts_kernel(const double* part, int nparts, int cols, double scale, double* out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += part[static_cast<int64_t>(b) * cols + c];
    out[c] = s * scale;
}

// Y[i, c] = sum_f (x_if - mu_f) R[f, c] in FP32, thread per point, rows read
// 16 bytes at a time; R (FP32, zero padded) is read warp-uniformly.
template <int DP>
__global__ void __launch_bounds__(128) project_kernel(const float* __restrict__ X, int64_t N, int D, int n4,
                                                      int xpitch, const double* __restrict__ mu,
                                                      const float* __restrict__ R, float* Y) {
    extern __shared__ float s_mu[];
    for (int f = threadIdx.x; f < 4 * n4; f += blockDim.x) s_mu[f] = f < D ? static_cast<float>(mu[f]) : 0.f;
    __syncthreads();
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float acc[DP];
#pragma unroll
    for (int c = 0; c < DP; ++c) acc[c] = 0.f;
    const float4* xr = reinterpret_cast<const float4*>(X + i * xpitch);
    for (int q = 0; q < n4; ++q) {
        const float4 x = __ldg(xr + q);
        const float v[4] = {x.x - s_mu[4 * q], x.y - s_mu[4 * q + 1], x.z - s_mu[4 * q + 2], x.w - s_mu[4 * q + 3]};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float* r = R + (4 * q + k) * DP;
#pragma unroll
            for (int c = 0; c < DP; ++c) acc[c] = __fmaf_rn(v[k], __ldg(r + c), acc[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < DP; ++c) Y[i * DP + c] = acc[c];
}

// Scale factors of the columns: target_std / std_c (1 for a zero variance),
// from the FP64 moments.
__global__ void col_scale_kernel(const double* var, int d, int DP, double target_std, float* sc) {
    const int c = threadIdx.x;
    if (c >= DP) return;
    const double sd = c < d ? sqrt(var[c]) : 0.0;
    sc[c] = static_cast<float>(sd > 0.0 ? target_std / sd : 1.0);
}

// Y[:, c] *= sc[c] (DP a power of two).
__global__ void scale_cols_kernel(float* Y, int64_t n, int DP, const float* __restrict__ sc) {
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= n) return;
    Y[e] *= __ldg(sc + (static_cast<int>(e) & (DP - 1)));
}

// Warp per point: z_i = sum_{j in S_i} w_ij + (N-1)/n_neg sum_s 1[j_s not in S_i] w_ij_s
// with S_i = HD u LD lists and negatives from counter (t, i, stream, s).
template <int DP>
__global__ void __launch_bounds__(256) zinit_kernel(ZinitParams z) {
    __shared__ int32_t s_list[8][96];
    __shared__ double s_z[8];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double acc = 0.0;
    const uint32_t N = static_cast<uint32_t>(z.N);
    for (int64_t gi = static_cast<int64_t>(blockIdx.x) * 8 + wib; gi < z.N;
         gi += static_cast<int64_t>(gridDim.x) * 8) {
        const uint32_t i = static_cast<uint32_t>(gi);
        float yi[DP];
        load_row<DP>(z.Y + gi * DP, yi);
        for (int e = lane; e < z.k_hd; e += 32) s_list[wib][e] = z.hd_idx[gi * z.k_hd + e];
        if (lane < z.k_ld) s_list[wib][64 + lane] = z.ld_idx[gi * z.k_ld + lane];
        __syncwarp();
        float zi = 0.f;
        auto wfun = [&](int32_t j) {
            float yj[DP];
            load_row<DP>(z.Y + static_cast<int64_t>(j) * DP, yj);
            const float r2 = sqdist_ld<DP>(yi, yj);
            const float winv = 1.f / __fmaf_rn(r2, z.inv_alpha, 1.f);
            return z.alpha == 1.f ? winv : powf(winv, z.alpha);
        };
        for (int e = lane; e < z.k_hd; e += 32) zi += wfun(s_list[wib][e]);
        if (lane < z.k_ld) {
            const int32_t j = s_list[wib][64 + lane];
            bool in_hd = false;
            for (int m = 0; m < z.k_hd; ++m) in_hd |= (s_list[wib][m] == j);
            if (!in_hd) zi += wfun(j);
        }
        const uint4 w = philox(z.t, i, z.stream, static_cast<uint32_t>(lane), z.seed);
        for (int s = lane; s < z.n_neg; s += 32) {
            const int32_t j = static_cast<int32_t>(map_other(negative_word(w.y, w.w, static_cast<uint32_t>(s >> 5)), N, i));
            bool in_s = false;
            for (int m = 0; m < z.k_hd; ++m) in_s |= (s_list[wib][m] == j);
            for (int m = 0; m < z.k_ld; ++m) in_s |= (s_list[wib][64 + m] == j);
            if (!in_s) zi = __fmaf_rn(z.neg_scale, wfun(j), zi);
        }
        acc += static_cast<double>(warp_sum(zi));
        __syncwarp();
    }
    if (lane == 0) s_z[wib] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += s_z[w];
        z.part[blockIdx.x] = s;
    }
}

__global__ void zinit_finish_kernel(const double* part, int n, DevScalars* sc) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < n; ++b) s += part[b];
    sc->Zhat = s;
    sc->last_Z = s;
}

// Upper bound of a row's rounding error norm from per-lane sums of squared
// errors, all in FP32 with upward rounding: every square, every sum and the
// square root round up, so the result is >= the exact norm. The warp sum is
// a butterfly of upward additions (commutative, so every lane ends equal).
__device__ __forceinline__ float err_norm_bound(float s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = __fadd_ru(s, __shfl_xor_sync(kFull, s, o));
    return __fsqrt_ru(s);
}

// BF16 copy, one warp per row: round to nearest even, zero padding up to
// `err_off`, then at byte `err_off` a bound E >= ||x - x~|| of the row's own
// rounding error (err_norm_bound).
__global__ void quantize_bf16_kernel(const float* __restrict__ X, int64_t N, int D, int xpitch,
                                     int qpitch, int err_off, uint8_t* Q) {
    const int lane = threadIdx.x & 31;
    const int64_t i = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= N) return;
    __nv_bfloat16* row = reinterpret_cast<__nv_bfloat16*>(Q + i * qpitch);
    float s = 0.f;
    for (int f = lane; f < err_off / 2; f += 32) {
        const float x = f < D ? X[i * xpitch + f] : 0.f;
        const __nv_bfloat16 b = __float2bfloat16_rn(x);
        row[f] = b;
        // exact in FP32: both are multiples of x's FP32 ulp and differ by at
        // most half a BF16 ulp
        const float e = __fsub_rn(x, __bfloat162float(b));
        s = __fadd_ru(s, __fmul_ru(e, e));
    }
    const float E = err_norm_bound(s);
    if (lane == 0) *reinterpret_cast<float*>(Q + i * qpitch + err_off) = E;
}

// FP8-E4M3 copy with per-row scale s = max|x| / 448 (s = 1 for a zero row),
// codes = RNE(x / s) (saturating), zero codes up to byte scale_off - 4, the
// bound E >= ||x - x~|| of the row's own error at scale_off - 4 and the
// scale at scale_off (the row's last eight bytes). x~ is decoded by
// fp8x4_to_float, the same FP32 arithmetic as the distance kernels use.
__global__ void quantize_fp8_kernel(const float* __restrict__ X, int64_t N, int D, int xpitch,
                                    int qpitch, int scale_off, uint8_t* Q) {
    const int lane = threadIdx.x & 31;
    const int64_t i = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= N) return;
    float m = 0.f;
    for (int f = lane; f < D; f += 32) m = fmaxf(m, fabsf(X[i * xpitch + f]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
    const float s = m > 0.f ? m / 448.f : 1.f;
    uint8_t* row = Q + i * qpitch;
    const int err_off = scale_off - 4;
    float es = 0.f;
    for (int w = lane; w < err_off / 4; w += 32) {
        float x[4];
        uint32_t word = 0u;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int f = 4 * w + k;
            x[k] = f < D ? X[i * xpitch + f] : 0.f;
            const uint32_t c = __nv_cvt_float_to_fp8(x[k] / s, __NV_SATFINITE, __NV_E4M3);
            word |= c << (8 * k);
        }
        *reinterpret_cast<uint32_t*>(row + 4 * w) = word;
        float v[4];
        fp8x4_to_float(word, s, v);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            // |x - x~| rounded up (the difference need not be exact in FP32)
            const float e = __fsub_ru(fmaxf(x[k], v[k]), fminf(x[k], v[k]));
            es = __fadd_ru(es, __fmul_ru(e, e));
        }
    }
    const float E = err_norm_bound(es);
    if (lane == 0) {
        *reinterpret_cast<float*>(row + err_off) = E;
        *reinterpret_cast<float*>(row + scale_off) = s;
    }
}

// Import check: every list entry in [0, N), not the point itself, distinct.
__global__ void check_lists_kernel(const int32_t* idx, int64_t N, int k, uint32_t* err) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= N) return;
    bool bad = false;
    for (int a = 0; a < k; ++a) {
        const int32_t j = idx[i * k + a];
        bad |= (j < 0) || (j >= N) || (j == i);
        for (int b = 0; b < a; ++b) bad |= (idx[i * k + b] == j);
    }
    if (bad) atomicOr(err, kErrIndex);
}

// Non-finite check of the input rows.
__global__ void check_finite_kernel(const float* X, int64_t n, uint32_t* err) {
    bool bad = false;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < n;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x)
        bad |= !isfinite(X[e]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, kErrNonFinite);
}

// ---------------------------------------------------------------- launchers
static int grid_for(int64_t n, int threads) {
    return static_cast<int>((n + threads - 1) / threads);
}

cudaError_t launch_init_lists(int64_t N, int k, uint32_t stream, uint64_t seed, int32_t* out, cudaStream_t s) {
    init_lists_kernel<<<grid_for(N, 128), 128, 0, s>>>(N, k, stream, seed, out);
    return cudaGetLastError();
}

cudaError_t launch_hd_finalize(const FinalizeParams& f, int blocks, cudaStream_t s) {
    const size_t smem = static_cast<size_t>(8) * f.xpitch * sizeof(float);
    if (f.k_hd <= 32) {
        cudaFuncSetAttribute(hd_finalize_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        hd_finalize_kernel<1><<<blocks, 256, smem, s>>>(f);
    } else {
        cudaFuncSetAttribute(hd_finalize_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        hd_finalize_kernel<2><<<blocks, 256, smem, s>>>(f);
    }
    return cudaGetLastError();
}

// FP64 words of scratch launch_init_y needs: R (FP32, D4 x DP), mu (D), the
// moments (2 DP), the scale factors (FP32, DP) and up to 1024 blocks of
// column partials.
int64_t init_y_scratch_len(int D, int d, int DP) {
    (void)d;
    const int64_t D4 = (D + 3) / 4 * 4;
    const int64_t cols = D > DP ? D : DP;
    return (D4 * DP + 1) / 2 + D + 2 * DP + (DP + 1) / 2 + 1024 * cols;
}

cudaError_t launch_init_y(const float* X32, int64_t N, int D, int xpitch, int d, int DP, uint64_t seed,
                          uint32_t ctr, float* Y, double* scratch, int64_t scratch_len, cudaStream_t s) {
    // scratch layout: R (FP32, D4 x DP) | mu (D) | mean, var (DP each) |
    // scale factors (FP32, DP) | partials
    const int n4 = (D + 3) / 4, D4 = 4 * n4;
    float* R = reinterpret_cast<float*>(scratch);
    double* mu = scratch + (static_cast<int64_t>(D4) * DP + 1) / 2;
    double* mean = mu + D;
    double* var = mean + DP;
    float* sc = reinterpret_cast<float*>(var + DP);
    double* part = var + DP + (DP + 1) / 2;
    const int64_t avail = scratch_len - (part - scratch);
    const int cols = D > DP ? D : DP;
    int nb = static_cast<int>(avail / cols);
    if (nb > 1024) nb = 1024;
    if (nb < 1) return cudaErrorInvalidValue;
    const int64_t rpb = (N + nb - 1) / nb;
    nb = static_cast<int>((N + rpb - 1) / rpb);
    gauss_matrix_kernel<<<grid_for(static_cast<int64_t>(D4) * DP, 128), 128, 0, s>>>(D, D4, d, DP, ctr, seed, R);
    col_sums_kernel<<<nb, 256, 0, s>>>(X32, N, D, xpitch, rpb, nullptr, 0, part);
    reduce_parts_kernel<<<grid_for(D, 128), 128, 0, s>>>(part, nb, D, 1.0 / static_cast<double>(N), mu);
    const size_t psmem = static_cast<size_t>(D4) * sizeof(float);
    switch (DP) {
        case 2: project_kernel<2><<<grid_for(N, 128), 128, psmem, s>>>(X32, N, D, n4, xpitch, mu, R, Y); break;
        case 4: project_kernel<4><<<grid_for(N, 128), 128, psmem, s>>>(X32, N, D, n4, xpitch, mu, R, Y); break;
        case 8: project_kernel<8><<<grid_for(N, 128), 128, psmem, s>>>(X32, N, D, n4, xpitch, mu, R, Y); break;
        case 16: project_kernel<16><<<grid_for(N, 128), 128, psmem, s>>>(X32, N, D, n4, xpitch, mu, R, Y); break;
        case 32: project_kernel<32><<<grid_for(N, 128), 128, psmem, s>>>(X32, N, D, n4, xpitch, mu, R, Y); break;
        default: return cudaErrorInvalidValue;
    }
    col_sums_kernel<<<nb, 256, 0, s>>>(Y, N, DP, DP, rpb, nullptr, 0, part);
    reduce_parts_kernel<<<grid_for(DP, 128), 128, 0, s>>>(part, nb, DP, 1.0 / static_cast<double>(N), mean);
    col_sums_kernel<<<nb, 256, 0, s>>>(Y, N, DP, DP, rpb, mean, 1, part);
    reduce_parts_kernel<<<grid_for(DP, 128), 128, 0, s>>>(part, nb, DP, 1.0 / static_cast<double>(N), var);
    col_scale_kernel<<<1, 32, 0, s>>>(var, d, DP, kInitYStd, sc);
    scale_cols_kernel<<<grid_for(N * DP, 256), 256, 0, s>>>(Y, N * DP, DP, sc);
    return cudaGetLastError();
}

cudaError_t launch_zinit(const ZinitParams& z, int DP, int blocks, DevScalars* sc, cudaStream_t s) {
    switch (DP) {
        case 2: zinit_kernel<2><<<blocks, 256, 0, s>>>(z); break;
        case 4: zinit_kernel<4><<<blocks, 256, 0, s>>>(z); break;
        case 8: zinit_kernel<8><<<blocks, 256, 0, s>>>(z); break;
        case 16: zinit_kernel<16><<<blocks, 256, 0, s>>>(z); break;
        case 32: zinit_kernel<32><<<blocks, 256, 0, s>>>(z); break;
        default: return cudaErrorInvalidValue;
    }
    zinit_finish_kernel<<<1, 32, 0, s>>>(z.part, blocks, sc);
    return cudaGetLastError();
}

cudaError_t launch_quantize(const float* X32, int64_t N, int D, int xpitch, int precision, int qpitch,
                            int scale_off, uint8_t* Q, cudaStream_t s) {
    if (precision == 1)
        quantize_bf16_kernel<<<grid_for(N * 32, 256), 256, 0, s>>>(X32, N, D, xpitch, qpitch, scale_off, Q);
    else
        quantize_fp8_kernel<<<grid_for(N * 32, 256), 256, 0, s>>>(X32, N, D, xpitch, qpitch, scale_off, Q);
    return cudaGetLastError();
}

cudaError_t launch_check_lists(const int32_t* idx, int64_t N, int k, uint32_t* err, cudaStream_t s) {
    check_lists_kernel<<<grid_for(N, 128), 128, 0, s>>>(idx, N, k, err);
    return cudaGetLastError();
}

cudaError_t launch_check_finite(const float* X, int64_t n, uint32_t* err, cudaStream_t s) {
    int blocks = grid_for(n, 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    check_finite_kernel<<<blocks, 256, 0, s>>>(X, n, err);
    return cudaGetLastError();
}

}  // namespace fsne
