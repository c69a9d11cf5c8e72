// Host-side launchers of the FUnc-SNE kernels (one declaration per kernel
// family; definitions live next to the kernels).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "params.h"

namespace fsne {

struct FinalizeParams {
    int64_t N;
    int32_t k_hd, n4, xpitch;
    int32_t g;        // lanes per FP32 row (the iteration's grouping)
    float log_perp;
    const float* X32;
    int32_t* idx;     // N x k_hd, sorted in place
    float* d2;        // N x k_hd out
    float* P;         // N x k_hd out
    float* beta;      // N out (cold start only)
    const float* Pin; // imported P (aligned with idx before sorting) or NULL
};

struct ZinitParams {
    int64_t N;
    int32_t k_hd, k_ld, n_neg;
    float alpha, inv_alpha, neg_scale;
    uint32_t t, stream;
    uint64_t seed;
    const float* Y;
    const int32_t* hd_idx;
    const int32_t* ld_idx;
    double* part;
};

struct KnnParams {
    int64_t N;
    int32_t n4, xpitch, k, n_split, RK;
    int64_t n_q;
    const float* X32;
    const int32_t* queries;
    unsigned long long* part;  // n_q x n_split x (32*RK) keys
    int32_t* idx;              // n_q x k
    float* d2;                 // n_q x k
};

struct InsertParams {
    int64_t N, n_old;
    int32_t k_hd, k_ld, n4, xpitch;
    int32_t g;         // lanes per FP32 row (the iteration's grouping)
    int32_t rounds;    // neighbour-of-neighbour rounds (slots 64 + 32 r + s)
    float log_perp;
    uint32_t t;
    uint64_t seed;
    const float* X32;
    float* Y;
    float* V;
    float* A;
    float* R;
    int32_t* hd_idx;   // current HD buffer (rows of existing points are read)
    float* hd_d2;
    int32_t* ld_idx;   // current LD buffer
    float* P;
    float* beta;
};

// phase kernels of the iteration (HD refinement: one translation unit per
// HD storage precision)
cudaError_t hd_refine_launch_f32(const StepParams& p, int RH, int G, int blocks, size_t smem, cudaStream_t s);
cudaError_t hd_refine_launch_bf16(const StepParams& p, int RH, int G, int blocks, size_t smem, cudaStream_t s);
cudaError_t hd_refine_launch_fp8(const StepParams& p, int RH, int G, int blocks, size_t smem, cudaStream_t s);
int hd_refine_occupancy_f32(int RH, int G, bool pf, size_t smem);
int hd_refine_occupancy_bf16(int RH, int G, bool pf, size_t smem);
int hd_refine_occupancy_fp8(int RH, int G, bool pf, size_t smem);
cudaError_t ld_refine_launch(const StepParams& p, int DP, int RH, bool pair, int blocks, size_t smem, cudaStream_t s);
cudaError_t forces_launch(const StepParams& p, int DP, int RH, int CW, int blocks, size_t smem, cudaStream_t s);
int ld_refine_occupancy(int DP, int RH, bool pair, size_t smem);
int forces_occupancy(int DP, int RH, int CW, size_t smem);
// copy of the insertion window's new HD lists into the current buffer
// (iterations that refined only the window)
cudaError_t fresh_lists_launch(const StepParams& p, int blocks, cudaStream_t s);
// forces with the row-pair layout (DP = 8, 16 or 32)
cudaError_t forces_pair_launch(const StepParams& p, int DP, int RH, int blocks, size_t smem, cudaStream_t s);
int forces_pair_occupancy(int DP, int RH, size_t smem);
cudaError_t update_launch(const UpdateParams& u, int blocks, cudaStream_t s);

// set-up
cudaError_t launch_init_lists(int64_t N, int k, uint32_t stream, uint64_t seed, int32_t* out, cudaStream_t s);
cudaError_t launch_hd_finalize(const FinalizeParams& f, int blocks, cudaStream_t s);
int64_t init_y_scratch_len(int D, int d, int DP);
cudaError_t launch_init_y(const float* X32, int64_t N, int D, int xpitch, int d, int DP, uint64_t seed,
                          uint32_t ctr, float* Y, double* scratch, int64_t scratch_len, cudaStream_t s);
cudaError_t launch_zinit(const ZinitParams& z, int DP, int blocks, DevScalars* sc, cudaStream_t s);
cudaError_t launch_quantize(const float* X32, int64_t N, int D, int xpitch, int precision, int qpitch,
                            int scale_off, uint8_t* Q, cudaStream_t s);
cudaError_t launch_check_lists(const int32_t* idx, int64_t N, int k, uint32_t* err, cudaStream_t s);
cudaError_t launch_check_finite(const float* X, int64_t n, uint32_t* err, cudaStream_t s);
// live changes of the point set (live_kernels.cu)
// dst[r, c] = src[r, c] for r < rows, c < cols; pitches in 4-byte words.
cudaError_t launch_repack_rows(void* dst, int64_t dpitch, const void* src, int64_t spitch, int64_t rows,
                               int64_t cols, cudaStream_t s);
cudaError_t launch_gather_rows(uint32_t* dst, const uint32_t* src, int64_t pitch, const int32_t* old,
                               int64_t n_rows, cudaStream_t s);
cudaError_t launch_scatter_rows(float* X32, int xpitch, const int64_t* ids, const float* rows, int64_t n, int D,
                                cudaStream_t s);
cudaError_t launch_scale_rows(float* Y, float* V, int64_t n_elem, float factor, cudaStream_t s);
cudaError_t launch_remap_lists(int32_t* list, int k, const int32_t* new_of, int64_t N, uint32_t t, uint64_t seed,
                               uint32_t salt, cudaStream_t s);
cudaError_t launch_ld_distances(const float* Y, const int32_t* idx, int64_t N, int k, int DP, float* d2,
                                cudaStream_t s);

cudaError_t launch_insert(const InsertParams& q, int DP, cudaStream_t s);

struct MlpParams {
    int64_t N;                  // points the batches are drawn from
    int32_t B, D, H, d, DP, xpitch;
    int64_t n_params;
    uint64_t seed;
    float lr, beta1, beta2, eps;
    const float* X32;
    const float* Y;
    const float* mu;            // D
    const float* sigma;         // D
    float* theta;               // FP32 master parameters (flat)
    float* m;
    float* v;
    float* grad;
    __nv_bfloat16* wb;          // bfloat16 copy of theta
    int32_t* idx;               // B batch indices
    float* T;                   // B x d targets (scaled)
    __nv_bfloat16* Xb;          // B x D inputs
    __nv_bfloat16* H1;          // B x H
    __nv_bfloat16* H2;          // B x H
    __nv_bfloat16* G3;          // B x d
    __nv_bfloat16* G2;          // B x H
    __nv_bfloat16* G1;          // B x H
    float* O;                   // B x d outputs
    double* part;               // reduction partials
    float* ws;                  // split-K slices of the weight gradients
    uint32_t* err;              // device error word (kErrTimeout)
    int64_t ws_floats;
    double* loss;               // device scalar
    float* scale;               // device scalar: RMS of the last batch's targets
    uint32_t* step;             // device scalar: Adam steps taken
};

cudaError_t launch_mlp_stats(const float* X, int64_t N, int D, int xpitch, float* mu, float* sigma, cudaStream_t s);
cudaError_t launch_mlp_init(float* theta, __nv_bfloat16* wb, int D, int H, int d, uint64_t seed, cudaStream_t s);
cudaError_t launch_mlp_train_step(const MlpParams& q, cudaStream_t s);
cudaError_t launch_mlp_place(const MlpParams& q, const float* X, int xpitch, int64_t first, int64_t rows, float* Y,
                             int DP, cudaStream_t s);
cudaError_t launch_bf16_to_f32(const __nv_bfloat16* in, int64_t n, float* out, cudaStream_t s);
cudaError_t launch_bounded_wait(uint32_t* err, uint32_t polls, cudaStream_t s);

// evaluation
cudaError_t launch_exact_knn(const KnnParams& kp, cudaStream_t s);

}  // namespace fsne
