// Host runtime behind the C ABI of include/funcsne.h: the handle, argument
// checks, device memory layout, CUDA-graph replay of the iteration, and the
// copy-in / copy-out entry points.
//
// Device layout (N points, LD rows padded to DP = 2, 4, 8, 16 or 32 floats):
//   X32   N x xpitch FP32 (xpitch = D rounded up to 4; zero padding)
//   Xq    N x qpitch BF16 / FP8 copy (only in reduced-precision modes)
//   Y V A R  N x DP FP32 (element count rounded up to a multiple of 4)
//   hd_idx[2] hd_d2[2]  N x k_hd ping-pong lists;  ld_idx[2]  N x k_ld
//   P N x k_hd, beta N; DevScalars; per-block Z partials and counters.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/funcsne.h"
#include "launch.h"
#include "params.h"

using namespace fsne;

struct funcsne {
    int64_t N = 0;
    int64_t cap = 0;  // rows allocated (N <= cap; rows beyond N are zero)
    int32_t D = 0, d = 0, DP = 0, k_hd = 0, k_ld = 0, n_neg = 0, RH = 1;
    float alpha = 1.f, perplexity = 30.f;
    uint64_t seed = 0;
    // options
    double lr = 200.0, momentum = 0.8, att = 1.0, rep = 1.0, exaggeration = 1.0;
    int32_t exag_iters = 0, hd_mode = kHdAdaptive, precision = FUNCSNE_FP32;
    double coin_floor = kCoinFloor, gamma_e = kGammaE, gamma_z = kGammaZ;
    // layout
    int32_t xpitch = 0, n4 = 0, xs_floats = 0, qpitch = 0, nq = 0, qscale_off = 0;
    int64_t yelem = 0;
    // device memory
    float* X32 = nullptr;
    uint8_t* Xq = nullptr;
    float *Y = nullptr, *V = nullptr, *A = nullptr, *R = nullptr;
    int32_t* hd_idx[2] = {nullptr, nullptr};
    float* hd_d2[2] = {nullptr, nullptr};
    int32_t* ld_idx[2] = {nullptr, nullptr};
    float *P = nullptr, *beta = nullptr;
    DevScalars* sc = nullptr;
    double* zpart = nullptr;
    unsigned long long* cnt = nullptr;
    int32_t max_blocks = 0;
    // execution
    cudaStream_t own_stream = nullptr;
    cudaStream_t side_stream = nullptr;  // second branch of the captured iteration
    // asynchronous read-out of the embedding: a device snapshot of Y, copied
    // out on copy_stream while the next iterations run
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t snap_ev = nullptr, copy_ev = nullptr;
    float* Ysnap = nullptr;
    int64_t snap_rows = 0;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    bool concurrent = false;  // run the two refinements side by side in the graph
    int32_t forces_cw = 8;    // floats of an LD row per lane in the forces kernel
    int32_t forces_pair = 1;  // the row-pair layout of the forces (rows of 8+ floats)
    int32_t ld_pair = 1;      // the row-pair layout of the LD refinement's distances
    int32_t hd_prefetch = 1;  // HD refinement pipelined over the points of a warp (option)
    int32_t fresh_iters = 0;  // iterations an inserted point is refined for, whatever the coin
    int32_t hd_pf_used = 0;   // ... in use: rows read by two lanes, room for four blocks
    int32_t hd_lanes_opt = 0; // lanes per gathered HD row (0: chosen from the row bytes)
    int32_t insert_rounds = 64; // neighbour-of-neighbour rounds of an insertion
    int32_t jump_iters = 0, jump_parts = 2;  // jump start by linear projections
    bool frozen = false;      // an iteration of the jump start: no gradient step
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    int hd_blocks = 0, ld_blocks = 0, fo_blocks = 0, update_blocks = 0;
    size_t hd_smem = 0, ld_smem = 0, fo_smem = 0;
    cudaGraphExec_t graph1 = nullptr, graph8 = nullptr;
    uint32_t t_host = 0;  // host mirror of the iteration counter
    // learned placement (MLP surrogate)
    int32_t mlp_H = 256, mlp_B = 4096, mlp_every = 10;
    float mlp_lr = 1e-3f;
    bool surrogate = false;
    uint32_t mlp_steps = 0;  // host mirror of the Adam step count
    struct {
        bool ready = false;
        int64_t n_params = 0;
        float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *mu = nullptr, *sigma = nullptr;
        __nv_bfloat16* wb = nullptr;
        int32_t* idx = nullptr;
        float *T = nullptr, *O = nullptr, *scale = nullptr;
        __nv_bfloat16 *Xb = nullptr, *H1 = nullptr, *H2 = nullptr, *G3 = nullptr, *G2 = nullptr, *G1 = nullptr;
        double *part = nullptr, *loss = nullptr;
        uint32_t* step = nullptr;
        float* ws = nullptr;  // split-K slices of the weight gradients
        int64_t ws_floats = 0;
    } mlp;
    std::string err;
};

namespace {

thread_local std::string g_create_error;

int fail(funcsne* h, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h)
        h->err = buf;
    else
        g_create_error = buf;
    return code;
}

#define FSNE_CUDA(h, call)                                                                          \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return fail((h), e_ == cudaErrorMemoryAllocation ? FUNCSNE_E_OOM : FUNCSNE_E_CUDA,      \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);       \
    } while (0)

// Allocation-failure injection (funcsne_debug_fail_alloc): allocations left
// before one fails; -1: off.
int64_t g_fail_alloc_after = -1;

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    if (g_fail_alloc_after == 0) {
        g_fail_alloc_after = -1;
        return cudaErrorMemoryAllocation;
    }
    if (g_fail_alloc_after > 0) --g_fail_alloc_after;
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

int round_up(int v, int m) { return (v + m - 1) / m * m; }

// An NVTX range over the host side of an entry point (what a profiler's
// timeline shows for each call; inert without one attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

void drop_graphs(funcsne* h) {
    if (h->graph1) cudaGraphExecDestroy(h->graph1);
    if (h->graph8) cudaGraphExecDestroy(h->graph8);
    h->graph1 = h->graph8 = nullptr;
}

// Lanes per gathered HD row in the refinement: of the FP32 rows, or of the
// BF16 / FP8 rows in reduced-precision modes.
int hd_lanes(const funcsne* h) {
    if (h->hd_lanes_opt) return h->hd_lanes_opt;
    return lanes_per_row(h->precision == FUNCSNE_FP32 || h->qpitch == 0 ? 4 * h->xpitch : h->qpitch);
}

// Lanes per FP32 row: the FP32 path's grouping, which the exact re-rank of
// the reduced-precision modes repeats.
int hd_lanes_f32(const funcsne* h) {
    return h->hd_lanes_opt ? h->hd_lanes_opt : lanes_per_row(4 * h->xpitch);
}

StepParams step_params(const funcsne* h) {
    StepParams p{};
    p.N = h->N;
    p.k_hd = h->k_hd;
    p.k_ld = h->k_ld;
    p.n_neg = h->n_neg;
    p.n4 = h->n4;
    p.xpitch = h->xpitch;
    p.nq = h->nq;
    p.qpitch = h->qpitch;
    p.qscale_off = h->qscale_off;
    p.hd_mode = h->hd_mode;
    p.coin_p0 = h->coin_floor;
    p.coin_p1 = 1.0 - h->coin_floor;
    p.xs_floats = h->xs_floats;
    p.smem_per_warp = (h->hd_pf_used ? 2 : 1) * h->xs_floats * 4 + kHashSlots * 4;
    p.hd_prefetch = h->hd_pf_used;
    p.gf = hd_lanes_f32(h);
    p.ga = hd_lanes(h);
    p.alpha = h->alpha;
    p.inv_alpha = 1.f / h->alpha;
    p.inv2N = static_cast<float>(1.0 / (2.0 * static_cast<double>(h->N)));
    p.neg_scale = static_cast<float>(static_cast<double>(h->N - 1) / h->n_neg);
    p.log_perp = std::log(h->perplexity);
    const float gamma = static_cast<float>((h->xs_floats + 4) * std::ldexp(1.0, -24) * 1.01);
    p.q_gamma = gamma;
    p.seed = h->seed;
    p.pk = philox_keys(h->seed);
    p.X32 = h->X32;
    p.Xq = h->Xq;
    p.Y = h->Y;
    p.A = h->A;
    p.R = h->R;
    p.hd_idx0 = h->hd_idx[0];
    p.hd_idx1 = h->hd_idx[1];
    p.hd_d20 = h->hd_d2[0];
    p.hd_d21 = h->hd_d2[1];
    p.ld_idx0 = h->ld_idx[0];
    p.ld_idx1 = h->ld_idx[1];
    p.P = h->P;
    p.beta = h->beta;
    p.sc = h->sc;
    p.zpart = h->zpart;
    p.cnt = h->cnt;
    return p;
}

UpdateParams update_params(const funcsne* h, float* dbg_att, float* dbg_rep) {
    UpdateParams u{};
    u.n_elem = h->yelem;
    u.n_zpart = h->fo_blocks;
    u.n_cnt = h->hd_blocks;
    u.hd_mode = h->hd_mode;
    u.coin_p0 = h->coin_floor;
    u.coin_p1 = 1.0 - h->coin_floor;
    u.gamma_e = h->gamma_e;
    u.gamma_z = h->gamma_z;
    u.N = h->N;
    u.lr = h->frozen ? 0.f : static_cast<float>(h->lr);
    u.momentum = h->frozen ? 0.f : static_cast<float>(h->momentum);
    u.att = static_cast<float>(h->att);
    u.rep = static_cast<float>(h->rep);
    u.exaggeration = static_cast<float>(h->exaggeration);
    u.exag_iters = h->exag_iters;
    u.seed = h->seed;
    u.Y = h->Y;
    u.V = h->V;
    u.A = h->A;
    u.R = h->R;
    u.dbg_att = dbg_att;
    u.dbg_rep = dbg_rep;
    u.sc = h->sc;
    u.zpart = h->zpart;
    u.cnt = h->cnt;
    return u;
}

// The row-pair forces kernel runs fewer instructions only on rows of 8
// floats (measured on GB300: 0.166 against 0.180 ms on the 200,000-point
// swiss roll at d = 8; slower at d = 16 and 32, where its extra shuffles
// outweigh the halved cache-line wavefronts).
bool use_forces_pair(const funcsne* h) { return h->forces_pair && h->DP == 8; }
bool use_ld_pair(const funcsne* h) { return h->ld_pair && h->DP >= 8; }

// The phase kernels of one iteration: 0 HD refinement, 1 LD refinement,
// 2 forces, 3 update.
constexpr int kPhases = 4;

cudaError_t launch_phase(const funcsne* h, int phase, const StepParams& p, cudaStream_t s) {
    switch (phase) {
        case 0:
            switch (h->precision) {
                case FUNCSNE_FP32: return hd_refine_launch_f32(p, h->RH, p.ga, h->hd_blocks, h->hd_smem, s);
                case FUNCSNE_BF16: return hd_refine_launch_bf16(p, h->RH, p.ga, h->hd_blocks, h->hd_smem, s);
                default: return hd_refine_launch_fp8(p, h->RH, p.ga, h->hd_blocks, h->hd_smem, s);
            }
        case 1: return ld_refine_launch(p, h->DP, h->RH, use_ld_pair(h), h->ld_blocks, h->ld_smem, s);
        case 2: {
            // the insertion window's lists first (a no-op outside window-only iterations)
            const cudaError_t e = fresh_lists_launch(p, h->update_blocks, s);
            if (e != cudaSuccess) return e;
            if (use_forces_pair(h)) return forces_pair_launch(p, h->DP, h->RH, h->fo_blocks, h->fo_smem, s);
            return forces_launch(p, h->DP, h->RH, h->forces_cw, h->fo_blocks, h->fo_smem, s);
        }
        default: return update_launch(update_params(h, nullptr, nullptr), h->update_blocks, s);
    }
}

// Persistent grids: resident blocks per SM x SMs, at most one warp per point.
int grid_for_occupancy(const funcsne* h, int occ) {
    if (occ < 1) occ = 1;
    int64_t blocks = static_cast<int64_t>(occ) * h->num_sms;
    const int64_t need = (h->N + 7) / 8;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    if (blocks > h->max_blocks) blocks = h->max_blocks;
    return static_cast<int>(blocks);
}

int configure_step(funcsne* h) {
    auto hd_occ = [&](bool pf, size_t smem) {
        switch (h->precision) {
            case FUNCSNE_FP32: return hd_refine_occupancy_f32(h->RH, hd_lanes(h), pf, smem);
            case FUNCSNE_BF16: return hd_refine_occupancy_bf16(h->RH, hd_lanes(h), pf, smem);
            default: return hd_refine_occupancy_fp8(h->RH, hd_lanes(h), pf, smem);
        }
    };
    const size_t smem1 = static_cast<size_t>(8) * (h->xs_floats * 4 + kHashSlots * 4);
    const size_t smem2 = static_cast<size_t>(8) * (2 * h->xs_floats * 4 + kHashSlots * 4);
    // Pipelining pays where two lanes read a gathered row (rows up to 224
    // bytes). Measured on GB300, HD refinement per iteration: 1M points at
    // D = 50, FP32 1.228 to 1.133 ms, BF16 1.231 to 1.190 ms; 200,000
    // points at D = 128 with FP8 rows 0.501 to 0.471 ms. Rows read by four
    // or eight lanes gained at most 1% or lost (FP32 at D = 128: 0.319 to
    // 0.412 ms). The kernel is built for four resident blocks; rows whose two
    // buffers leave room for fewer run the single-buffer kernel.
    h->hd_pf_used = h->hd_prefetch && hd_lanes(h) <= 2 && hd_occ(true, smem2) >= 4 ? 1 : 0;
    h->hd_smem = h->hd_pf_used ? smem2 : smem1;
    h->ld_smem = static_cast<size_t>(8) * kHashSlots * 4;
    h->fo_smem = static_cast<size_t>(8) * (kForceHashSlots + (use_forces_pair(h) ? kRepRing : 0)) * 4;
    const int occ = hd_occ(h->hd_pf_used != 0, h->hd_smem);
    // the two refinements share the SMs when they run side by side
    const int ld_occ = ld_refine_occupancy(h->DP, h->RH, use_ld_pair(h), h->ld_smem);
    h->hd_blocks = grid_for_occupancy(h, h->concurrent ? (occ + 1) / 2 : occ);
    h->ld_blocks = grid_for_occupancy(h, h->concurrent ? (ld_occ + 1) / 2 : ld_occ);
    h->fo_blocks = grid_for_occupancy(h, use_forces_pair(h) ? forces_pair_occupancy(h->DP, h->RH, h->fo_smem)
                                                            : forces_occupancy(h->DP, h->RH, h->forces_cw, h->fo_smem));
    int64_t ub = (h->yelem / 4 + 255) / 256;
    if (ub > 4L * h->num_sms) ub = 4L * h->num_sms;
    if (ub < 1) ub = 1;
    h->update_blocks = static_cast<int>(ub);
    drop_graphs(h);
    return FUNCSNE_OK;
}

int enqueue_iteration(funcsne* h, cudaStream_t s, float* dbg_att, float* dbg_rep) {
    const StepParams p = step_params(h);
    for (int ph = 0; ph < 3; ++ph) FSNE_CUDA(h, launch_phase(h, ph, p, s));
    FSNE_CUDA(h, update_launch(update_params(h, dbg_att, dbg_rep), h->update_blocks, s));
    return FUNCSNE_OK;
}

int build_graph(funcsne* h, int iters, cudaGraphExec_t* out) {
    // capture on the handle's own stream; the graph may then run on any stream
    cudaGraph_t g = nullptr;
    FSNE_CUDA(h, cudaStreamBeginCapture(h->own_stream, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < iters; ++k) {
        const StepParams p = step_params(h);
        cudaError_t e = cudaSuccess;
        if (h->concurrent) {
            // fork: HD refinement here, LD refinement on the side stream; join before the forces
            e = cudaEventRecord(h->fork_ev, h->own_stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(h->side_stream, h->fork_ev, 0);
            if (e == cudaSuccess) e = launch_phase(h, 0, p, h->own_stream);
            if (e == cudaSuccess) e = launch_phase(h, 1, p, h->side_stream);
            if (e == cudaSuccess) e = cudaEventRecord(h->join_ev, h->side_stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(h->own_stream, h->join_ev, 0);
            for (int ph = 2; ph < kPhases && e == cudaSuccess; ++ph) e = launch_phase(h, ph, p, h->own_stream);
        } else {
            for (int ph = 0; ph < kPhases && e == cudaSuccess; ++ph) e = launch_phase(h, ph, p, h->own_stream);
        }
        if (e != cudaSuccess) {
            cudaStreamEndCapture(h->own_stream, &g);
            if (g) cudaGraphDestroy(g);
            return fail(h, FUNCSNE_E_CUDA, "graph capture: %s", cudaGetErrorString(e));
        }
    }
    FSNE_CUDA(h, cudaStreamEndCapture(h->own_stream, &g));
    cudaError_t e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    FSNE_CUDA(h, e);
    return FUNCSNE_OK;
}

int read_scalars(funcsne* h, DevScalars* out) {
    FSNE_CUDA(h, cudaMemcpyAsync(out, h->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h->stream));
    FSNE_CUDA(h, cudaStreamSynchronize(h->stream));
    return FUNCSNE_OK;
}

bool is_device_memory(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Copy `rows` rows of `cols` 4-byte elements between arrays of pitches
// dst_pitch and src_pitch (elements), either side in host or device memory.
// The copy engines move a pitched copy to or from host memory row by row:
// rows of a few hundred bytes go at about 7 GB/s, one contiguous block at
// about 200 GB/s (pinned memory, GB300). So a pitched copy with a host side
// goes through a contiguous device staging buffer (stream-ordered
// allocation) and the repacking kernel.
cudaError_t copy_rows_raw(void* dst, size_t dst_pitch, const void* src, size_t src_pitch, int64_t rows, size_t cols,
                          cudaStream_t s) {
    if (rows <= 0 || cols == 0) return cudaSuccess;
    const size_t bytes = static_cast<size_t>(rows) * cols * 4;
    if (dst_pitch == cols && src_pitch == cols) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s);
    const bool dd = is_device_memory(dst), sd = is_device_memory(src);
    if (dd && sd) return launch_repack_rows(dst, dst_pitch, src, src_pitch, rows, cols, s);
    if (!dd && !sd)
        return cudaMemcpy2DAsync(dst, dst_pitch * 4, src, src_pitch * 4, cols * 4, static_cast<size_t>(rows),
                                 cudaMemcpyDefault, s);
    void* stage = nullptr;
    cudaError_t e = cudaMallocAsync(&stage, bytes, s);
    if (e != cudaSuccess) return e;
    if (sd) {
        e = launch_repack_rows(stage, cols, src, src_pitch, rows, cols, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, stage, bytes, cudaMemcpyDefault, s);
    } else {
        e = cudaMemcpyAsync(stage, src, bytes, cudaMemcpyDefault, s);
        if (e == cudaSuccess) e = launch_repack_rows(dst, dst_pitch, stage, cols, rows, cols, s);
    }
    const cudaError_t e2 = cudaFreeAsync(stage, s);
    return e != cudaSuccess ? e : e2;
}

// Copy an N x cols row-major array between a caller buffer (pitch cols) and
// a device array of pitch `dpitch` elements.
template <typename T>
int copy_rows(funcsne* h, T* dst, size_t dst_pitch, const T* src, size_t src_pitch, int64_t rows, size_t cols) {
    static_assert(sizeof(T) == 4, "rows of 4-byte elements");
    FSNE_CUDA(h, copy_rows_raw(dst, dst_pitch, src, src_pitch, rows, cols, h->stream));
    return FUNCSNE_OK;
}

void free_all(funcsne* h) {
    drop_graphs(h);
    cudaFree(h->X32);
    cudaFree(h->Xq);
    cudaFree(h->Y);
    cudaFree(h->V);
    cudaFree(h->A);
    cudaFree(h->R);
    for (int b = 0; b < 2; ++b) {
        cudaFree(h->hd_idx[b]);
        cudaFree(h->hd_d2[b]);
        cudaFree(h->ld_idx[b]);
    }
    cudaFree(h->P);
    cudaFree(h->beta);
    cudaFree(h->sc);
    cudaFree(h->zpart);
    cudaFree(h->cnt);
    auto& q = h->mlp;
    for (void* p : {static_cast<void*>(q.theta), static_cast<void*>(q.m), static_cast<void*>(q.v),
                    static_cast<void*>(q.grad), static_cast<void*>(q.mu), static_cast<void*>(q.sigma),
                    static_cast<void*>(q.wb), static_cast<void*>(q.idx), static_cast<void*>(q.T),
                    static_cast<void*>(q.O), static_cast<void*>(q.scale), static_cast<void*>(q.Xb),
                    static_cast<void*>(q.H1), static_cast<void*>(q.H2), static_cast<void*>(q.G3),
                    static_cast<void*>(q.G2), static_cast<void*>(q.G1), static_cast<void*>(q.part), static_cast<void*>(q.ws),
                    static_cast<void*>(q.loss), static_cast<void*>(q.step)})
        cudaFree(p);
    if (h->copy_stream) cudaStreamSynchronize(h->copy_stream);
    cudaFree(h->Ysnap);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    if (h->snap_ev) cudaEventDestroy(h->snap_ev);
    if (h->copy_ev) cudaEventDestroy(h->copy_ev);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    if (h->side_stream) cudaStreamDestroy(h->side_stream);
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    if (h->join_ev) cudaEventDestroy(h->join_ev);
}

int quantize(funcsne* h) {
    cudaFree(h->Xq);
    h->Xq = nullptr;
    if (h->precision == FUNCSNE_FP32) {
        h->qpitch = h->nq = h->qscale_off = 0;
        return FUNCSNE_OK;
    }
    if (h->precision == FUNCSNE_BF16) {
        // data chunks, then a 16-byte chunk holding the row-error bound
        h->nq = (2 * h->D + 15) / 16;
        h->qscale_off = 16 * h->nq;
        h->qpitch = h->qscale_off + 16;
    } else {
        // code words, then the row-error bound and the scale in the last 8 bytes
        const int nw = (h->D + 3) / 4;
        h->qpitch = round_up(4 * nw + 8, 16);
        h->nq = nw;
        h->qscale_off = h->qpitch - 4;
    }
    // sized for the capacity: insertions below it write rows N .. cap - 1
    FSNE_CUDA(h, dalloc(&h->Xq, static_cast<size_t>(h->cap) * h->qpitch));
    FSNE_CUDA(h, cudaMemsetAsync(h->Xq, 0, static_cast<size_t>(h->cap) * h->qpitch, h->stream));
    FSNE_CUDA(h, launch_quantize(h->X32, h->N, h->D, h->xpitch, h->precision, h->qpitch, h->qscale_off, h->Xq,
                                 h->stream));
    return FUNCSNE_OK;
}

int check_errors(funcsne* h) {
    DevScalars s;
    int rc = read_scalars(h, &s);
    if (rc) return rc;
    if (s.err & kErrIndex) return fail(h, FUNCSNE_E_RANGE, "device index check failed (error word 0x%x)", s.err);
    if (s.err & kErrNonFinite) return fail(h, FUNCSNE_E_NAN, "non-finite values (error word 0x%x)", s.err);
    if (s.err & kErrTimeout) return fail(h, FUNCSNE_E_CUDA, "a device wait timed out (error word 0x%x)", s.err);
    return FUNCSNE_OK;
}

int clear_error_word(funcsne* h) {
    FSNE_CUDA(h, cudaMemsetAsync(&h->sc->err, 0, sizeof(uint32_t), h->stream));
    return FUNCSNE_OK;
}

ZinitParams zinit_params(const funcsne* h, const int32_t* hd, const int32_t* ld, double* part) {
    ZinitParams z{};
    z.N = h->N;
    z.k_hd = h->k_hd;
    z.k_ld = h->k_ld;
    z.n_neg = h->n_neg;
    z.alpha = h->alpha;
    z.inv_alpha = 1.f / h->alpha;
    z.neg_scale = static_cast<float>(static_cast<double>(h->N - 1) / h->n_neg);
    z.t = 0;
    z.stream = kStreamZinit;
    z.seed = h->seed;
    z.Y = h->Y;
    z.hd_idx = hd;
    z.ld_idx = ld;
    z.part = part;
    return z;
}

MlpParams mlp_params(const funcsne* h) {
    const auto& q = h->mlp;
    MlpParams p{};
    p.N = h->N;
    p.B = h->mlp_B;
    p.D = h->D;
    p.H = h->mlp_H;
    p.d = h->d;
    p.DP = h->DP;
    p.xpitch = h->xpitch;
    p.n_params = q.n_params;
    p.seed = h->seed;
    p.lr = h->mlp_lr;
    p.beta1 = 0.9f;
    p.beta2 = 0.999f;
    p.eps = 1e-8f;
    p.X32 = h->X32;
    p.Y = h->Y;
    p.mu = q.mu;
    p.sigma = q.sigma;
    p.theta = q.theta;
    p.m = q.m;
    p.v = q.v;
    p.grad = q.grad;
    p.wb = q.wb;
    p.idx = q.idx;
    p.T = q.T;
    p.Xb = q.Xb;
    p.H1 = q.H1;
    p.H2 = q.H2;
    p.G3 = q.G3;
    p.G2 = q.G2;
    p.G1 = q.G1;
    p.O = q.O;
    p.part = q.part;
    p.ws = q.ws;
    p.ws_floats = q.ws_floats;
    p.err = &h->sc->err;
    p.loss = q.loss;
    p.scale = q.scale;
    p.step = q.step;
    return p;
}

// Allocate and initialise the surrogate on first use: input statistics of
// the current points, initial parameters, zero moments.
int ensure_mlp(funcsne* h) {
    auto& q = h->mlp;
    if (q.ready) return FUNCSNE_OK;
    const int64_t D = h->D, H = h->mlp_H, d = h->d, B = h->mlp_B;
    q.n_params = H * D + H + H * H + H + d * H + d;
    FSNE_CUDA(h, dalloc(&q.theta, q.n_params));
    FSNE_CUDA(h, dalloc(&q.m, q.n_params));
    FSNE_CUDA(h, dalloc(&q.v, q.n_params));
    FSNE_CUDA(h, dalloc(&q.grad, q.n_params));
    FSNE_CUDA(h, dalloc(&q.wb, q.n_params));
    FSNE_CUDA(h, dalloc(&q.mu, D));
    FSNE_CUDA(h, dalloc(&q.sigma, D));
    FSNE_CUDA(h, dalloc(&q.idx, B));
    FSNE_CUDA(h, dalloc(&q.T, B * d));
    FSNE_CUDA(h, dalloc(&q.O, B * d));
    FSNE_CUDA(h, dalloc(&q.Xb, B * D));
    FSNE_CUDA(h, dalloc(&q.H1, B * H));
    FSNE_CUDA(h, dalloc(&q.H2, B * H));
    FSNE_CUDA(h, dalloc(&q.G3, B * d));
    FSNE_CUDA(h, dalloc(&q.G2, B * H));
    FSNE_CUDA(h, dalloc(&q.G1, B * H));
    FSNE_CUDA(h, dalloc(&q.part, (B * d + 255) / 256 + (B + 255) / 256 + 8));
    {
        // up to 32 split-K slices of the largest weight gradient, 64 MB at most
        const int64_t per = std::max(std::max(H * H, H * D), d * H) + std::max(H, d);
        q.ws_floats = std::max<int64_t>(std::min<int64_t>(32 * per, int64_t(1) << 24), per);
        FSNE_CUDA(h, dalloc(&q.ws, q.ws_floats));
    }
    FSNE_CUDA(h, dalloc(&q.loss, 1));
    FSNE_CUDA(h, dalloc(&q.scale, 1));
    FSNE_CUDA(h, dalloc(&q.step, 1));
    FSNE_CUDA(h, cudaMemsetAsync(q.m, 0, q.n_params * sizeof(float), h->stream));
    FSNE_CUDA(h, cudaMemsetAsync(q.v, 0, q.n_params * sizeof(float), h->stream));
    FSNE_CUDA(h, cudaMemsetAsync(q.step, 0, sizeof(uint32_t), h->stream));
    FSNE_CUDA(h, cudaMemsetAsync(q.loss, 0, sizeof(double), h->stream));
    const float one = 1.f;
    FSNE_CUDA(h, cudaMemcpyAsync(q.scale, &one, sizeof(float), cudaMemcpyHostToDevice, h->stream));
    FSNE_CUDA(h, launch_mlp_stats(h->X32, h->N, h->D, h->xpitch, q.mu, q.sigma, h->stream));
    FSNE_CUDA(h, launch_mlp_init(q.theta, q.wb, h->D, h->mlp_H, h->d, h->seed, h->stream));
    FSNE_CUDA(h, cudaStreamSynchronize(h->stream));
    q.ready = true;
    h->mlp_steps = 0;
    return FUNCSNE_OK;
}

int mlp_train_now(funcsne* h, int n) {
    int rc = ensure_mlp(h);
    if (rc) return rc;
    const MlpParams q = mlp_params(h);
    for (int k = 0; k < n; ++k) {
        FSNE_CUDA(h, launch_mlp_train_step(q, h->stream));
        ++h->mlp_steps;
    }
    return FUNCSNE_OK;
}

// Reallocate every per-point array for new_cap rows (N rows kept, the rest zero).
int grow(funcsne* h, int64_t new_cap) {
    const int64_t N = h->N;
    // the arrays move one by one: graphs captured with the old addresses go
    // first, so a failure part-way (some arrays moved, h->cap unchanged,
    // every array still holding at least cap rows) leaves a usable handle
    drop_graphs(h);
    auto move = [&](auto** p, size_t row_elems) -> int {
        using T = std::remove_pointer_t<std::remove_reference_t<decltype(*p)>>;
        T* q = nullptr;
        FSNE_CUDA(h, dalloc(&q, static_cast<size_t>(new_cap) * row_elems));
        FSNE_CUDA(h, cudaMemsetAsync(q, 0, static_cast<size_t>(new_cap) * row_elems * sizeof(T), h->stream));
        if (*p) {
            FSNE_CUDA(h, cudaMemcpyAsync(q, *p, static_cast<size_t>(N) * row_elems * sizeof(T), cudaMemcpyDeviceToDevice,
                                         h->stream));
            FSNE_CUDA(h, cudaStreamSynchronize(h->stream));
            cudaFree(*p);
        }
        *p = q;
        return FUNCSNE_OK;
    };
    int rc;
    if ((rc = move(&h->X32, h->xpitch))) return rc;
    if (h->Xq && (rc = move(&h->Xq, h->qpitch))) return rc;
    // LD rows: DP floats each, plus one spare row so that the element count
    // rounded up to a multiple of 4 stays inside the allocation
    const int64_t spare = new_cap + 1;
    auto move_rows = [&](float** p) -> int {
        float* q = nullptr;
        FSNE_CUDA(h, dalloc(&q, static_cast<size_t>(spare) * h->DP));
        FSNE_CUDA(h, cudaMemsetAsync(q, 0, static_cast<size_t>(spare) * h->DP * sizeof(float), h->stream));
        FSNE_CUDA(h, cudaMemcpyAsync(q, *p, static_cast<size_t>(h->yelem) * sizeof(float), cudaMemcpyDeviceToDevice,
                                     h->stream));
        FSNE_CUDA(h, cudaStreamSynchronize(h->stream));
        cudaFree(*p);
        *p = q;
        return FUNCSNE_OK;
    };
    if ((rc = move_rows(&h->Y)) || (rc = move_rows(&h->V)) || (rc = move_rows(&h->A)) || (rc = move_rows(&h->R)))
        return rc;
    for (int b = 0; b < 2; ++b) {
        if ((rc = move(&h->hd_idx[b], h->k_hd))) return rc;
        if ((rc = move(&h->hd_d2[b], h->k_hd))) return rc;
        if ((rc = move(&h->ld_idx[b], h->k_ld))) return rc;
    }
    if ((rc = move(&h->P, h->k_hd))) return rc;
    if ((rc = move(&h->beta, 1))) return rc;
    h->cap = new_cap;
    return FUNCSNE_OK;
}

}  // namespace

namespace fsne {
// Message for funcsne_last_error(NULL) from entry points that have no handle.
void set_global_error(const char* msg) { g_create_error = msg; }
}  // namespace fsne

extern "C" {

int funcsne_create(const float* X, int64_t N, int32_t D, int32_t d, int32_t k_hd, int32_t k_ld, int32_t n_neg,
                   float alpha, float perplexity, uint64_t seed, funcsne_t** out) {
    NvtxRange nvtx_range("funcsne_create");
    if (!out) return fail(nullptr, FUNCSNE_E_ARG, "out is NULL");
    *out = nullptr;
    if (!X) return fail(nullptr, FUNCSNE_E_ARG, "X is NULL");
    if (D < 1 || D > 4096) return fail(nullptr, FUNCSNE_E_ARG, "D must be in [1, 4096] (got %d)", D);
    if (d < 1 || d > 32) return fail(nullptr, FUNCSNE_E_ARG, "d must be in [1, 32] (got %d)", d);
    if (k_hd < 2 || k_hd > 64) return fail(nullptr, FUNCSNE_E_ARG, "k_hd must be in [2, 64] (got %d)", k_hd);
    if (k_ld < 1 || k_ld > 32) return fail(nullptr, FUNCSNE_E_ARG, "k_ld must be in [1, 32] (got %d)", k_ld);
    if (N <= k_hd || N <= k_ld || N >= (int64_t(1) << 31) - 1)
        return fail(nullptr, FUNCSNE_E_ARG, "N must exceed k_hd and k_ld and be < 2^31 - 1 (got %lld)",
                    static_cast<long long>(N));
    if (n_neg < 1 || n_neg > 1024) return fail(nullptr, FUNCSNE_E_ARG, "n_neg must be in [1, 1024]");
    if (!(alpha > 0.f) || !std::isfinite(alpha)) return fail(nullptr, FUNCSNE_E_ARG, "alpha must be > 0");
    if (!(perplexity > 1.f) || !(perplexity < static_cast<float>(k_hd) + 1.f))
        return fail(nullptr, FUNCSNE_E_ARG, "perplexity must be in (1, k_hd + 1)");

    funcsne* h = new funcsne();
    h->N = N;
    h->D = D;
    h->d = d;
    h->DP = d <= 2 ? 2 : d <= 4 ? 4 : d <= 8 ? 8 : d <= 16 ? 16 : 32;
    h->k_hd = k_hd;
    h->k_ld = k_ld;
    h->n_neg = n_neg;
    h->RH = k_hd <= 32 ? 1 : 2;
    h->alpha = alpha;
    h->perplexity = perplexity;
    h->seed = seed;
    h->lr = std::fmax(static_cast<double>(N) / 12.0, 200.0);
    h->xpitch = round_up(D, 4);
    h->n4 = h->xpitch / 4;
    h->xs_floats = round_up(D, 16);
    h->yelem = (N * h->DP + 3) / 4 * 4;
    h->cap = N;

    auto bail = [&](int rc) {
        g_create_error = h->err;
        free_all(h);
        delete h;
        return rc;
    };
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        fail(h, FUNCSNE_E_CUDA, "no CUDA device available");
        return bail(FUNCSNE_E_CUDA);
    }
    h->max_blocks = 64 * h->num_sms;
#define CREATE_CUDA(call)                                                                           \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) {                                                                    \
            fail(h, e_ == cudaErrorMemoryAllocation ? FUNCSNE_E_OOM : FUNCSNE_E_CUDA, "%s: %s", #call, \
                 cudaGetErrorString(e_));                                                           \
            return bail(e_ == cudaErrorMemoryAllocation ? FUNCSNE_E_OOM : FUNCSNE_E_CUDA);          \
        }                                                                                           \
    } while (0)
    CREATE_CUDA(cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking));
    CREATE_CUDA(cudaStreamCreateWithFlags(&h->side_stream, cudaStreamNonBlocking));
    CREATE_CUDA(cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming));
    CREATE_CUDA(cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming));
    h->stream = h->own_stream;
    const size_t nk_hd = static_cast<size_t>(N) * k_hd, nk_ld = static_cast<size_t>(N) * k_ld;
    CREATE_CUDA(dalloc(&h->X32, static_cast<size_t>(N) * h->xpitch));
    CREATE_CUDA(dalloc(&h->Y, h->yelem));
    CREATE_CUDA(dalloc(&h->V, h->yelem));
    CREATE_CUDA(dalloc(&h->A, h->yelem));
    CREATE_CUDA(dalloc(&h->R, h->yelem));
    for (int b = 0; b < 2; ++b) {
        CREATE_CUDA(dalloc(&h->hd_idx[b], nk_hd));
        CREATE_CUDA(dalloc(&h->hd_d2[b], nk_hd));
        CREATE_CUDA(dalloc(&h->ld_idx[b], nk_ld));
    }
    CREATE_CUDA(dalloc(&h->P, nk_hd));
    CREATE_CUDA(dalloc(&h->beta, static_cast<size_t>(N)));
    CREATE_CUDA(dalloc(&h->sc, 1));
    CREATE_CUDA(dalloc(&h->zpart, static_cast<size_t>(h->max_blocks) + 1));
    CREATE_CUDA(dalloc(&h->cnt, 3 * static_cast<size_t>(h->max_blocks) + 3));
    cudaStream_t s = h->stream;
    CREATE_CUDA(cudaMemsetAsync(h->X32, 0, static_cast<size_t>(N) * h->xpitch * sizeof(float), s));
    CREATE_CUDA(copy_rows_raw(h->X32, h->xpitch, X, D, N, D, s));
    CREATE_CUDA(cudaMemsetAsync(h->Y, 0, h->yelem * sizeof(float), s));
    CREATE_CUDA(cudaMemsetAsync(h->V, 0, h->yelem * sizeof(float), s));
    CREATE_CUDA(cudaMemsetAsync(h->A, 0, h->yelem * sizeof(float), s));
    CREATE_CUDA(cudaMemsetAsync(h->R, 0, h->yelem * sizeof(float), s));
    DevScalars init{};
    init.E = 1.0;
    init.Zhat = 1.0;
    init.fresh_lo = N;  // no insertion window
    init.fresh_until = 0;
    CREATE_CUDA(cudaMemcpyAsync(h->sc, &init, sizeof(init), cudaMemcpyHostToDevice, s));
    CREATE_CUDA(launch_check_finite(h->X32, static_cast<int64_t>(N) * h->xpitch, &h->sc->err, s));
    {
        DevScalars chk;
        CREATE_CUDA(cudaMemcpyAsync(&chk, h->sc, sizeof(chk), cudaMemcpyDeviceToHost, s));
        CREATE_CUDA(cudaStreamSynchronize(s));
        if (chk.err) {
            fail(h, FUNCSNE_E_NAN, "X holds non-finite values");
            return bail(FUNCSNE_E_NAN);
        }
    }
    // initial state
    CREATE_CUDA(launch_init_lists(N, k_hd, kStreamInitHd, seed, h->hd_idx[0], s));
    CREATE_CUDA(launch_init_lists(N, k_ld, kStreamInitLd, seed, h->ld_idx[0], s));
    {
        FinalizeParams f{};
        f.N = N;
        f.k_hd = k_hd;
        f.n4 = h->n4;
        f.g = hd_lanes_f32(h);
        f.xpitch = h->xpitch;
        f.log_perp = std::log(perplexity);
        f.X32 = h->X32;
        f.idx = h->hd_idx[0];
        f.d2 = h->hd_d2[0];
        f.P = h->P;
        f.beta = h->beta;
        f.Pin = nullptr;
        int blocks = 8 * h->num_sms;
        CREATE_CUDA(launch_hd_finalize(f, blocks, s));
    }
    {
        // scratch for the projection (launch_init_y), then the first Z estimate
        const int64_t len = init_y_scratch_len(D, d, h->DP);
        double* scratch = nullptr;
        CREATE_CUDA(dalloc(&scratch, static_cast<size_t>(len)));
        cudaError_t e = launch_init_y(h->X32, N, D, h->xpitch, d, h->DP, seed, 0u, h->Y, scratch, len, s);
        if (e == cudaSuccess) {
            ZinitParams z = zinit_params(h, h->hd_idx[0], h->ld_idx[0], scratch);
            int blocks = 4 * h->num_sms;
            if (blocks > 1024) blocks = 1024;
            e = launch_zinit(z, h->DP, blocks, h->sc, s);
        }
        cudaError_t e2 = cudaStreamSynchronize(s);
        cudaFree(scratch);
        CREATE_CUDA(e);
        CREATE_CUDA(e2);
    }
#undef CREATE_CUDA
    configure_step(h);
    *out = h;
    return FUNCSNE_OK;
}

int recalibrate(funcsne* h);

int funcsne_set_option(funcsne_t* h, const char* key, double v) {
    if (!h || !key) return fail(h, FUNCSNE_E_ARG, "NULL handle or key");
    const std::string k(key);
    if (!std::isfinite(v)) return fail(h, FUNCSNE_E_ARG, "option %s: value must be finite", key);
    if (k == "lr") {
        if (!(v > 0)) return fail(h, FUNCSNE_E_ARG, "lr must be > 0");
        h->lr = v;
    } else if (k == "momentum") {
        if (v < 0 || v >= 1) return fail(h, FUNCSNE_E_ARG, "momentum must be in [0, 1)");
        h->momentum = v;
    } else if (k == "att_ratio") {
        if (v < 0) return fail(h, FUNCSNE_E_ARG, "att_ratio must be >= 0");
        h->att = v;
    } else if (k == "rep_ratio") {
        if (v < 0) return fail(h, FUNCSNE_E_ARG, "rep_ratio must be >= 0");
        h->rep = v;
    } else if (k == "exaggeration") {
        if (v <= 0) return fail(h, FUNCSNE_E_ARG, "exaggeration must be > 0");
        h->exaggeration = v;
    } else if (k == "exag_iters") {
        if (v < 0 || v > 2e9) return fail(h, FUNCSNE_E_ARG, "exag_iters out of range");
        h->exag_iters = static_cast<int32_t>(v);
    } else if (k == "hd_mode") {
        const int m = static_cast<int>(v);
        if (m != v || m < 0 || m > 2) return fail(h, FUNCSNE_E_ARG, "hd_mode must be 0, 1 or 2");
        h->hd_mode = m;
    } else if (k == "coin_floor" || k == "gamma_e" || k == "gamma_z") {
        if (!(v >= 0 && v <= 1) || (k != "coin_floor" && v == 0))
            return fail(h, FUNCSNE_E_ARG, "%s must be in %s", key, k == "coin_floor" ? "[0, 1]" : "(0, 1]");
        (k == "coin_floor" ? h->coin_floor : k == "gamma_e" ? h->gamma_e : h->gamma_z) = v;
    } else if (k == "alpha") {
        if (!(v > 0)) return fail(h, FUNCSNE_E_ARG, "alpha must be > 0");
        h->alpha = static_cast<float>(v);
    } else if (k == "forces_cw") {
        if (v != 4 && v != 8 && v != 16) return fail(h, FUNCSNE_E_ARG, "forces_cw must be 4, 8 or 16");
        h->forces_cw = static_cast<int32_t>(v);
        configure_step(h);
    } else if (k == "forces_pair" || k == "ld_pair" || k == "hd_prefetch") {
        if (v != 0 && v != 1) return fail(h, FUNCSNE_E_ARG, "%s must be 0 or 1", key);
        (k == "forces_pair" ? h->forces_pair : k == "ld_pair" ? h->ld_pair : h->hd_prefetch) = static_cast<int32_t>(v);
        configure_step(h);
    } else if (k == "perplexity") {
        if (!(v > 1) || !(v < h->k_hd + 1))
            return fail(h, FUNCSNE_E_ARG, "perplexity must be in (1, k_hd + 1)");
        h->perplexity = static_cast<float>(v);
        drop_graphs(h);
        return recalibrate(h);
    } else if (k == "jump_iters" || k == "jump_parts") {
        if (v < (k == "jump_parts" ? 1 : 0) || v > 1e7 || v != static_cast<int>(v))
            return fail(h, FUNCSNE_E_ARG, "%s must be an integer (jump_iters >= 0, jump_parts >= 1)", key);
        (k == "jump_iters" ? h->jump_iters : h->jump_parts) = static_cast<int32_t>(v);
    } else if (k == "fresh_iters") {
        if (v < 0 || v > 1e6 || v != std::floor(v)) return fail(h, FUNCSNE_E_ARG, "fresh_iters must be an integer in [0, 1e6]");
        h->fresh_iters = static_cast<int32_t>(v);
    } else if (k == "insert_rounds") {
        if (v < 0 || v > 256 || v != static_cast<int>(v))
            return fail(h, FUNCSNE_E_ARG, "insert_rounds must be an integer in [0, 256]");
        h->insert_rounds = static_cast<int32_t>(v);
    } else if (k == "hd_lanes") {
        if (v != 0 && v != 1 && v != 2 && v != 4 && v != 8)
            return fail(h, FUNCSNE_E_ARG, "hd_lanes must be 0, 1, 2, 4 or 8");
        h->hd_lanes_opt = static_cast<int32_t>(v);
        configure_step(h);
    } else if (k == "concurrent") {
        if (v != 0 && v != 1) return fail(h, FUNCSNE_E_ARG, "concurrent must be 0 or 1");
        h->concurrent = v != 0;
        configure_step(h);
    } else if (k == "surrogate") {
        if (v != 0 && v != 1) return fail(h, FUNCSNE_E_ARG, "surrogate must be 0 or 1");
        h->surrogate = v != 0;
    } else if (k == "mlp_every") {
        if (v < 1 || v > 1e6 || v != static_cast<int>(v)) return fail(h, FUNCSNE_E_ARG, "mlp_every must be a positive integer");
        h->mlp_every = static_cast<int32_t>(v);
    } else if (k == "mlp_lr") {
        if (!(v > 0)) return fail(h, FUNCSNE_E_ARG, "mlp_lr must be > 0");
        h->mlp_lr = static_cast<float>(v);
    } else if (k == "mlp_batch" || k == "mlp_hidden") {
        if (h->mlp.ready) return fail(h, FUNCSNE_E_STATE, "%s must be set before the surrogate is first used", key);
        if (v < 16 || v > 65536 || v != static_cast<int>(v)) return fail(h, FUNCSNE_E_ARG, "%s must be an integer in [16, 65536]", key);
        (k == "mlp_batch" ? h->mlp_B : h->mlp_H) = static_cast<int32_t>(v);
    } else if (k == "precision") {
        const int m = static_cast<int>(v);
        if (m != v || m < 0 || m > 2) return fail(h, FUNCSNE_E_ARG, "precision must be 0, 1 or 2");
        if (m != h->precision) {
            h->precision = m;
            int rc = quantize(h);
            if (rc) return rc;
            configure_step(h);
        }
    } else {
        return fail(h, FUNCSNE_E_ARG, "unknown option '%s'", key);
    }
    drop_graphs(h);
    return FUNCSNE_OK;
}

int funcsne_get_option(const funcsne_t* hc, const char* key, double* v) {
    funcsne* h = const_cast<funcsne*>(hc);
    if (!h || !key || !v) return fail(h, FUNCSNE_E_ARG, "NULL argument");
    const std::string k(key);
    if (k == "lr") *v = h->lr;
    else if (k == "momentum") *v = h->momentum;
    else if (k == "att_ratio") *v = h->att;
    else if (k == "rep_ratio") *v = h->rep;
    else if (k == "exaggeration") *v = h->exaggeration;
    else if (k == "exag_iters") *v = h->exag_iters;
    else if (k == "hd_mode") *v = h->hd_mode;
    else if (k == "coin_floor") *v = h->coin_floor;
    else if (k == "gamma_e") *v = h->gamma_e;
    else if (k == "gamma_z") *v = h->gamma_z;
    else if (k == "alpha") *v = h->alpha;
    else if (k == "precision") *v = h->precision;
    else if (k == "concurrent") *v = h->concurrent ? 1 : 0;
    else if (k == "forces_cw") *v = h->forces_cw;
    else if (k == "forces_pair") *v = h->forces_pair;
    else if (k == "ld_pair") *v = h->ld_pair;
    else if (k == "hd_prefetch") *v = h->hd_prefetch;
    else if (k == "hd_prefetch_used") *v = h->hd_pf_used;
    else if (k == "hd_lanes") *v = h->hd_lanes_opt;
    else if (k == "hd_lanes_used") *v = hd_lanes(h);
    else if (k == "insert_rounds") *v = h->insert_rounds;
    else if (k == "fresh_iters") *v = h->fresh_iters;
    else if (k == "jump_iters") *v = h->jump_iters;
    else if (k == "jump_parts") *v = h->jump_parts;
    else if (k == "perplexity") *v = h->perplexity;
    else if (k == "surrogate") *v = h->surrogate ? 1 : 0;
    else if (k == "mlp_every") *v = h->mlp_every;
    else if (k == "mlp_lr") *v = h->mlp_lr;
    else if (k == "mlp_batch") *v = h->mlp_B;
    else if (k == "mlp_hidden") *v = h->mlp_H;
    else if (k == "hd_blocks") *v = h->hd_blocks;
    else if (k == "ld_blocks") *v = h->ld_blocks;
    else if (k == "forces_blocks") *v = h->fo_blocks;
    else return fail(h, FUNCSNE_E_ARG, "unknown option '%s'", key);
    return FUNCSNE_OK;
}

int funcsne_set_stream(funcsne_t* h, void* stream) {
    if (!h) return fail(h, FUNCSNE_E_ARG, "NULL handle");
    // order the new stream after all work already queued on the old one
    cudaEvent_t ev;
    FSNE_CUDA(h, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    FSNE_CUDA(h, cudaEventRecord(ev, h->stream));
    h->stream = stream ? static_cast<cudaStream_t>(stream) : h->own_stream;
    cudaError_t e = cudaStreamWaitEvent(h->stream, ev, 0);
    cudaEventDestroy(ev);
    FSNE_CUDA(h, e);
    return FUNCSNE_OK;
}

// Y = a random linear projection of the data, Philox counter (ctr, f,
// INIT_Y, c), each LD dimension at the initial scale.
int project_embedding(funcsne* h, uint32_t ctr) {
    const int64_t len = init_y_scratch_len(h->D, h->d, h->DP);
    double* scratch = nullptr;
    FSNE_CUDA(h, dalloc(&scratch, static_cast<size_t>(len)));
    cudaError_t e = launch_init_y(h->X32, h->N, h->D, h->xpitch, h->d, h->DP, h->seed, ctr, h->Y, scratch, len,
                                  h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(scratch);
    FSNE_CUDA(h, e);
    return FUNCSNE_OK;
}

// One iteration of the jump start (Section 3): at the start of each of
// jump_parts equal parts of the first jump_iters iterations the embedding is
// replaced by a fresh random linear projection of the data; the iteration
// refines both neighbour sets and estimates Z, but applies no gradient.
int jump_iteration(funcsne* h) {
    const int64_t t = h->t_host, J = h->jump_iters, P = h->jump_parts;
    for (int64_t p = 0; p < P; ++p)
        if (t == p * J / P) {
            int rc = project_embedding(h, static_cast<uint32_t>(p + 1));
            if (rc) return rc;
        }
    h->frozen = true;
    int rc = enqueue_iteration(h, h->stream, nullptr, nullptr);
    h->frozen = false;
    if (rc) return rc;
    ++h->t_host;
    return FUNCSNE_OK;
}

int funcsne_step(funcsne_t* h, int32_t n_iters) {
    NvtxRange nvtx_range("funcsne_step");
    if (!h) return fail(h, FUNCSNE_E_ARG, "NULL handle");
    if (n_iters < 0) return fail(h, FUNCSNE_E_ARG, "n_iters must be >= 0");
    while (n_iters > 0 && h->t_host < static_cast<uint32_t>(h->jump_iters)) {
        int rc = jump_iteration(h);
        if (rc) return rc;
        --n_iters;
    }
    if (n_iters == 0) return FUNCSNE_OK;
    if (!h->graph1) {
        int rc = build_graph(h, 1, &h->graph1);
        if (rc) return rc;
    }
    if (h->surrogate) {
        // the surrogate trains on (x_i, y_i) of the current state before every
        // mlp_every-th iteration
        for (int k = 0; k < n_iters; ++k) {
            if (h->t_host % static_cast<uint32_t>(h->mlp_every) == 0) {
                int rc = mlp_train_now(h, 1);
                if (rc) return rc;
            }
            FSNE_CUDA(h, cudaGraphLaunch(h->graph1, h->stream));
            ++h->t_host;
        }
        return FUNCSNE_OK;
    }
    if (n_iters >= 8 && !h->graph8) {
        int rc = build_graph(h, 8, &h->graph8);
        if (rc) return rc;
    }
    int left = n_iters;
    while (left >= 8) {
        FSNE_CUDA(h, cudaGraphLaunch(h->graph8, h->stream));
        left -= 8;
    }
    while (left-- > 0) FSNE_CUDA(h, cudaGraphLaunch(h->graph1, h->stream));
    h->t_host += static_cast<uint32_t>(n_iters);
    return FUNCSNE_OK;
}

int funcsne_mlp_train(funcsne_t* h, int32_t n_steps) {
    NvtxRange nvtx_range("funcsne_mlp_train");
    if (!h) return fail(h, FUNCSNE_E_ARG, "NULL handle");
    if (n_steps < 0) return fail(h, FUNCSNE_E_ARG, "n_steps must be >= 0");
    return mlp_train_now(h, n_steps);
}

int funcsne_mlp_predict(const funcsne_t* hc, const float* X, int64_t n, float* Y_out) {
    funcsne* h = const_cast<funcsne*>(hc);
    if (!h || !X || !Y_out) return fail(h, FUNCSNE_E_ARG, "NULL argument");
    if (n < 0) return fail(h, FUNCSNE_E_ARG, "n must be >= 0");
    if (n == 0) return FUNCSNE_OK;
    int rc = ensure_mlp(h);
    if (rc) return rc;
    float *xd = nullptr, *yd = nullptr;
    cudaError_t e = dalloc(&xd, static_cast<size_t>(n) * h->xpitch);
    if (e == cudaSuccess) e = dalloc(&yd, static_cast<size_t>(n) * h->DP);
    if (e == cudaSuccess) e = cudaMemsetAsync(xd, 0, static_cast<size_t>(n) * h->xpitch * 4, h->stream);
    if (e == cudaSuccess)
        e = copy_rows_raw(xd, h->xpitch, X, h->D, n, h->D, h->stream);
    if (e == cudaSuccess) e = launch_mlp_place(mlp_params(h), xd, h->xpitch, 0, n, yd, h->DP, h->stream);
    if (e == cudaSuccess)
        e = copy_rows_raw(Y_out, h->d, yd, h->DP, n, h->d, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(xd);
    cudaFree(yd);
    FSNE_CUDA(h, e);
    return FUNCSNE_OK;
}

int funcsne_debug_fail_alloc(int64_t after) {
    g_fail_alloc_after = after < 0 ? -1 : after;
    return FUNCSNE_OK;
}

int funcsne_debug_bounded_wait(funcsne_t* h, uint32_t polls) {
    if (!h) return fail(h, FUNCSNE_E_ARG, "NULL handle");
    if (polls < 1 || polls > (1u << 24)) return fail(h, FUNCSNE_E_ARG, "polls must be in [1, 2^24]");
    FSNE_CUDA(h, launch_bounded_wait(&h->sc->err, polls, h->stream));
    return FUNCSNE_OK;
}

int funcsne_mlp_debug_step(funcsne_t* h, funcsne_mlp_debug_t* out) {
    if (!h || !out) return fail(h, FUNCSNE_E_ARG, "NULL argument");
    int rc = ensure_mlp(h);
    if (rc) return rc;
    auto& q = h->mlp;
    const size_t np = static_cast<size_t>(q.n_params);
    const size_t B = static_cast<size_t>(h->mlp_B), D = static_cast<size_t>(h->D), d = static_cast<size_t>(h->d);
    float* tmp = nullptr;
    FSNE_CUDA(h, dalloc(&tmp, np > B * D ? np : B * D));
    auto finish = [&](cudaError_t e) -> int {
        cudaFree(tmp);
        FSNE_CUDA(h, e);
        return static_cast<int>(FUNCSNE_OK);
    };
    cudaError_t e = cudaSuccess;
    if (out->theta_before) e = cudaMemcpyAsync(out->theta_before, q.theta, np * 4, cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess && out->weights_bf16) {
        e = launch_bf16_to_f32(q.wb, static_cast<int64_t>(np), tmp, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out->weights_bf16, tmp, np * 4, cudaMemcpyDefault, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    }
    uint32_t step0 = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&step0, q.step, 4, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = launch_mlp_train_step(mlp_params(h), h->stream);
    if (e != cudaSuccess) return finish(e);
    ++h->mlp_steps;
    if (out->batch_idx) e = cudaMemcpyAsync(out->batch_idx, q.idx, B * 4, cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess && out->target) e = cudaMemcpyAsync(out->target, q.T, B * d * 4, cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess && out->output) e = cudaMemcpyAsync(out->output, q.O, B * d * 4, cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess && out->grad) e = cudaMemcpyAsync(out->grad, q.grad, np * 4, cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess && out->theta_after) e = cudaMemcpyAsync(out->theta_after, q.theta, np * 4, cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess && out->xhat) {
        e = cudaStreamSynchronize(h->stream);
        if (e == cudaSuccess) e = launch_bf16_to_f32(q.Xb, static_cast<int64_t>(B * D), tmp, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out->xhat, tmp, B * D * 4, cudaMemcpyDefault, h->stream);
    }
    double loss = 0.0;
    float scale = 1.f;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&loss, q.loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&scale, q.scale, sizeof(float), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    out->loss = loss;
    out->scale = scale;
    out->step = static_cast<int32_t>(step0) + 1;
    out->n_params = q.n_params;
    return finish(e);
}

int funcsne_sync(funcsne_t* h) {
    if (!h) return fail(h, FUNCSNE_E_ARG, "NULL handle");
    FSNE_CUDA(h, cudaStreamSynchronize(h->stream));
    if (h->copy_stream) FSNE_CUDA(h, cudaStreamSynchronize(h->copy_stream));
    FSNE_CUDA(h, cudaGetLastError());
    return check_errors(h);
}

int funcsne_insert(funcsne_t* h, const float* X_new, int64_t n_new, int32_t placement, int64_t* first_id) {
    NvtxRange nvtx_range("funcsne_insert");
    if (!h || !X_new || !first_id) return fail(h, FUNCSNE_E_ARG, "NULL argument");
    if (n_new < 1) return fail(h, FUNCSNE_E_ARG, "n_new must be >= 1");
    if (placement != FUNCSNE_PLACE_MEAN && placement != FUNCSNE_PLACE_SURROGATE)
        return fail(h, FUNCSNE_E_ARG, "placement must be FUNCSNE_PLACE_MEAN or FUNCSNE_PLACE_SURROGATE");
    const int64_t n_old = h->N, N2 = h->N + n_new;
    if (N2 >= (int64_t(1) << 31) - 1) return fail(h, FUNCSNE_E_ARG, "N + n_new must stay below 2^31 - 1");
    DevScalars s;
    int rc = read_scalars(h, &s);
    if (rc) return rc;
    if (N2 > h->cap) {
        int64_t nc = h->cap + h->cap / 2;
        if (nc < N2) nc = N2;
        if ((rc = grow(h, nc))) return rc;
    }
    float* xdst = h->X32 + n_old * h->xpitch;
    FSNE_CUDA(h, copy_rows_raw(xdst, h->xpitch, X_new, h->D, n_new, h->D, h->stream));
    FSNE_CUDA(h, launch_check_finite(xdst, n_new * h->xpitch, &h->sc->err, h->stream));
    {
        DevScalars chk;
        if ((rc = read_scalars(h, &chk))) return rc;
        if (chk.err & kErrNonFinite) {
            FSNE_CUDA(h, cudaMemsetAsync(xdst, 0, static_cast<size_t>(n_new) * h->xpitch * sizeof(float), h->stream));
            clear_error_word(h);
            return fail(h, FUNCSNE_E_NAN, "X_new holds non-finite values");
        }
    }
    if (h->precision != FUNCSNE_FP32)
        FSNE_CUDA(h, launch_quantize(xdst, n_new, h->D, h->xpitch, h->precision, h->qpitch, h->qscale_off,
                                     h->Xq + n_old * h->qpitch, h->stream));
    InsertParams q{};
    q.N = N2;
    q.n_old = n_old;
    q.k_hd = h->k_hd;
    q.k_ld = h->k_ld;
    q.n4 = h->n4;
    q.g = hd_lanes_f32(h);
    q.rounds = h->insert_rounds;
    q.xpitch = h->xpitch;
    q.log_perp = std::log(h->perplexity);
    q.t = s.t;
    q.seed = h->seed;
    q.X32 = h->X32;
    q.Y = h->Y;
    q.V = h->V;
    q.A = h->A;
    q.R = h->R;
    q.hd_idx = h->hd_idx[s.hd_cur];
    q.hd_d2 = h->hd_d2[s.hd_cur];
    q.ld_idx = h->ld_idx[s.ld_cur];
    q.P = h->P;
    q.beta = h->beta;
    FSNE_CUDA(h, launch_insert(q, h->DP, h->stream));
    if (placement == FUNCSNE_PLACE_SURROGATE && h->mlp.ready && h->mlp_steps > 0)
        FSNE_CUDA(h, launch_mlp_place(mlp_params(h), h->X32, h->xpitch, n_old, n_new, h->Y, h->DP, h->stream));
    // the scalars of the grown state: Zhat scaled by the ordered pair count,
    // inserted points count as points with new neighbours
    s.Zhat *= (static_cast<double>(N2) * static_cast<double>(N2 - 1)) /
              (static_cast<double>(n_old) * static_cast<double>(n_old - 1));
    const double frac = static_cast<double>(n_new) / static_cast<double>(N2);
    if (frac > s.E) s.E = frac;
    // the new points' refinement window: the next fresh_iters iterations; a
    // window still open keeps its older points in it
    if (h->fresh_iters > 0) {
        if (!(s.t < s.fresh_until)) s.fresh_lo = n_old;
        s.fresh_until = s.t + static_cast<uint32_t>(h->fresh_iters);
        FSNE_CUDA(h, cudaMemcpyAsync(&h->sc->fresh_lo, &s.fresh_lo, sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
        FSNE_CUDA(h, cudaMemcpyAsync(&h->sc->fresh_until, &s.fresh_until, sizeof(uint32_t), cudaMemcpyHostToDevice,
                                     h->stream));
    }
    FSNE_CUDA(h, cudaMemcpyAsync(&h->sc->Zhat, &s.Zhat, sizeof(double), cudaMemcpyHostToDevice, h->stream));
    FSNE_CUDA(h, cudaMemcpyAsync(&h->sc->E, &s.E, sizeof(double), cudaMemcpyHostToDevice, h->stream));
    FSNE_CUDA(h, cudaStreamSynchronize(h->stream));
    h->N = N2;
    h->yelem = (N2 * h->DP + 3) / 4 * 4;
    configure_step(h);
    *first_id = n_old;
    return FUNCSNE_OK;
}

// Every point's HD list distances recomputed from X32, its list reordered
// by (d2, idx), beta and P calibrated from a cold start (Eq. 1).
int recalibrate(funcsne* h) {
    DevScalars s;
    int rc = read_scalars(h, &s);
    if (rc) return rc;
    FinalizeParams f{};
    f.N = h->N;
    f.k_hd = h->k_hd;
    f.n4 = h->n4;
    f.g = hd_lanes_f32(h);
    f.xpitch = h->xpitch;
    f.log_perp = std::log(h->perplexity);
    f.X32 = h->X32;
    f.idx = h->hd_idx[s.hd_cur];
    f.d2 = h->hd_d2[s.hd_cur];
    f.P = h->P;
    f.beta = h->beta;
    f.Pin = nullptr;
    FSNE_CUDA(h, launch_hd_finalize(f, 8 * h->num_sms, h->stream));
    FSNE_CUDA(h, cudaStreamSynchronize(h->stream));
    return FUNCSNE_OK;
}

// Host copy of n point ids (host or device memory), checked to be distinct
// and in [0, N).
int host_ids(funcsne* h, const int64_t* ids, int64_t n, std::vector<int64_t>& out) {
    out.resize(static_cast<size_t>(n));
    FSNE_CUDA(h, cudaMemcpy(out.data(), ids, static_cast<size_t>(n) * sizeof(int64_t), cudaMemcpyDefault));
    std::vector<int64_t> s(out);
    std::sort(s.begin(), s.end());
    for (size_t a = 0; a < s.size(); ++a) {
        if (s[a] < 0 || s[a] >= h->N) return fail(h, FUNCSNE_E_ARG, "point id %lld out of range", (long long)s[a]);
        if (a && s[a] == s[a - 1]) return fail(h, FUNCSNE_E_ARG, "point id %lld repeated", (long long)s[a]);
    }
    return FUNCSNE_OK;
}

int funcsne_update_points(funcsne_t* h, const int64_t* ids, int64_t n, const float* X_rows) {
    NvtxRange nvtx_range("funcsne_update_points");
    if (!h || !ids || !X_rows) return fail(h, FUNCSNE_E_ARG, "NULL argument");
    if (n < 1) return fail(h, FUNCSNE_E_ARG, "n must be >= 1");
    std::vector<int64_t> hid;
    int rc = host_ids(h, ids, n, hid);
    if (rc) return rc;
    int64_t* did = nullptr;
    float* drows = nullptr;
    FSNE_CUDA(h, dalloc(&did, static_cast<size_t>(n)));
    cudaError_t e = dalloc(&drows, static_cast<size_t>(n) * h->D);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(did, hid.data(), static_cast<size_t>(n) * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(drows, X_rows, static_cast<size_t>(n) * h->D * sizeof(float), cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess) e = launch_check_finite(drows, static_cast<int64_t>(n) * h->D, &h->sc->err, h->stream);
    DevScalars chk{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&chk, h->sc, sizeof(chk), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess && !(chk.err & kErrNonFinite))
        e = launch_scatter_rows(h->X32, h->xpitch, did, drows, n, h->D, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(did);
    cudaFree(drows);
    FSNE_CUDA(h, e);
    if (chk.err & kErrNonFinite) {
        clear_error_word(h);
        return fail(h, FUNCSNE_E_NAN, "X_rows holds non-finite values");
    }
    if (h->precision != FUNCSNE_FP32 && (rc = quantize(h))) return rc;
    drop_graphs(h);
    return recalibrate(h);
}

int funcsne_remove(funcsne_t* h, const int64_t* ids, int64_t n) {
    NvtxRange nvtx_range("funcsne_remove");
    if (!h || !ids) return fail(h, FUNCSNE_E_ARG, "NULL argument");
    if (n < 1) return fail(h, FUNCSNE_E_ARG, "n must be >= 1");
    std::vector<int64_t> hid;
    int rc = host_ids(h, ids, n, hid);
    if (rc) return rc;
    const int64_t N = h->N, Nk = N - n;
    if (Nk <= h->k_hd || Nk <= h->k_ld)
        return fail(h, FUNCSNE_E_ARG, "removal would leave %lld points, at most k_hd or k_ld", (long long)Nk);
    DevScalars s;
    if ((rc = read_scalars(h, &s))) return rc;
    std::vector<int32_t> new_of(static_cast<size_t>(N), 0), old_of;
    for (int64_t id : hid) new_of[static_cast<size_t>(id)] = -1;
    old_of.reserve(static_cast<size_t>(Nk));
    for (int64_t o = 0; o < N; ++o)
        if (new_of[static_cast<size_t>(o)] == 0) {
            new_of[static_cast<size_t>(o)] = static_cast<int32_t>(old_of.size());
            old_of.push_back(static_cast<int32_t>(o));
        } else {
            new_of[static_cast<size_t>(o)] = -1;
        }
    int32_t *d_new = nullptr, *d_old = nullptr;
    uint32_t* tmp = nullptr;
    const int64_t widest = std::max<int64_t>({h->xpitch, static_cast<int64_t>(h->DP), h->k_hd, h->k_ld});
    FSNE_CUDA(h, dalloc(&d_new, static_cast<size_t>(N)));
    cudaError_t e = dalloc(&d_old, static_cast<size_t>(Nk));
    if (e == cudaSuccess) e = dalloc(&tmp, static_cast<size_t>(Nk * widest));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_new, new_of.data(), static_cast<size_t>(N) * 4, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_old, old_of.data(), static_cast<size_t>(Nk) * 4, cudaMemcpyHostToDevice, h->stream);
    // compact the kept rows of each array, in order, through tmp
    auto compact = [&](void* arr, int64_t pitch) {
        if (e != cudaSuccess) return;
        e = launch_gather_rows(tmp, static_cast<const uint32_t*>(arr), pitch, d_old, Nk, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(arr, tmp, static_cast<size_t>(Nk * pitch) * 4, cudaMemcpyDeviceToDevice, h->stream);
    };
    compact(h->X32, h->xpitch);
    compact(h->Y, h->DP);
    compact(h->V, h->DP);
    compact(h->beta, 1);
    compact(h->hd_idx[s.hd_cur], h->k_hd);
    compact(h->ld_idx[s.ld_cur], h->k_ld);
    if (e == cudaSuccess)
        e = launch_remap_lists(h->hd_idx[s.hd_cur], h->k_hd, d_new, Nk, s.t, h->seed, 0u, h->stream);
    if (e == cudaSuccess)
        e = launch_remap_lists(h->ld_idx[s.ld_cur], h->k_ld, d_new, Nk, s.t, h->seed, 1024u, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(d_new);
    cudaFree(d_old);
    cudaFree(tmp);
    FSNE_CUDA(h, e);
    h->N = Nk;
    h->yelem = (Nk * h->DP + 3) / 4 * 4;
    FSNE_CUDA(h, cudaMemsetAsync(h->Y + Nk * h->DP, 0, static_cast<size_t>(N - Nk) * h->DP * 4, h->stream));
    FSNE_CUDA(h, cudaMemsetAsync(h->A, 0, static_cast<size_t>(h->cap) * h->DP * 4, h->stream));
    if (h->precision != FUNCSNE_FP32 && (rc = quantize(h))) return rc;
    // removed points count as points whose neighbourhood changed; Zhat
    // follows the ordered pair count
    s.Zhat *= (static_cast<double>(Nk) * static_cast<double>(Nk - 1)) /
              (static_cast<double>(N) * static_cast<double>(N - 1));
    const double frac = static_cast<double>(n) / static_cast<double>(N);
    if (frac > s.E) s.E = frac;
    FSNE_CUDA(h, cudaMemcpyAsync(&h->sc->Zhat, &s.Zhat, sizeof(double), cudaMemcpyHostToDevice, h->stream));
    FSNE_CUDA(h, cudaMemcpyAsync(&h->sc->E, &s.E, sizeof(double), cudaMemcpyHostToDevice, h->stream));
    // renumbering closes the refinement window of recent insertions
    s.fresh_lo = Nk;
    s.fresh_until = s.t;
    FSNE_CUDA(h, cudaMemcpyAsync(&h->sc->fresh_lo, &s.fresh_lo, sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
    FSNE_CUDA(h, cudaMemcpyAsync(&h->sc->fresh_until, &s.fresh_until, sizeof(uint32_t), cudaMemcpyHostToDevice,
                                 h->stream));
    configure_step(h);
    return recalibrate(h);
}

int funcsne_get_embedding(const funcsne_t* hc, float* Y_out, int64_t cap_rows) {
    NvtxRange nvtx_range("funcsne_get_embedding");
    funcsne* h = const_cast<funcsne*>(hc);
    if (!h || !Y_out) return fail(h, FUNCSNE_E_ARG, "NULL argument");
    const int64_t rows = cap_rows < h->N ? cap_rows : h->N;
    int rc = copy_rows<float>(h, Y_out, h->d, h->Y, h->DP, rows, h->d);
    if (rc) return rc;
    FSNE_CUDA(h, cudaStreamSynchronize(h->stream));
    return FUNCSNE_OK;
}

int funcsne_get_embedding_async(funcsne_t* h, float* Y_out, int64_t cap_rows) {
    if (!h || !Y_out) return fail(h, FUNCSNE_E_ARG, "NULL argument");
    const int64_t rows = cap_rows < h->N ? cap_rows : h->N;
    if (rows <= 0) return FUNCSNE_OK;
    if (!h->copy_stream) {
        FSNE_CUDA(h, cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
        FSNE_CUDA(h, cudaEventCreateWithFlags(&h->snap_ev, cudaEventDisableTiming));
        FSNE_CUDA(h, cudaEventCreateWithFlags(&h->copy_ev, cudaEventDisableTiming));
    }
    if (rows > h->snap_rows) {
        // the old snapshot may still be in flight
        FSNE_CUDA(h, cudaStreamSynchronize(h->copy_stream));
        cudaFree(h->Ysnap);
        h->Ysnap = nullptr;
        h->snap_rows = 0;
        FSNE_CUDA(h, dalloc(&h->Ysnap, static_cast<size_t>(h->cap) * h->d));
        h->snap_rows = h->cap;
    }
    // the snapshot is overwritten only after the previous copy out of it
    FSNE_CUDA(h, cudaStreamWaitEvent(h->stream, h->copy_ev, 0));
    FSNE_CUDA(h, copy_rows_raw(h->Ysnap, h->d, h->Y, h->DP, rows, h->d, h->stream));
    FSNE_CUDA(h, cudaEventRecord(h->snap_ev, h->stream));
    FSNE_CUDA(h, cudaStreamWaitEvent(h->copy_stream, h->snap_ev, 0));
    FSNE_CUDA(h, cudaMemcpyAsync(Y_out, h->Ysnap, static_cast<size_t>(rows) * h->d * sizeof(float),
                                 cudaMemcpyDefault, h->copy_stream));
    FSNE_CUDA(h, cudaEventRecord(h->copy_ev, h->copy_stream));
    return FUNCSNE_OK;
}

int funcsne_wait_embedding(funcsne_t* h) {
    if (!h) return fail(h, FUNCSNE_E_ARG, "NULL handle");
    if (h->copy_ev) FSNE_CUDA(h, cudaEventSynchronize(h->copy_ev));
    return FUNCSNE_OK;
}

int funcsne_get_data(const funcsne_t* hc, float* X_out, int64_t cap_rows) {
    funcsne* h = const_cast<funcsne*>(hc);
    if (!h || !X_out) return fail(h, FUNCSNE_E_ARG, "NULL argument");
    const int64_t rows = cap_rows < h->N ? cap_rows : h->N;
    int rc = copy_rows<float>(h, X_out, h->D, h->X32, h->xpitch, rows, h->D);
    if (rc) return rc;
    FSNE_CUDA(h, cudaStreamSynchronize(h->stream));
    return FUNCSNE_OK;
}

int funcsne_debug_row_bounds(const funcsne_t* hc, float* E_out, int64_t cap_rows) {
    funcsne* h = const_cast<funcsne*>(hc);
    if (!h || !E_out) return fail(h, FUNCSNE_E_ARG, "NULL argument");
    if (h->precision == FUNCSNE_FP32 || !h->Xq)
        return fail(h, FUNCSNE_E_STATE, "debug_row_bounds: no reduced-precision rows in FP32 mode");
    const int64_t rows = cap_rows < h->N ? cap_rows : h->N;
    // the bound sits at byte qscale_off of a BF16 row, four bytes before the
    // scale of an FP8 row
    const int off = h->precision == FUNCSNE_BF16 ? h->qscale_off : h->qscale_off - 4;
    const float* src = reinterpret_cast<const float*>(h->Xq + off);
    int rc = copy_rows<float>(h, E_out, 1, src, static_cast<size_t>(h->qpitch / 4), rows, 1);
    if (rc) return rc;
    FSNE_CUDA(h, cudaStreamSynchronize(h->stream));
    return FUNCSNE_OK;
}

int funcsne_scale_embedding(funcsne_t* h, float factor) {
    if (!h) return fail(h, FUNCSNE_E_ARG, "NULL handle");
    if (!(factor > 0.f) || !std::isfinite(factor)) return fail(h, FUNCSNE_E_ARG, "factor must be > 0 and finite");
    DevScalars s;
    int rc = read_scalars(h, &s);
    if (rc) return rc;
    FSNE_CUDA(h, launch_scale_rows(h->Y, h->V, h->N * h->DP, factor, h->stream));
    // Zhat re-estimated at the scaled embedding, negatives from (t, i, ZINIT, s)
    double* part = nullptr;
    int blocks = 4 * h->num_sms;
    if (blocks > 1024) blocks = 1024;
    FSNE_CUDA(h, dalloc(&part, static_cast<size_t>(blocks)));
    ZinitParams z = zinit_params(h, h->hd_idx[s.hd_cur], h->ld_idx[s.ld_cur], part);
    z.t = s.t;
    cudaError_t e = launch_zinit(z, h->DP, blocks, h->sc, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(part);
    FSNE_CUDA(h, e);
    return FUNCSNE_OK;
}

int funcsne_get_knn(const funcsne_t* hc, int32_t space, int32_t* idx, float* d2) {
    funcsne* h = const_cast<funcsne*>(hc);
    if (!h || !idx) return fail(h, FUNCSNE_E_ARG, "NULL argument");
    DevScalars s;
    int rc = read_scalars(h, &s);
    if (rc) return rc;
    if (space == FUNCSNE_SPACE_HD) {
        const size_t n = static_cast<size_t>(h->N) * h->k_hd;
        FSNE_CUDA(h, cudaMemcpyAsync(idx, h->hd_idx[s.hd_cur], n * sizeof(int32_t), cudaMemcpyDefault, h->stream));
        if (d2) FSNE_CUDA(h, cudaMemcpyAsync(d2, h->hd_d2[s.hd_cur], n * sizeof(float), cudaMemcpyDefault, h->stream));
    } else if (space == FUNCSNE_SPACE_LD) {
        const size_t n = static_cast<size_t>(h->N) * h->k_ld;
        FSNE_CUDA(h, cudaMemcpyAsync(idx, h->ld_idx[s.ld_cur], n * sizeof(int32_t), cudaMemcpyDefault, h->stream));
        if (d2) {
            float* tmp = nullptr;
            FSNE_CUDA(h, dalloc(&tmp, n));
            cudaError_t e = launch_ld_distances(h->Y, h->ld_idx[s.ld_cur], h->N, h->k_ld, h->DP, tmp, h->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d2, tmp, n * sizeof(float), cudaMemcpyDefault, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            cudaFree(tmp);
            FSNE_CUDA(h, e);
        }
    } else {
        return fail(h, FUNCSNE_E_ARG, "space must be FUNCSNE_SPACE_HD or FUNCSNE_SPACE_LD");
    }
    FSNE_CUDA(h, cudaStreamSynchronize(h->stream));
    return FUNCSNE_OK;
}

int funcsne_get_stats(const funcsne_t* hc, funcsne_stats_t* st) {
    funcsne* h = const_cast<funcsne*>(hc);
    if (!h || !st) return fail(h, FUNCSNE_E_ARG, "NULL argument");
    DevScalars s;
    int rc = read_scalars(h, &s);
    if (rc) return rc;
    st->N = h->N;
    st->t = s.t;
    st->E = s.E;
    st->Zhat = s.Zhat;
    st->last_Z = s.last_Z;
    st->last_n_new = static_cast<int64_t>(s.last_n_new);
    st->last_coin = s.last_coin;
    st->precision = h->precision;
    st->error_word = s.err;
    st->cand_scored = static_cast<int64_t>(s.cand_scored);
    st->cand_reranked = static_cast<int64_t>(s.cand_reranked);
    st->mlp_steps = h->mlp_steps;
    st->n_refined = static_cast<int64_t>(s.n_refined);
    st->mlp_loss = 0.0;
    if (h->mlp.ready) {
        FSNE_CUDA(h, cudaMemcpyAsync(&st->mlp_loss, h->mlp.loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        FSNE_CUDA(h, cudaStreamSynchronize(h->stream));
    }
    return FUNCSNE_OK;
}

int funcsne_export_state(const funcsne_t* hc, funcsne_state_t* st) {
    funcsne* h = const_cast<funcsne*>(hc);
    if (!h || !st) return fail(h, FUNCSNE_E_ARG, "NULL argument");
    DevScalars s;
    int rc = read_scalars(h, &s);
    if (rc) return rc;
    const size_t nh = static_cast<size_t>(h->N) * h->k_hd, nl = static_cast<size_t>(h->N) * h->k_ld;
    if (st->Y && (rc = copy_rows<float>(h, st->Y, h->d, h->Y, h->DP, h->N, h->d))) return rc;
    if (st->V && (rc = copy_rows<float>(h, st->V, h->d, h->V, h->DP, h->N, h->d))) return rc;
    if (st->hd_idx) FSNE_CUDA(h, cudaMemcpyAsync(st->hd_idx, h->hd_idx[s.hd_cur], nh * 4, cudaMemcpyDefault, h->stream));
    if (st->hd_d2) FSNE_CUDA(h, cudaMemcpyAsync(st->hd_d2, h->hd_d2[s.hd_cur], nh * 4, cudaMemcpyDefault, h->stream));
    if (st->ld_idx) FSNE_CUDA(h, cudaMemcpyAsync(st->ld_idx, h->ld_idx[s.ld_cur], nl * 4, cudaMemcpyDefault, h->stream));
    if (st->beta) FSNE_CUDA(h, cudaMemcpyAsync(st->beta, h->beta, static_cast<size_t>(h->N) * 4, cudaMemcpyDefault, h->stream));
    if (st->P) FSNE_CUDA(h, cudaMemcpyAsync(st->P, h->P, nh * 4, cudaMemcpyDefault, h->stream));
    FSNE_CUDA(h, cudaStreamSynchronize(h->stream));
    st->Zhat = s.Zhat;
    st->E = s.E;
    st->t = s.t;
    st->fresh_lo = s.fresh_lo;
    st->fresh_until = s.fresh_until;
    return FUNCSNE_OK;
}

int funcsne_import_state(funcsne_t* h, const funcsne_state_t* st) {
    if (!h || !st) return fail(h, FUNCSNE_E_ARG, "NULL argument");
    if (!(st->Zhat > 0) || !std::isfinite(st->Zhat) || !(st->E >= 0 && st->E <= 1))
        return fail(h, FUNCSNE_E_ARG, "Zhat must be > 0 and E in [0, 1]");
    if (st->fresh_lo < 0 || st->fresh_lo > h->N) return fail(h, FUNCSNE_E_ARG, "fresh_lo must be in [0, N]");
    DevScalars s;
    int rc = read_scalars(h, &s);
    if (rc) return rc;
    const size_t nh = static_cast<size_t>(h->N) * h->k_hd, nl = static_cast<size_t>(h->N) * h->k_ld;
    if ((rc = clear_error_word(h))) return rc;
    if (st->hd_idx) {
        FSNE_CUDA(h, cudaMemcpyAsync(h->hd_idx[s.hd_cur], st->hd_idx, nh * 4, cudaMemcpyDefault, h->stream));
        FSNE_CUDA(h, launch_check_lists(h->hd_idx[s.hd_cur], h->N, h->k_hd, &h->sc->err, h->stream));
    }
    if (st->ld_idx) {
        FSNE_CUDA(h, cudaMemcpyAsync(h->ld_idx[s.ld_cur], st->ld_idx, nl * 4, cudaMemcpyDefault, h->stream));
        FSNE_CUDA(h, launch_check_lists(h->ld_idx[s.ld_cur], h->N, h->k_ld, &h->sc->err, h->stream));
    }
    if ((rc = check_errors(h))) {
        clear_error_word(h);
        return fail(h, FUNCSNE_E_ARG, "imported neighbour lists are invalid (out of range, self or repeated)");
    }
    if (st->Y) {
        FSNE_CUDA(h, cudaMemsetAsync(h->Y, 0, h->yelem * 4, h->stream));
        if ((rc = copy_rows<float>(h, h->Y, h->DP, st->Y, h->d, h->N, h->d))) return rc;
    }
    if (st->V) {
        FSNE_CUDA(h, cudaMemsetAsync(h->V, 0, h->yelem * 4, h->stream));
        if ((rc = copy_rows<float>(h, h->V, h->DP, st->V, h->d, h->N, h->d))) return rc;
    }
    if (st->beta) FSNE_CUDA(h, cudaMemcpyAsync(h->beta, st->beta, static_cast<size_t>(h->N) * 4, cudaMemcpyDefault, h->stream));
    float* pin = nullptr;
    if (st->P) {
        FSNE_CUDA(h, dalloc(&pin, nh));
        FSNE_CUDA(h, cudaMemcpyAsync(pin, st->P, nh * 4, cudaMemcpyDefault, h->stream));
    }
    if (st->hd_idx || st->P) {
        FinalizeParams f{};
        f.N = h->N;
        f.k_hd = h->k_hd;
        f.n4 = h->n4;
        f.g = hd_lanes_f32(h);
        f.xpitch = h->xpitch;
        f.log_perp = std::log(h->perplexity);
        f.X32 = h->X32;
        f.idx = h->hd_idx[s.hd_cur];
        f.d2 = h->hd_d2[s.hd_cur];
        f.P = h->P;
        f.beta = h->beta;
        f.Pin = pin;
        cudaError_t e = launch_hd_finalize(f, 8 * h->num_sms, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        cudaFree(pin);
        FSNE_CUDA(h, e);
    }
    FSNE_CUDA(h, cudaMemsetAsync(h->A, 0, h->yelem * 4, h->stream));
    s.Zhat = st->Zhat;
    s.E = st->E;
    s.t = st->t;
    s.fresh_lo = st->fresh_lo;
    s.fresh_until = st->fresh_until;
    h->t_host = st->t;
    s.err = 0;
    s.ticket = 0;
    s.n_new = 0;
    FSNE_CUDA(h, cudaMemcpyAsync(h->sc, &s, sizeof(s), cudaMemcpyHostToDevice, h->stream));
    FSNE_CUDA(h, cudaStreamSynchronize(h->stream));
    return FUNCSNE_OK;
}

int funcsne_debug_step(funcsne_t* h, float* att, float* rep) {
    if (!h || !att || !rep) return fail(h, FUNCSNE_E_ARG, "NULL argument");
    float *da = nullptr, *dr = nullptr;
    FSNE_CUDA(h, dalloc(&da, h->yelem));
    cudaError_t e = dalloc(&dr, h->yelem);
    if (e != cudaSuccess) {
        cudaFree(da);
        FSNE_CUDA(h, e);
    }
    int rc = enqueue_iteration(h, h->stream, da, dr);
    if (!rc) ++h->t_host;
    if (!rc) rc = copy_rows<float>(h, att, h->d, da, h->DP, h->N, h->d);
    if (!rc) rc = copy_rows<float>(h, rep, h->d, dr, h->DP, h->N, h->d);
    e = cudaStreamSynchronize(h->stream);
    cudaFree(da);
    cudaFree(dr);
    if (rc) return rc;
    FSNE_CUDA(h, e);
    return check_errors(h);
}

int funcsne_profile_step(funcsne_t* h, int32_t n_iters, double* ms_per_kernel) {
    NvtxRange nvtx_range("funcsne_profile_step");
    if (!h || !ms_per_kernel) return fail(h, FUNCSNE_E_ARG, "NULL argument");
    if (n_iters < 1) return fail(h, FUNCSNE_E_ARG, "n_iters must be >= 1");
    const int ne = kPhases + 1;
    std::vector<cudaEvent_t> ev(static_cast<size_t>(ne) * n_iters, nullptr);
    for (auto& e : ev) FSNE_CUDA(h, cudaEventCreate(&e));
    int rc = FUNCSNE_OK;
    for (int k = 0; k < n_iters && rc == FUNCSNE_OK; ++k) {
        const StepParams p = step_params(h);
        cudaError_t e = cudaEventRecord(ev[ne * k], h->stream);
        static const char* const kPhaseNames[kPhases] = {"hd_refine", "ld_refine", "forces", "update"};
        for (int ph = 0; ph < kPhases && e == cudaSuccess; ++ph) {
            NvtxRange phase_range(kPhaseNames[ph]);
            e = launch_phase(h, ph, p, h->stream);
            if (e == cudaSuccess) e = cudaEventRecord(ev[ne * k + ph + 1], h->stream);
        }
        if (e != cudaSuccess) rc = fail(h, FUNCSNE_E_CUDA, "profile_step: %s", cudaGetErrorString(e));
    }
    double acc[kPhases] = {0.0, 0.0, 0.0, 0.0};
    if (rc == FUNCSNE_OK) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        for (int k = 0; k < n_iters && e == cudaSuccess; ++k)
            for (int ph = 0; ph < kPhases && e == cudaSuccess; ++ph) {
                float x = 0.f;
                e = cudaEventElapsedTime(&x, ev[ne * k + ph], ev[ne * k + ph + 1]);
                acc[ph] += x;
            }
        if (e != cudaSuccess) rc = fail(h, FUNCSNE_E_CUDA, "profile_step: %s", cudaGetErrorString(e));
    }
    for (auto& e : ev) cudaEventDestroy(e);
    for (int ph = 0; ph < kPhases; ++ph) ms_per_kernel[ph] = acc[ph];
    h->t_host += static_cast<uint32_t>(n_iters);
    return rc;
}

int funcsne_exact_knn(const funcsne_t* hc, const int32_t* queries, int64_t n_q, int32_t k, int32_t* idx, float* d2) {
    NvtxRange nvtx_range("funcsne_exact_knn");
    funcsne* h = const_cast<funcsne*>(hc);
    if (!h || !queries || !idx) return fail(h, FUNCSNE_E_ARG, "NULL argument");
    if (k < 1 || k > 64 || k >= h->N) return fail(h, FUNCSNE_E_ARG, "k must be in [1, min(64, N-1)]");
    if (n_q < 1) return FUNCSNE_OK;
    std::vector<int32_t> hq(static_cast<size_t>(n_q));
    FSNE_CUDA(h, cudaMemcpy(hq.data(), queries, static_cast<size_t>(n_q) * 4, cudaMemcpyDefault));
    for (int32_t q : hq)
        if (q < 0 || q >= h->N) return fail(h, FUNCSNE_E_ARG, "query index out of range");
    KnnParams kp{};
    kp.N = h->N;
    kp.n4 = h->n4;
    kp.xpitch = h->xpitch;
    kp.k = k;
    kp.RK = k <= 32 ? 1 : 2;
    kp.n_q = n_q;
    const int64_t qb = (n_q + 7) / 8;
    int64_t ns = (8LL * h->num_sms + qb - 1) / qb;
    if (ns < 1) ns = 1;
    if (ns > 256) ns = 256;
    if (ns > h->N / 64 + 1) ns = h->N / 64 + 1;
    kp.n_split = static_cast<int32_t>(ns);
    kp.X32 = h->X32;
    int32_t* dq = nullptr;
    unsigned long long* part = nullptr;
    int32_t* didx = nullptr;
    float* dd2 = nullptr;
    cudaError_t e = dalloc(&dq, static_cast<size_t>(n_q));
    if (e == cudaSuccess) e = dalloc(&part, static_cast<size_t>(n_q) * ns * 32 * kp.RK);
    if (e == cudaSuccess) e = dalloc(&didx, static_cast<size_t>(n_q) * k);
    if (e == cudaSuccess) e = dalloc(&dd2, static_cast<size_t>(n_q) * k);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dq, hq.data(), static_cast<size_t>(n_q) * 4, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) {
        kp.queries = dq;
        kp.part = part;
        kp.idx = didx;
        kp.d2 = dd2;
        e = launch_exact_knn(kp, h->stream);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(idx, didx, static_cast<size_t>(n_q) * k * 4, cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess && d2) e = cudaMemcpyAsync(d2, dd2, static_cast<size_t>(n_q) * k * 4, cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(dq);
    cudaFree(part);
    cudaFree(didx);
    cudaFree(dd2);
    FSNE_CUDA(h, e);
    return FUNCSNE_OK;
}

const char* funcsne_last_error(const funcsne_t* h) {
    return h ? h->err.c_str() : g_create_error.c_str();
}

void funcsne_destroy(funcsne_t* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

}  // extern "C"
