// Constants, device-resident scalars and kernel parameter blocks of the
// FUnc-SNE iteration. Shared by the host runtime and the kernels.
#pragma once

#include <cstdint>

namespace fsne {

// Random-stream identifiers: every draw uses the Philox counter
// (iteration, point, stream, slot) under the 64-bit seed.
constexpr uint32_t kStreamCoin = 0;
// One block per (iteration, point, slot) drives both refinements: words 0-1
// the HD candidate of slot s, words 2-3 the LD candidate of slot s.
constexpr uint32_t kStreamRefine = 1;
constexpr uint32_t kStreamMlp = 4;       // training batches
constexpr uint32_t kStreamMlpInit = 10;  // initial MLP parameters
constexpr uint32_t kStreamInsert = 5;
constexpr uint32_t kStreamInitHd = 6;
constexpr uint32_t kStreamInitLd = 7;
constexpr uint32_t kStreamInitY = 8;
constexpr uint32_t kStreamZinit = 9;
constexpr uint32_t kStreamRemove = 11;  // replacements for removed neighbours

// Candidate layout (32 per point and refinement; the paper names the
// sources but not their counts).
//   HD: slots 0-15 HD neighbour of an HD neighbour, 16-19 LD neighbour,
//       20-23 LD neighbour of an LD neighbour, 24-31 uniform random point.
//   LD: slots 0-15 LD neighbour of an LD neighbour, 16-23 HD neighbour,
//       24-31 uniform random point.
constexpr int kCand = 32;
constexpr int kHdNnEnd = 16, kHdLdNbEnd = 20, kHdLdNnEnd = 24;
constexpr int kLdNnEnd = 16, kLdHdNbEnd = 24;

// Defaults of the options coin_floor, gamma_e and gamma_z (the paper sets
// the floor to 0.05 and leaves both smoothing rates open).
constexpr double kCoinFloor = 0.05;  // refinement probability when E = 0
constexpr double kGammaE = 0.1;     // smoothing of E[N_new / N]
constexpr double kGammaZ = 0.1;     // smoothing of the normalisation estimate
constexpr double kInitYStd = 1e-4;

constexpr float kBisectTol = 1e-5f;  // |H - ln perp| in FP32
constexpr int kBisectMaxIt = 64;

constexpr int kHdAdaptive = 0, kHdAlways = 1, kHdNever = 2;

constexpr int kHashSlots = 256;  // per-warp membership set in shared memory
// The forces' set S_i = HD u LD holds up to k_hd + k_ld entries: a lower
// load factor shortens the probes (spectrum-1m forces 1.291 to 1.272 ms
// against 256 slots; 128 slots made them 1.38 ms).
constexpr int kForceHashSlots = 512;
// Per-warp queue of repulsion-only rows in the row-pair forces kernel: it
// holds fewer than (rows per pass) + 32 <= 64 entries at any time.
constexpr int kRepRing = 64;

// Device-resident scalars of the method (one per handle).
struct DevScalars {
    double E;            // smoothed fraction of points with new HD neighbours
    double Zhat;         // running estimate of sum_{k != l} w_kl
    double last_Z;       // Z_t of the last step
    uint32_t t;          // iteration counter
    int32_t hd_cur;      // current HD list buffer (0 / 1)
    int32_t ld_cur;      // current LD list buffer (0 / 1)
    int32_t last_coin;
    unsigned long long n_new;       // points flagged in the running step
    unsigned long long last_n_new;
    unsigned long long cand_scored;
    unsigned long long cand_reranked;
    uint32_t err;        // error bits
    uint32_t ticket;     // last-block detection of the update kernel
    unsigned long long n_refined;  // iterations whose coin fired (cumulative)
    // refinement window of recently inserted points: points fresh_lo .. N-1
    // refine their HD lists in every iteration with t < fresh_until, also
    // when the coin does not fire (fresh_lo = N: none)
    int64_t fresh_lo;
    uint32_t fresh_until;
};

// True when iteration t refines only the points of the insertion window.
__host__ __device__ inline bool fresh_only(const DevScalars* s, uint32_t t, bool fire, int64_t N) {
    return !fire && t < s->fresh_until && s->fresh_lo < N;
}

constexpr uint32_t kErrNonFinite = 1u;
constexpr uint32_t kErrIndex = 2u;
constexpr uint32_t kErrTimeout = 4u;  // a bounded device wait ran out

// Lanes per row for gathering rows of `bytes` bytes in the HD refinement
// (measured on GB300 over 1M-2M points, rows of 64 to 3136 bytes): two lanes
// up to 224 bytes, four up to 800, eight beyond. Wide rows read one lane per
// row thrash L1 (44 ms against 7.6 ms at 1 KB rows and 2M points).
inline int lanes_per_row(int bytes) {
    if (bytes <= 224) return 2;
    if (bytes <= 800) return 4;
    return 8;
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): multipliers of the two
// 32x32->64-bit products and the Weyl constants that bump the 64-bit key
// between rounds.
constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

// The ten round keys of a seed (round r: seed + r Weyl constants, mod 2^32
// per word). The iteration kernels draw one block per lane and point; they
// take the keys from their launch parameters instead of bumping them.
struct PhiloxKeys {
    uint32_t k0[10], k1[10];
};
inline PhiloxKeys philox_keys(uint64_t seed) {
    PhiloxKeys K;
    uint32_t a = static_cast<uint32_t>(seed), b = static_cast<uint32_t>(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        K.k0[r] = a;
        K.k1[r] = b;
        a += kPhiloxW0;
        b += kPhiloxW1;
    }
    return K;
}

struct StepParams {
    int64_t N;
    int32_t k_hd, k_ld, n_neg;
    int32_t n4;          // float4 chunks per FP32 row
    int32_t xpitch;      // floats per FP32 row
    int32_t nq;          // BF16: 16-byte chunks per row; FP8: 4-byte code words per row
    int32_t qpitch;      // bytes per quantised row
    int32_t qscale_off;  // byte offset of the FP8 row scale (error bound 4 bytes before) / the BF16 row-error bound
    int32_t hd_mode;
    double coin_p0, coin_p1;  // refinement probability coin_p0 + coin_p1 E
    int32_t smem_per_warp;  // bytes
    int32_t hd_prefetch;    // HD refinement pipelined over a warp's points (two row buffers)
    int32_t xs_floats;      // own-row floats staged per warp
    int32_t gf, ga;         // lanes per row: FP32 rows, reduced-precision rows (1, 2, 4 or 8)
    float alpha, inv_alpha, inv2N, neg_scale, log_perp;
    float q_gamma;          // relative FP32 rounding bound of a distance evaluation
    uint64_t seed;
    PhiloxKeys pk;          // round keys of seed
    const float* X32;
    const uint8_t* Xq;
    float* Y;
    float* A;
    float* R;
    int32_t* hd_idx0;
    int32_t* hd_idx1;
    float* hd_d20;
    float* hd_d21;
    int32_t* ld_idx0;
    int32_t* ld_idx1;
    float* P;
    float* beta;
    DevScalars* sc;
    double* zpart;               // one FP64 partial of Z_t per forces block
    unsigned long long* cnt;     // per HD-refinement block: n_new, scored, reranked
};

struct UpdateParams {
    int64_t n_elem;       // N * DP
    int32_t n_zpart;      // blocks of the forces kernel (Z partials)
    int32_t n_cnt;        // blocks of the HD refinement kernel (counters)
    int32_t hd_mode;
    double coin_p0, coin_p1;  // refinement probability coin_p0 + coin_p1 E
    double gamma_e, gamma_z;  // smoothing of E and of the normalisation estimate
    int64_t N;
    float lr, momentum, att, rep, exaggeration;
    int32_t exag_iters;
    uint64_t seed;
    float* Y;
    float* V;
    float* A;
    float* R;
    float* dbg_att;       // optional copies of the forces (NULL = none)
    float* dbg_rep;
    DevScalars* sc;
    const double* zpart;
    unsigned long long* cnt;
};

}  // namespace fsne
