/*
 * FUnc-SNE reference oracle: a plain, slow, double-precision CPU restatement
 * of one iteration of the method (Lambert, Couplet, Verleysen, Lee,
 * "FUnc-SNE", arXiv 2509.07681).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library. It shares no code,
 * header, table or constant generator with the CUDA path: every constant
 * used here is restated below from the written method description.
 *
 * Passages followed (paper sections / equations):
 *   Eq. 1      HD conditional affinities p_{j|i}, symmetrisation p_ij.
 *   Eq. 4      variable-tail LD kernel w_ij = (1 + |y_i - y_j|^2/alpha)^-alpha.
 *   Eq. 5      gradient 4 sum_j (p_ij - q_ij) w_ij^{1/alpha} (y_i - y_j).
 *   Eq. 6      split of the sum into HD neighbours, LD-but-not-HD neighbours,
 *              and the rest (estimated by negative sampling, Section 2.2).
 *   Section 3  joint HD/LD neighbour refinement from neighbours of neighbours
 *              and cross-space proposals; new-neighbour flags; warm-restart
 *              bandwidth recalibration; HD refinement with probability
 *              0.05 + 0.95 E[N_new/N] (floor 0.05 is an option); LD
 *              refinement every iteration;
 *              separate attraction / repulsion scaling.
 * Readings where the paper is silent (candidate counts, random-number
 * mapping, tie-break, Jacobi update order, bisection details, Z estimator,
 * smoothing rates, optimiser) are the builder's and are stated in the
 * comments next to the code that implements them.
 *
 * Parity status: every function below is pinned by a CPU test against a
 * closed form, brute force, finite differences or published known-answer
 * vectors, except the whole-run trajectory (an approximation) which is
 * compared by statistics only.
 *
 * Compile with -ffp-contract=off so that x86 and Arm hosts give identical
 * results.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads over points. Every loop that runs in parallel writes only its own
 * point's results, and every sum over points or neighbours runs in a fixed
 * index order, so the results do not depend on the thread count. */
void oracle_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
#else
    (void)n;
#endif
}

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10, from Salmon, Moraes, Dror, Shaw, "Parallel random     */
/* numbers: as easy as 1, 2, 3" (SC'11): 10 rounds of two 32x32->64     */
/* multiplies, with a Weyl-sequence key schedule.                        */
/* ------------------------------------------------------------------ */
static const uint32_t PHILOX_MUL_A = 0xD2511F53u;
static const uint32_t PHILOX_MUL_B = 0xCD9E8D57u;
static const uint32_t PHILOX_WEYL_A = 0x9E3779B9u; /* golden ratio */
static const uint32_t PHILOX_WEYL_B = 0xBB67AE85u; /* sqrt(3) - 1 */

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_WEYL_A;
            k1 += PHILOX_WEYL_B;
        }
        uint64_t prod_a = (uint64_t)PHILOX_MUL_A * (uint64_t)x0;
        uint64_t prod_b = (uint64_t)PHILOX_MUL_B * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(prod_b >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)prod_b;
        uint32_t y2 = (uint32_t)(prod_a >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)prod_a;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Random-stream identifiers (builder's reading: one Philox counter per
 * (iteration, point, purpose, slot), key = the 64-bit seed). */
enum {
    STREAM_COIN = 0,
    STREAM_REFINE = 1, /* words 0-1: HD candidate of the slot, words 2-3: LD candidate,
                          words 1 and 3 also seed the negative samples */
    STREAM_MLP = 4,
    STREAM_INSERT = 5,
    STREAM_INIT_HD = 6,
    STREAM_INIT_LD = 7,
    STREAM_INIT_Y = 8,
    STREAM_ZINIT = 9,
    STREAM_REMOVE = 11  /* replacements for neighbours that were removed */
};

/* Builder constants (the paper gives none of these). */
#define CAND_HD 32             /* HD candidates per point and iteration     */
#define CAND_LD 32             /* LD candidates per point and iteration     */
#define HD_SLOTS_NN 16         /* HD slots 0..15: HD neighbour of neighbour */
#define HD_SLOTS_LDNB 20       /* HD slots 16..19: LD neighbour             */
#define HD_SLOTS_LDNN 24       /* HD slots 20..23: LD neighbour of neighbour*/
                               /* HD slots 24..31: uniform random           */
#define LD_SLOTS_NN 16         /* LD slots 0..15: LD neighbour of neighbour */
#define LD_SLOTS_HDNB 24       /* LD slots 16..23: HD neighbour             */
                               /* LD slots 24..31: uniform random           */
#define INIT_Y_STD 1e-4        /* per-dimension std of the initial layout   */
#define INSERT_SLOTS_NN 24     /* insertion slots 0..23: neighbour of neighbour */
                               /* insertion slots 24..31: random existing point */

static void draw4(uint64_t seed, uint32_t t, uint32_t i, uint32_t stream, uint32_t slot,
                  uint32_t out[4])
{
    uint32_t ctr[4] = {t, i, stream, slot};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    oracle_philox4x32_10(ctr, key, out);
}

/* uniform integer in [0, m): the high word of u * m (no modulo). */
static int64_t map_index(uint32_t u, int64_t m)
{
    return (int64_t)(((uint64_t)u * (uint64_t)m) >> 32);
}

/* Negative sample s seeded by words 1 and 3 of the Philox block of slot
 * s mod 32: the 32-bit finalizer of MurmurHash3 (Appleby) applied to
 * w1 xor (w3 + (s div 32 + 1) * 0x9E3779B9). */
static uint32_t negative_word(uint32_t w1, uint32_t w3, uint32_t pass)
{
    uint32_t h = w1 ^ (w3 + (pass + 1u) * 0x9E3779B9u);
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

/* uniform point index in [0, N) minus {i}. */
static int64_t map_other(uint32_t u, int64_t N, int64_t i)
{
    int64_t j = map_index(u, N - 1);
    return j >= i ? j + 1 : j;
}

/* ------------------------------------------------------------------ */
/* State (all arrays owned by the caller).                              */
/* ------------------------------------------------------------------ */
typedef struct {
    int64_t N;
    int32_t D, d, k_hd, k_ld, n_neg;
    double alpha, perplexity;
    uint64_t seed;
    /* options */
    double lr, momentum, att_ratio, rep_ratio, exaggeration;
    int32_t exag_iters;   /* exaggeration applies while t < exag_iters     */
    int32_t hd_mode;      /* 0 adaptive coin, 1 always refine, 2 never     */
    int32_t neg_mode;     /* 0 Philox negatives, 1 exhaustive (pin mode)   */
    int32_t jump_iters;   /* jump start: projections instead of gradients  */
    int32_t jump_parts;   /*   while t < jump_iters, in jump_parts parts    */
    double coin_floor;    /* refinement probability floor + (1-floor) E    */
    double gamma_e;       /* smoothing rate of E[N_new/N]                  */
    double gamma_z;       /* smoothing rate of the normalisation estimate  */
    int32_t fresh_iters;  /* iterations a new point is refined for (0: off) */
    /* state */
    const double *X;      /* N x D                                          */
    double *Y, *V;        /* N x d                                          */
    int32_t *hd_idx;      /* N x k_hd, ordered by (d2, idx)                 */
    double *hd_d2;        /* N x k_hd                                       */
    int32_t *ld_idx;      /* N x k_ld                                       */
    double *beta;         /* N: 1/(2 sigma_i^2)                              */
    double *P;            /* N x k_hd: p_{j|i} aligned with hd_idx           */
    double Zhat, E;
    uint32_t t;
    int64_t fresh_lo;     /* points fresh_lo .. N-1 were inserted recently   */
    uint32_t fresh_until; /* ... and are refined while t < fresh_until      */
} oracle_state;

/* Squared Euclidean distance, the plain definition. */
static double sqdist(const double *a, const double *b, int n)
{
    double s = 0.0;
    for (int f = 0; f < n; ++f) {
        double diff = a[f] - b[f];
        s += diff * diff;
    }
    return s;
}

double oracle_sqdist(const double *a, const double *b, int n) { return sqdist(a, b, n); }

/* Order on (distance, index): ascending distance, ties by smaller index. */
typedef struct { double d2; int64_t idx; } entry;

static int entry_cmp(const void *pa, const void *pb)
{
    const entry *a = (const entry *)pa, *b = (const entry *)pb;
    if (a->d2 < b->d2) return -1;
    if (a->d2 > b->d2) return 1;
    if (a->idx < b->idx) return -1;
    if (a->idx > b->idx) return 1;
    return 0;
}

static int contains(const int32_t *list, int n, int64_t v)
{
    for (int a = 0; a < n; ++a)
        if (list[a] == v) return 1;
    return 0;
}

/*
 * Top-k merge (Section 3, neighbour-set refinement): the new set is the k
 * smallest (d2, idx) among the old set and the candidates. Candidates equal
 * to i, already in the old set, or repeated among earlier candidates are
 * dropped first. Returns 1 when at least one candidate entered the set.
 */
int oracle_topk_merge(int64_t i, int k, const int32_t *old_idx, const double *old_d2,
                      int n_cand, const int64_t *cand_idx, const double *cand_d2,
                      int32_t *new_idx, double *new_d2)
{
    entry *u = (entry *)malloc(sizeof(entry) * (size_t)(k + n_cand));
    int n = 0;
    for (int a = 0; a < k; ++a) {
        u[n].d2 = old_d2[a];
        u[n].idx = old_idx[a];
        ++n;
    }
    for (int s = 0; s < n_cand; ++s) {
        int64_t c = cand_idx[s];
        if (c == i || contains(old_idx, k, c)) continue;
        int seen = 0;
        for (int r = 0; r < s; ++r)
            if (cand_idx[r] == c) seen = 1;
        if (seen) continue;
        u[n].d2 = cand_d2[s];
        u[n].idx = c;
        ++n;
    }
    qsort(u, (size_t)n, sizeof(entry), entry_cmp);
    int changed = 0;
    for (int a = 0; a < k; ++a)
        if (!contains(old_idx, k, u[a].idx)) changed = 1;
    /* an unchanged set keeps its stored order (its p_{j|i} stay aligned) */
    for (int a = 0; a < k; ++a) {
        new_idx[a] = changed ? (int32_t)u[a].idx : old_idx[a];
        new_d2[a] = changed ? u[a].d2 : old_d2[a];
    }
    free(u);
    return changed;
}

/*
 * LD merge (Section 3, LD refinement). The LD list is re-ordered every
 * iteration: the old entries (with their distances at Y_t) and the
 * candidates that are not i, not listed and not repeated in an earlier slot
 * are ordered by (d2, idx), and the first k are the new list, even when no
 * candidate entered (the old order was by the distances at Y_{t-1}). idx and
 * d2 are replaced in place. Returns 1 when the set changed.
 */
int oracle_ld_merge(int64_t i, int k, int32_t *idx, double *d2, int n_cand, const int64_t *cand_idx,
                    const double *cand_d2)
{
    entry *u = (entry *)malloc(sizeof(entry) * (size_t)(k + n_cand));
    int n = 0;
    for (int a = 0; a < k; ++a) {
        u[n].d2 = d2[a];
        u[n].idx = idx[a];
        ++n;
    }
    for (int s = 0; s < n_cand; ++s) {
        int64_t c = cand_idx[s];
        if (c == i || contains(idx, k, c)) continue;
        int seen = 0;
        for (int r = 0; r < s; ++r)
            if (cand_idx[r] == c) seen = 1;
        if (seen) continue;
        u[n].d2 = cand_d2[s];
        u[n].idx = c;
        ++n;
    }
    qsort(u, (size_t)n, sizeof(entry), entry_cmp);
    int changed = 0;
    for (int a = 0; a < k; ++a)
        if (!contains(idx, k, u[a].idx)) changed = 1;
    for (int a = 0; a < k; ++a) {
        idx[a] = (int32_t)u[a].idx;
        d2[a] = u[a].d2;
    }
    free(u);
    return changed;
}

/*
 * HD candidates of point i at iteration t (Section 3: neighbours of
 * neighbours, with the LD sets proposing candidates for the HD set).
 * Slot s uses words w0, w1 of the Philox block at counter (t, i, REFINE, s):
 *   s in [0,16):  a = N_HD(i)[w0 * k_hd], c = N_HD(a)[w1 * k_hd]
 *   s in [16,20): c = N_LD(i)[w0 * k_ld]
 *   s in [20,24): a = N_LD(i)[w0 * k_ld], c = N_LD(a)[w1 * k_ld]
 *   s in [24,32): c uniform over the other points (w0)
 * where "w * m" denotes the high word of the 64-bit product.
 */
void oracle_hd_candidates(const oracle_state *st, int64_t i, int64_t *cand)
{
    for (int s = 0; s < CAND_HD; ++s) {
        uint32_t w[4];
        draw4(st->seed, st->t, (uint32_t)i, STREAM_REFINE, (uint32_t)s, w);
        int64_t c;
        if (s < HD_SLOTS_NN) {
            int64_t a = st->hd_idx[i * st->k_hd + map_index(w[0], st->k_hd)];
            c = st->hd_idx[a * st->k_hd + map_index(w[1], st->k_hd)];
        } else if (s < HD_SLOTS_LDNB) {
            c = st->ld_idx[i * st->k_ld + map_index(w[0], st->k_ld)];
        } else if (s < HD_SLOTS_LDNN) {
            int64_t a = st->ld_idx[i * st->k_ld + map_index(w[0], st->k_ld)];
            c = st->ld_idx[a * st->k_ld + map_index(w[1], st->k_ld)];
        } else {
            c = map_other(w[0], st->N, i);
        }
        cand[s] = c;
    }
}

/*
 * LD candidates of point i at iteration t. Slot s uses words w2, w3 of the
 * Philox block at counter (t, i, REFINE, s) (the HD slot s uses w0, w1):
 *   s in [0,16):  a = N_LD(i)[w2 * k_ld], c = N_LD(a)[w3 * k_ld]
 *   s in [16,24): c = N_HD(i)[w2 * k_hd]   (HD set of iteration t)
 *   s in [24,32): c uniform over the other points (w2)
 */
void oracle_ld_candidates(const oracle_state *st, int64_t i, int64_t *cand)
{
    for (int s = 0; s < CAND_LD; ++s) {
        uint32_t w[4];
        draw4(st->seed, st->t, (uint32_t)i, STREAM_REFINE, (uint32_t)s, w);
        int64_t c;
        if (s < LD_SLOTS_NN) {
            int64_t a = st->ld_idx[i * st->k_ld + map_index(w[2], st->k_ld)];
            c = st->ld_idx[a * st->k_ld + map_index(w[3], st->k_ld)];
        } else if (s < LD_SLOTS_HDNB) {
            c = st->hd_idx[i * st->k_hd + map_index(w[2], st->k_hd)];
        } else {
            c = map_other(w[2], st->N, i);
        }
        cand[s] = c;
    }
}

/* Shannon entropy (natural log) of p_{.|i} for bandwidth beta = 1/(2 sigma^2),
 * from Eq. 1 restricted to the k listed neighbours. Writes P when non-NULL. */
double oracle_entropy(const double *d2, int k, double beta, double *P)
{
    double dmin = d2[0];
    for (int a = 1; a < k; ++a)
        if (d2[a] < dmin) dmin = d2[a];
    double *e = (double *)malloc(sizeof(double) * (size_t)k);
    double sum = 0.0;
    for (int a = 0; a < k; ++a) {
        e[a] = exp(-beta * (d2[a] - dmin));
        sum += e[a];
    }
    double h = 0.0;
    for (int a = 0; a < k; ++a) {
        double p = e[a] / sum;
        if (P) P[a] = p;
        if (p > 0.0) h -= p * log(p);
    }
    free(e);
    return h;
}

/*
 * Perplexity calibration of sigma_i (Eq. 1): find beta with entropy equal
 * to ln(perplexity). The entropy decreases in beta, so: start from beta0
 * (the previous value: warm restart, Section 3) or, when beta0 <= 0, from
 * 1 / mean(d2 - d2_min); double beta until the entropy drops below the
 * target, then bisect, stopping when |H - ln perp| < tol or after maxit
 * evaluations. When ln k <= ln perp no beta reaches the target and the
 * uniform distribution (beta = 0) is returned.
 * Returns the number of entropy evaluations.
 */
int oracle_bisect(const double *d2, int k, double perplexity, double beta0, double tol,
                  int maxit, double *beta_out, double *P)
{
    double target = log(perplexity);
    if (log((double)k) <= target) {
        for (int a = 0; a < k; ++a) P[a] = 1.0 / k;
        *beta_out = 0.0;
        return 0;
    }
    double beta = beta0;
    if (!(beta > 0.0)) {
        double dmin = d2[0], mean = 0.0;
        for (int a = 1; a < k; ++a)
            if (d2[a] < dmin) dmin = d2[a];
        for (int a = 0; a < k; ++a) mean += d2[a] - dmin;
        mean /= k;
        beta = mean > 0.0 ? 1.0 / mean : 1.0;
    }
    double lo = 0.0, hi = INFINITY;
    int it = 0;
    while (it < maxit) {
        double h = oracle_entropy(d2, k, beta, NULL);
        ++it;
        if (fabs(h - target) < tol) break;
        if (h > target) {
            lo = beta;
            beta = isinf(hi) ? 2.0 * beta : 0.5 * (lo + hi);
        } else {
            hi = beta;
            beta = 0.5 * (lo + hi);
        }
    }
    oracle_entropy(d2, k, beta, P);
    *beta_out = beta;
    return it;
}

/* Eq. 4: w = (1 + r2/alpha)^-alpha and its power w^{1/alpha} = 1/(1 + r2/alpha). */
static double kernel_w(double r2, double alpha) { return pow(1.0 + r2 / alpha, -alpha); }
static double kernel_w_inv_alpha(double r2, double alpha) { return 1.0 / (1.0 + r2 / alpha); }

/* Initial neighbour list: k distinct other points. Slot l draws an offset
 * o_l uniform in [0, N-1) from counter (0, i, stream, l); an offset already
 * taken moves to the next free one (linear probing mod N-1). The neighbour
 * is (i + 1 + o_l) mod N. */
void oracle_initial_list(uint64_t seed, int64_t N, int64_t i, int k, uint32_t stream, int32_t *out)
{
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    for (int l = 0; l < k; ++l) {
        uint32_t w[4];
        draw4(seed, 0u, (uint32_t)i, stream, (uint32_t)l, w);
        int64_t o = map_index(w[0], N - 1);
        for (;;) {
            int taken = 0;
            for (int m = 0; m < l; ++m)
                if (off[m] == o) taken = 1;
            if (!taken) break;
            o = (o + 1) % (N - 1);
        }
        off[l] = o;
        out[l] = (int32_t)((i + 1 + o) % N);
    }
    free(off);
}

/* Gaussian N(0,1) from two uniform words (Box-Muller). */
static double gauss_from(uint32_t a, uint32_t b)
{
    double u1 = ((double)a + 0.5) * (1.0 / 4294967296.0);
    double u2 = ((double)b + 0.5) * (1.0 / 4294967296.0);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* Sorts one HD list of point i by (d2, idx) with distances recomputed. */
static void sort_hd_list(oracle_state *st, int64_t i)
{
    int k = st->k_hd;
    entry *u = (entry *)malloc(sizeof(entry) * (size_t)k);
    for (int a = 0; a < k; ++a) {
        int64_t j = st->hd_idx[i * k + a];
        u[a].idx = j;
        u[a].d2 = sqdist(st->X + i * st->D, st->X + j * st->D, st->D);
    }
    qsort(u, (size_t)k, sizeof(entry), entry_cmp);
    for (int a = 0; a < k; ++a) {
        st->hd_idx[i * k + a] = (int32_t)u[a].idx;
        st->hd_d2[i * k + a] = u[a].d2;
    }
    free(u);
}

/*
 * Repulsion, attraction and the normalisation estimate (Eq. 5 split as in
 * Eq. 6), for the lists currently in hd_idx / ld_idx, with Y, P and Zhat of
 * the state. A and R are N x d, zeroed here. Returns Z_t, the estimate of
 * sum_{k != l} w_kl. In exhaustive mode the third term of Eq. 6 is summed
 * over every other point with factor 1 instead of being sampled.
 *
 *   attraction: for j in N_HD(i), f = 4 (p_{j|i} / 2N) w^{1/alpha} (y_i - y_j)
 *               is added to A_i and subtracted from A_j, which realises
 *               p_ij = (p_{j|i} + p_{i|j}) / 2N with p_{i|j} = 0 when i is
 *               not in N_HD(j);
 *   repulsion:  for j in S_i = N_HD(i) u N_LD(i):
 *               R_i += 4 (w_ij / Zhat) w^{1/alpha} (y_i - y_j);
 *               negatives s < n_neg: j_s uniform over the other points from
 *               negative_word of the block (t, i, stream, s mod 32), where
 *               stream is REFINE in an iteration (the block that also draws
 *               the candidates of slot s) and ZINIT for the first estimate;
 *               a draw inside S_i contributes 0; the others are scaled by
 *               (N-1)/n_neg.
 */
double oracle_forces(const oracle_state *st, uint32_t t, uint32_t neg_stream, double zhat,
                     double *A, double *R, double *z_per_point)
{
    int64_t N = st->N;
    int d = st->d, kh = st->k_hd, kl = st->k_ld;
    double alpha = st->alpha;
    /* the lists that hold each point: (source i, slot a) with
     * hd_idx[i kh + a] = j, by increasing i, for the reverse attraction */
    int64_t *rstart = (int64_t *)calloc((size_t)(N + 1), sizeof(int64_t));
    int64_t *rsrc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N * kh > 0 ? N * kh : 1));
    for (int64_t e = 0; e < N * kh; ++e) rstart[st->hd_idx[e] + 1] += 1;
    for (int64_t j = 0; j < N; ++j) rstart[j + 1] += rstart[j];
    {
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
        memcpy(fill, rstart, sizeof(int64_t) * (size_t)N);
        for (int64_t e = 0; e < N * kh; ++e) rsrc[fill[st->hd_idx[e]]++] = e;
        free(fill);
    }
    double *zpt = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
#pragma omp parallel
    {
        int32_t *S = (int32_t *)malloc(sizeof(int32_t) * (size_t)(kh + kl));
        char *inS = NULL;
        if (st->neg_mode == 1) inS = (char *)malloc((size_t)N);
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < N; ++i) {
            const double *yi = st->Y + i * d;
            double *Ai = A + i * d, *Ri = R + i * d;
            for (int c = 0; c < d; ++c) Ai[c] = Ri[c] = 0.0;
            /* attraction: the pairs of i's own list, in list order ... */
            for (int a = 0; a < kh; ++a) {
                int64_t j = st->hd_idx[i * kh + a];
                const double *yj = st->Y + j * d;
                double r2 = sqdist(yi, yj, d);
                double coef = 4.0 * (st->P[i * kh + a] / (2.0 * (double)N)) * kernel_w_inv_alpha(r2, alpha);
                for (int c = 0; c < d; ++c) Ai[c] += coef * (yi[c] - yj[c]);
            }
            /* ... then the pairs of the lists that hold i (p_{i|s} of Eq. 1,
             * symmetrised), by increasing source s */
            for (int64_t q = rstart[i]; q < rstart[i + 1]; ++q) {
                int64_t e = rsrc[q], src = e / kh;
                const double *ys = st->Y + src * d;
                double r2 = sqdist(ys, yi, d);
                double coef = 4.0 * (st->P[e] / (2.0 * (double)N)) * kernel_w_inv_alpha(r2, alpha);
                for (int c = 0; c < d; ++c) Ai[c] -= coef * (ys[c] - yi[c]);
            }
            /* S_i = HD list, then LD entries not in the HD list */
            int ns = 0;
            for (int a = 0; a < kh; ++a) S[ns++] = st->hd_idx[i * kh + a];
            for (int a = 0; a < kl; ++a) {
                int32_t j = st->ld_idx[i * kl + a];
                if (!contains(st->hd_idx + i * kh, kh, j)) S[ns++] = j;
            }
            double zi = 0.0;
            for (int a = 0; a < ns; ++a) {
                const double *yj = st->Y + (int64_t)S[a] * d;
                double r2 = sqdist(yi, yj, d);
                double w = kernel_w(r2, alpha);
                double coef = 4.0 * (w / zhat) * kernel_w_inv_alpha(r2, alpha);
                for (int c = 0; c < d; ++c) Ri[c] += coef * (yi[c] - yj[c]);
                zi += w;
            }
            if (st->neg_mode == 1) {
                memset(inS, 0, (size_t)N);
                for (int a = 0; a < ns; ++a) inS[S[a]] = 1;
                for (int64_t j = 0; j < N; ++j) {
                    if (j == i || inS[j]) continue;
                    const double *yj = st->Y + j * d;
                    double r2 = sqdist(yi, yj, d);
                    double w = kernel_w(r2, alpha);
                    double coef = 4.0 * (w / zhat) * kernel_w_inv_alpha(r2, alpha);
                    for (int c = 0; c < d; ++c) Ri[c] += coef * (yi[c] - yj[c]);
                    zi += w;
                }
            } else {
                double scale = (double)(N - 1) / (double)st->n_neg;
                for (int s = 0; s < st->n_neg; ++s) {
                    uint32_t w4[4];
                    draw4(st->seed, t, (uint32_t)i, neg_stream, (uint32_t)(s % 32), w4);
                    int64_t j = map_other(negative_word(w4[1], w4[3], (uint32_t)(s / 32)), N, i);
                    if (contains(S, ns, j)) continue;
                    const double *yj = st->Y + j * d;
                    double r2 = sqdist(yi, yj, d);
                    double w = kernel_w(r2, alpha);
                    double coef = scale * 4.0 * (w / zhat) * kernel_w_inv_alpha(r2, alpha);
                    for (int c = 0; c < d; ++c) Ri[c] += coef * (yi[c] - yj[c]);
                    zi += scale * w;
                }
            }
            zpt[i] = zi;
        }
        free(S);
        free(inS);
    }
    double ztotal = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        if (z_per_point) z_per_point[i] = zpt[i];
        ztotal += zpt[i];
    }
    free(zpt);
    free(rstart);
    free(rsrc);
    return ztotal;
}

/*
 * Y = (X - mean) R, a random linear projection of the data: R_fc ~ N(0, 1)
 * by Box-Muller from the Philox block at counter (ctr, f, INIT_Y, c), each
 * LD dimension then rescaled to standard deviation INIT_Y_STD. ctr = 0 is
 * the initial layout; the jump start uses ctr = 1, 2, ... (Section 3).
 */
static void project_y(oracle_state *st, uint32_t ctr)
{
    int64_t N = st->N;
    int D = st->D, d = st->d;
    double *Rm = (double *)malloc(sizeof(double) * (size_t)(D * d));
    for (int f = 0; f < D; ++f)
        for (int c = 0; c < d; ++c) {
            uint32_t w[4];
            draw4(st->seed, ctr, (uint32_t)f, STREAM_INIT_Y, (uint32_t)c, w);
            Rm[f * d + c] = gauss_from(w[0], w[1]);
        }
    double *mu = (double *)calloc((size_t)(D > 0 ? D : 1), sizeof(double));
    for (int64_t i = 0; i < N; ++i)
        for (int f = 0; f < D; ++f) mu[f] += st->X[i * D + f];
    for (int f = 0; f < D; ++f) mu[f] /= (double)N;
    for (int64_t i = 0; i < N; ++i)
        for (int c = 0; c < d; ++c) {
            double s = 0.0;
            for (int f = 0; f < D; ++f) s += (st->X[i * D + f] - mu[f]) * Rm[f * d + c];
            st->Y[i * d + c] = s;
        }
    for (int c = 0; c < d; ++c) {
        double m = 0.0, v = 0.0;
        for (int64_t i = 0; i < N; ++i) m += st->Y[i * d + c];
        m /= (double)N;
        for (int64_t i = 0; i < N; ++i) v += (st->Y[i * d + c] - m) * (st->Y[i * d + c] - m);
        double sd = sqrt(v / (double)N);
        double scale = sd > 0.0 ? INIT_Y_STD / sd : 1.0;
        for (int64_t i = 0; i < N; ++i) st->Y[i * d + c] *= scale;
    }
    free(Rm);
    free(mu);
}

/*
 * Initial state: random distinct HD and LD lists (HD lists sorted by
 * (d2, idx)), Y0 = (X - mean) R with R_fc ~ N(0,1) from counter
 * (0, f, INIT_Y, c), each LD dimension rescaled to std 1e-4 (a random linear
 * projection, Section 3's jump-start idea), V = 0, every beta calibrated
 * from a cold start, E = 1, t = 0, and Zhat = the Z estimate of this state
 * with negatives from the ZINIT stream.
 */
void oracle_init(oracle_state *st, double bisect_tol, int bisect_maxit)
{
    int64_t N = st->N;
    int D = st->D, d = st->d, kh = st->k_hd, kl = st->k_ld;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < N; ++i) {
        oracle_initial_list(st->seed, N, i, kh, STREAM_INIT_HD, st->hd_idx + i * kh);
        sort_hd_list(st, i);
        oracle_initial_list(st->seed, N, i, kl, STREAM_INIT_LD, st->ld_idx + i * kl);
    }
    project_y(st, 0u);
    memset(st->V, 0, sizeof(double) * (size_t)(N * d));
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < N; ++i)
        oracle_bisect(st->hd_d2 + i * kh, kh, st->perplexity, 0.0, bisect_tol, bisect_maxit,
                      st->beta + i, st->P + i * kh);
    st->E = 1.0;
    st->t = 0;
    double *A = (double *)malloc(sizeof(double) * (size_t)(N * d));
    double *R = (double *)malloc(sizeof(double) * (size_t)(N * d));
    st->Zhat = 1.0;
    st->Zhat = oracle_forces(st, 0u, STREAM_ZINIT, 1.0, A, R, NULL);
    free(A);
    free(R);
}

/* Coin for HD refinement at iteration t: refine iff the uniform draw from
 * counter (t, 0, COIN, 0) is below floor + (1 - floor) E; the paper sets
 * the floor to 0.05 (Section 3). */
int oracle_coin(const oracle_state *st)
{
    if (st->hd_mode == 1) return 1;
    if (st->hd_mode == 2) return 0;
    uint32_t w[4];
    draw4(st->seed, st->t, 0u, STREAM_COIN, 0u, w);
    double p = st->coin_floor + (1.0 - st->coin_floor) * st->E;
    double u = (double)w[0] * (1.0 / 4294967296.0);
    return u < p;
}

/*
 * One iteration (Jacobi: every point reads the state of iteration t and
 * writes iteration t+1):
 *   1. coin; if it fires, HD refinement of every point from the lists of t,
 *      flags for points whose set changed, and warm-restart recalibration of
 *      beta and P for flagged points; if it does not fire but points were
 *      inserted within the last fresh_iters iterations (t < fresh_until),
 *      the same refinement of only those points (fresh_lo .. N-1), which
 *      leaves E unchanged;
 *   2. LD refinement of every point from the lists of t and Y_t;
 *   3. forces with the new lists, P and Y_t, Zhat_t;
 *   4. g = att * exag * A - rep * R; V = momentum V - lr g; Y += V;
 *      Zhat <- (1 - gamma_z) Zhat + gamma_z Z_t; E <- (1 - gamma_e) E +
 *      gamma_e N_new/N when the coin fired (both rates 0.1 by default);
 *      t <- t + 1.
 * A_out / R_out (N x d) receive the forces of step 3; flags (N bytes) the
 * new-neighbour flags; info[0] = coin, info[1] = N_new. z_out (N) receives
 * the per-point Z terms when non-NULL.
 */
void oracle_step(oracle_state *st, double bisect_tol, int bisect_maxit, double *A_out,
                 double *R_out, uint8_t *flags, int64_t *info, double *z_out)
{
    int64_t N = st->N;
    int D = st->D, d = st->d, kh = st->k_hd, kl = st->k_ld;
    int32_t *nh_idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N * kh));
    double *nh_d2 = (double *)malloc(sizeof(double) * (size_t)(N * kh));
    int32_t *nl_idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N * kl));
    memcpy(nh_idx, st->hd_idx, sizeof(int32_t) * (size_t)(N * kh));
    memcpy(nh_d2, st->hd_d2, sizeof(double) * (size_t)(N * kh));
    memset(flags, 0, (size_t)N);

    /* jump start (Section 3): while t < jump_iters, Y is a random linear
     * projection of the data, renewed at the start of each of jump_parts
     * equal parts (t = floor(p * jump_iters / jump_parts)), and no gradient
     * is applied */
    int jump = st->t < (uint32_t)st->jump_iters;
    if (jump) {
        int parts = st->jump_parts > 0 ? st->jump_parts : 1;
        for (int p = 0; p < parts; ++p)
            if ((int64_t)st->t == ((int64_t)p * st->jump_iters) / parts) project_y(st, (uint32_t)(p + 1));
    }
    int fire = oracle_coin(st);
    /* recently inserted points are refined in every iteration of their
     * window (an addition for points added on the fly, Section 3) */
    int fresh = !fire && st->fresh_iters > 0 && st->t < st->fresh_until && st->fresh_lo < N;
    int64_t lo = fire ? 0 : st->fresh_lo;
    int64_t n_new = 0;
    if (fire || fresh) {
#pragma omp parallel
        {
            int64_t cand[CAND_HD];
            double cd2[CAND_HD];
            double *old_d2 = (double *)malloc(sizeof(double) * (size_t)kh);
#pragma omp for schedule(dynamic, 64)
            for (int64_t i = lo; i < N; ++i) {
                oracle_hd_candidates(st, i, cand);
                for (int s = 0; s < CAND_HD; ++s)
                    cd2[s] = (cand[s] == i) ? 0.0 : sqdist(st->X + i * D, st->X + cand[s] * D, D);
                for (int a = 0; a < kh; ++a)
                    old_d2[a] = sqdist(st->X + i * D, st->X + (int64_t)st->hd_idx[i * kh + a] * D, D);
                flags[i] = (uint8_t)oracle_topk_merge(i, kh, st->hd_idx + i * kh, old_d2, CAND_HD,
                                                      cand, cd2, nh_idx + i * kh, nh_d2 + i * kh);
            }
            free(old_d2);
        }
        for (int64_t i = lo; i < N; ++i) n_new += flags[i];
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t i = lo; i < N; ++i)
            if (flags[i])
                oracle_bisect(nh_d2 + i * kh, kh, st->perplexity, st->beta[i], bisect_tol,
                              bisect_maxit, st->beta + i, st->P + i * kh);
    }
#pragma omp parallel
    {
        int64_t cand[CAND_LD];
        double cd2[CAND_LD];
        double *ld_new_d2 = (double *)malloc(sizeof(double) * (size_t)kl);
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < N; ++i) {
            oracle_ld_candidates(st, i, cand);
            for (int s = 0; s < CAND_LD; ++s)
                cd2[s] = (cand[s] == i) ? 0.0 : sqdist(st->Y + i * d, st->Y + cand[s] * d, d);
            for (int a = 0; a < kl; ++a) {
                nl_idx[i * kl + a] = st->ld_idx[i * kl + a];
                ld_new_d2[a] = sqdist(st->Y + i * d, st->Y + (int64_t)st->ld_idx[i * kl + a] * d, d);
            }
            oracle_ld_merge(i, kl, nl_idx + i * kl, ld_new_d2, CAND_LD, cand, cd2);
        }
        free(ld_new_d2);
    }
    /* install the lists of iteration t+1 before the forces */
    memcpy(st->hd_idx, nh_idx, sizeof(int32_t) * (size_t)(N * kh));
    memcpy(st->hd_d2, nh_d2, sizeof(double) * (size_t)(N * kh));
    memcpy(st->ld_idx, nl_idx, sizeof(int32_t) * (size_t)(N * kl));
    free(nh_idx);
    free(nh_d2);
    free(nl_idx);

    double zt = oracle_forces(st, st->t, STREAM_REFINE, st->Zhat, A_out, R_out, z_out);
    double exag = (st->t < (uint32_t)st->exag_iters) ? st->exaggeration : 1.0;
    for (int64_t e = 0; e < N * d; ++e) {
        double g = st->att_ratio * exag * A_out[e] - st->rep_ratio * R_out[e];
        st->V[e] = jump ? 0.0 : st->momentum * st->V[e] - st->lr * g;
        st->Y[e] = st->Y[e] + st->V[e];
    }
    st->Zhat = (1.0 - st->gamma_z) * st->Zhat + st->gamma_z * zt;
    if (fire) st->E = (1.0 - st->gamma_e) * st->E + st->gamma_e * ((double)n_new / (double)N);
    st->t += 1;
    info[0] = fire;
    info[1] = n_new;
}

/* ------------------------------------------------------------------ */
/* Exact (dense) references, for small N.                               */
/* ------------------------------------------------------------------ */

/* Dense symmetric P (N x N) from sparse lists: p_ij = (p_{j|i} + p_{i|j}) / 2N
 * with p_{j|i} = 0 when j is not listed for i (Eq. 1). */
void oracle_dense_p(const oracle_state *st, double *Pd)
{
    int64_t N = st->N;
    int kh = st->k_hd;
    memset(Pd, 0, sizeof(double) * (size_t)(N * N));
    for (int64_t i = 0; i < N; ++i)
        for (int a = 0; a < kh; ++a) {
            int64_t j = st->hd_idx[i * kh + a];
            double v = st->P[i * kh + a] / (2.0 * (double)N);
            Pd[i * N + j] += v;
            Pd[j * N + i] += v;
        }
}

/* Z = sum_{k != l} w_kl (Eq. 4), exactly. */
double oracle_exact_z(const double *Y, int64_t N, int d, double alpha)
{
    double z = 0.0;
    for (int64_t k = 0; k < N; ++k)
        for (int64_t l = 0; l < N; ++l)
            if (k != l) z += kernel_w(sqdist(Y + k * d, Y + l * d, d), alpha);
    return z;
}

/* KL(P || Q) = sum_{i != j} p_ij log(p_ij / q_ij) with q_ij = w_ij / Z
 * (Section 2.2 and Eq. 4). Terms with p_ij = 0 contribute 0. */
double oracle_kl(const double *Pd, const double *Y, int64_t N, int d, double alpha)
{
    double z = oracle_exact_z(Y, N, d, alpha);
    double kl = 0.0;
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < N; ++j) {
            if (i == j) continue;
            double p = Pd[i * N + j];
            if (p <= 0.0) continue;
            double q = kernel_w(sqdist(Y + i * d, Y + j * d, d), alpha) / z;
            kl += p * log(p / q);
        }
    return kl;
}

/* Eq. 5: dL/dy_i = 4 sum_j (p_ij - q_ij) w_ij^{1/alpha} (y_i - y_j). */
void oracle_exact_grad(const double *Pd, const double *Y, int64_t N, int d, double alpha,
                       double *G)
{
    double z = oracle_exact_z(Y, N, d, alpha);
    memset(G, 0, sizeof(double) * (size_t)(N * d));
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < N; ++j) {
            if (i == j) continue;
            double r2 = sqdist(Y + i * d, Y + j * d, d);
            double q = kernel_w(r2, alpha) / z;
            double coef = 4.0 * (Pd[i * N + j] - q) * kernel_w_inv_alpha(r2, alpha);
            for (int c = 0; c < d; ++c) G[i * d + c] += coef * (Y[i * d + c] - Y[j * d + c]);
        }
}

/* Exact k nearest neighbours of every row of X by brute force, ordered by
 * (d2, idx); self excluded. */
void oracle_bruteforce_knn(const double *X, int64_t N, int D, int k, int32_t *idx, double *d2)
{
    entry *u = (entry *)malloc(sizeof(entry) * (size_t)N);
    for (int64_t i = 0; i < N; ++i) {
        int64_t n = 0;
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            u[n].idx = j;
            u[n].d2 = sqdist(X + i * D, X + j * D, D);
            ++n;
        }
        qsort(u, (size_t)n, sizeof(entry), entry_cmp);
        for (int a = 0; a < k; ++a) {
            idx[i * k + a] = (int32_t)u[a].idx;
            d2[i * k + a] = u[a].d2;
        }
    }
    free(u);
}

/* Exact k nearest neighbours of a few query rows (indices q) in X. */
void oracle_query_knn(const double *X, int64_t N, int D, const int64_t *q, int64_t nq, int k,
                      int32_t *idx, double *d2)
{
    entry *u = (entry *)malloc(sizeof(entry) * (size_t)N);
    for (int64_t a = 0; a < nq; ++a) {
        int64_t i = q[a];
        int64_t n = 0;
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            u[n].idx = j;
            u[n].d2 = sqdist(X + i * D, X + j * D, D);
            ++n;
        }
        qsort(u, (size_t)n, sizeof(entry), entry_cmp);
        for (int b = 0; b < k; ++b) {
            idx[a * k + b] = (int32_t)u[b].idx;
            d2[a * k + b] = u[b].d2;
        }
    }
    free(u);
}

/* ------------------------------------------------------------------ */
/* Insertion of new points (Section 3: points can be added on the fly;  */
/* the builder's reading of how a new point enters the state).          */
/* ------------------------------------------------------------------ */

/* Mean placement of a new point: the average LD position of its HD
 * neighbours (all of them existing points). */
static void place_mean(oracle_state *st, int64_t i)
{
    int d = st->d, kh = st->k_hd;
    for (int c = 0; c < d; ++c) {
        double s = 0.0;
        for (int a = 0; a < kh; ++a) s += st->Y[(int64_t)st->hd_idx[i * kh + a] * d + c];
        st->Y[i * d + c] = s / kh;
    }
}

/*
 * Insert the rows n_old .. st->N - 1 (their X rows already in place, every
 * other array already sized for st->N) at iteration t = st->t:
 *   1. HD list: k_hd distinct existing points, slot l drawing an offset in
 *      [0, n_old) from counter (t, i, INSERT, l), linear probing mod n_old;
 *      ordered by (d2, idx);
 *   2. `rounds` rounds of 32 candidates, round r slot s from counter
 *      (t, i, INSERT, 64 + 32 r + s): slots 0..23 a = list(i)[w0 * k_hd],
 *      c = list(a)[w1 * k_hd] (a is an existing point, its list of
 *      iteration t); slots 24..31 a uniform existing point; top-k merge;
 *   3. cold-start bisection for beta and P;
 *   4. Y = mean of the HD neighbours' Y (placement 0); V = 0;
 *   5. LD list = the first k_ld HD neighbours, completed (when k_ld > k_hd)
 *      by distinct random existing points from counter (t, i, INSERT, 2^30 + l)
 *      (above every round's slots);
 *   6. Zhat scaled by the ratio of ordered pair counts, E = max(E, n_new/N).
 * Placement 1 (a learned map) is handled by the caller, which overwrites Y.
 */
void oracle_insert(oracle_state *st, int64_t n_old, int rounds, double bisect_tol, int bisect_maxit)
{
    int64_t N = st->N;
    int D = st->D, kh = st->k_hd, kl = st->k_ld;
    int64_t cand[CAND_HD];
    double cd2[CAND_HD];
    int32_t *list = (int32_t *)malloc(sizeof(int32_t) * (size_t)kh);
    double *ld2 = (double *)malloc(sizeof(double) * (size_t)kh);
    int32_t *nl = (int32_t *)malloc(sizeof(int32_t) * (size_t)kh);
    double *nd2 = (double *)malloc(sizeof(double) * (size_t)kh);
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(kh > kl ? kh : kl));
    for (int64_t i = n_old; i < N; ++i) {
        for (int l = 0; l < kh; ++l) {
            uint32_t w[4];
            draw4(st->seed, st->t, (uint32_t)i, STREAM_INSERT, (uint32_t)l, w);
            int64_t o = map_index(w[0], n_old);
            for (;;) {
                int taken = 0;
                for (int m = 0; m < l; ++m)
                    if (off[m] == o) taken = 1;
                if (!taken) break;
                o = (o + 1) % n_old;
            }
            off[l] = o;
            st->hd_idx[i * kh + l] = (int32_t)o;
        }
        sort_hd_list(st, i);
        for (int r = 0; r < rounds; ++r) {
            for (int a = 0; a < kh; ++a) {
                list[a] = st->hd_idx[i * kh + a];
                ld2[a] = st->hd_d2[i * kh + a];
            }
            for (int s = 0; s < CAND_HD; ++s) {
                uint32_t w[4];
                draw4(st->seed, st->t, (uint32_t)i, STREAM_INSERT, (uint32_t)(64 + 32 * r + s), w);
                int64_t c;
                if (s < INSERT_SLOTS_NN) {
                    int64_t a = list[map_index(w[0], kh)];
                    c = st->hd_idx[a * kh + map_index(w[1], kh)];
                } else {
                    c = map_index(w[0], n_old);
                }
                cand[s] = c;
                cd2[s] = sqdist(st->X + i * D, st->X + c * D, D);
            }
            oracle_topk_merge(i, kh, list, ld2, CAND_HD, cand, cd2, nl, nd2);
            for (int a = 0; a < kh; ++a) {
                st->hd_idx[i * kh + a] = nl[a];
                st->hd_d2[i * kh + a] = nd2[a];
            }
        }
        oracle_bisect(st->hd_d2 + i * kh, kh, st->perplexity, 0.0, bisect_tol, bisect_maxit,
                      st->beta + i, st->P + i * kh);
        place_mean(st, i);
        for (int c = 0; c < st->d; ++c) st->V[i * st->d + c] = 0.0;
        int m = kl < kh ? kl : kh;
        for (int a = 0; a < m; ++a) st->ld_idx[i * kl + a] = st->hd_idx[i * kh + a];
        for (int l = m; l < kl; ++l) {
            uint32_t w[4];
            draw4(st->seed, st->t, (uint32_t)i, STREAM_INSERT, (uint32_t)(0x40000000 + l), w);
            int64_t o = map_index(w[0], n_old);
            for (;;) {
                if (!contains(st->ld_idx + i * kl, l, o)) break;
                o = (o + 1) % n_old;
            }
            st->ld_idx[i * kl + l] = (int32_t)o;
        }
    }
    double ratio = ((double)N * (double)(N - 1)) / ((double)n_old * (double)(n_old - 1));
    st->Zhat = st->Zhat * ratio;
    double frac = (double)(N - n_old) / (double)N;
    if (frac > st->E) st->E = frac;
    /* the new points' refinement window: the next fresh_iters iterations; a
     * window still open keeps its older points in it */
    if (st->fresh_iters > 0) {
        if (!(st->t < st->fresh_until)) st->fresh_lo = n_old;
        st->fresh_until = st->t + (uint32_t)st->fresh_iters;
    }
    free(list);
    free(ld2);
    free(nl);
    free(nd2);
    free(off);
}

/* ------------------------------------------------------------------ */
/* Learned placement: a D-H-H-d ReLU MLP trained online on the (x_i, y_i) */
/* pairs of the running embedding (an addition to the method; the paper   */
/* has no learned part). Parameters, flat: W1 (H x D) b1 (H) W2 (H x H)    */
/* b2 (H) W3 (d x H) b3 (d), row-major.                                    */
/* ------------------------------------------------------------------ */

/* Round to bfloat16, nearest-even, through binary32 (the value the device
 * rounds is a binary32). */
double oracle_bf16(double x)
{
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return x; /* inf / nan unchanged */
    u += 0x7fffu + ((u >> 16) & 1u);
    u &= 0xffff0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

static double maybe_bf16(double x, int round) { return round ? oracle_bf16(x) : x; }

/* Initial parameters: weights of layer l uniform in (-a, a), a =
 * sqrt(6 / fan_in) for the hidden layers and sqrt(3 / fan_in) for the
 * output layer; entry (r, c) from word c mod 4 of the Philox block at
 * counter (l, r, MLP_INIT, c div 4) as a (2 (w + 0.5) 2^-32 - 1), rounded
 * to binary32; biases 0. */
void oracle_mlp_init(int D, int H, int d, uint64_t seed, double *theta)
{
    int dims[3][2] = {{H, D}, {H, H}, {d, H}};
    double *p = theta;
    for (int l = 0; l < 3; ++l) {
        int rows = dims[l][0], cols = dims[l][1];
        double a = sqrt((l < 2 ? 6.0 : 3.0) / (double)cols);
        for (int r = 0; r < rows; ++r)
            for (int c = 0; c < cols; ++c) {
                uint32_t w[4];
                draw4(seed, (uint32_t)(l + 1), (uint32_t)r, 10u, (uint32_t)(c / 4), w);
                double u = ((double)w[c % 4] + 0.5) * (1.0 / 4294967296.0);
                p[r * cols + c] = (double)(float)(a * (2.0 * u - 1.0));
            }
        p += rows * cols;
        for (int r = 0; r < rows; ++r) p[r] = 0.0;
        p += rows;
    }
}

/*
 * Loss and gradient of one batch: X (B x D), targets T (B x d).
 *   H1 = r(relu(X W1^T + b1)), H2 = r(relu(H1 W2^T + b2)), O = H2 W3^T + b3,
 *   L = mean over B*d of (O - T)^2,
 *   G3 = r(2 (O - T) / (B d)), G2 = r((G3 W3) * [H2 > 0]),
 *   G1 = r((G2 W2) * [H1 > 0]),
 *   dW3 = G3^T H2, db3 = sum G3, dW2 = G2^T H1, db2 = sum G2,
 *   dW1 = G1^T X, db1 = sum G1,
 * where r() rounds to bfloat16 when `round` is set (the device's operand
 * precision) and is the identity otherwise. Weights are used as given.
 * Writes O (B x d) when non-NULL; returns L.
 */
double oracle_mlp_grad(int B, int D, int H, int d, const double *theta, const double *X, const double *T,
                       int round, double *grad, double *O_out)
{
    const double *W1 = theta, *b1 = W1 + (size_t)H * D, *W2 = b1 + H, *b2 = W2 + (size_t)H * H;
    const double *W3 = b2 + H, *b3 = W3 + (size_t)d * H;
    double *gW1 = grad, *gb1 = gW1 + (size_t)H * D, *gW2 = gb1 + H, *gb2 = gW2 + (size_t)H * H;
    double *gW3 = gb2 + H, *gb3 = gW3 + (size_t)d * H;
    size_t np = (size_t)H * D + H + (size_t)H * H + H + (size_t)d * H + d;
    memset(grad, 0, sizeof(double) * np);
    double *H1 = (double *)malloc(sizeof(double) * (size_t)H);
    double *H2 = (double *)malloc(sizeof(double) * (size_t)H);
    double *G2 = (double *)malloc(sizeof(double) * (size_t)H);
    double *G1 = (double *)malloc(sizeof(double) * (size_t)H);
    double *G3 = (double *)malloc(sizeof(double) * (size_t)d);
    double loss = 0.0;
    for (int b = 0; b < B; ++b) {
        const double *x = X + (size_t)b * D;
        for (int h = 0; h < H; ++h) {
            double z = b1[h];
            for (int f = 0; f < D; ++f) z += W1[(size_t)h * D + f] * x[f];
            H1[h] = maybe_bf16(z > 0.0 ? z : 0.0, round);
        }
        for (int h = 0; h < H; ++h) {
            double z = b2[h];
            for (int g = 0; g < H; ++g) z += W2[(size_t)h * H + g] * H1[g];
            H2[h] = maybe_bf16(z > 0.0 ? z : 0.0, round);
        }
        for (int c = 0; c < d; ++c) {
            double o = b3[c];
            for (int g = 0; g < H; ++g) o += W3[(size_t)c * H + g] * H2[g];
            if (O_out) O_out[(size_t)b * d + c] = o;
            double e = o - T[(size_t)b * d + c];
            loss += e * e;
            G3[c] = maybe_bf16(2.0 * e / ((double)B * d), round);
        }
        for (int c = 0; c < d; ++c) {
            for (int g = 0; g < H; ++g) gW3[(size_t)c * H + g] += G3[c] * H2[g];
            gb3[c] += G3[c];
        }
        for (int g = 0; g < H; ++g) {
            double s = 0.0;
            for (int c = 0; c < d; ++c) s += G3[c] * W3[(size_t)c * H + g];
            G2[g] = maybe_bf16(H2[g] > 0.0 ? s : 0.0, round);
        }
        for (int h = 0; h < H; ++h) {
            for (int g = 0; g < H; ++g) gW2[(size_t)h * H + g] += G2[h] * H1[g];
            gb2[h] += G2[h];
        }
        for (int g = 0; g < H; ++g) {
            double s = 0.0;
            for (int h = 0; h < H; ++h) s += G2[h] * W2[(size_t)h * H + g];
            G1[g] = maybe_bf16(H1[g] > 0.0 ? s : 0.0, round);
        }
        for (int h = 0; h < H; ++h) {
            for (int f = 0; f < D; ++f) gW1[(size_t)h * D + f] += G1[h] * x[f];
            gb1[h] += G1[h];
        }
    }
    free(H1);
    free(H2);
    free(G2);
    free(G1);
    free(G3);
    return loss / ((double)B * d);
}

/*
 * Magnitudes of the batch gradient and outputs of oracle_mlp_grad (rounded
 * network): the same forward and backward passes with every weight, bias,
 * input, target and intermediate replaced by its absolute value, gated by
 * the ReLU pattern of the actual pass:
 *   A1 = |b1| + |W1| |x|, A2 = |b2| + |W2| (A1 [H1 > 0]), AO = |b3| + |W3| (A2 [H2 > 0]),
 *   AG3 = 2 (AO + |T|) / (B d), AG2 = (AG3 |W3|) [H2 > 0], AG1 = (AG2 |W2|) [H1 > 0],
 *   M(dW3) = sum_b AG3 A2^T, M(dW2) = sum_b AG2 A1^T, M(dW1) = sum_b AG1 |x|^T,
 *   M(db) = sum_b AG.
 * Every result of the network is a sum of products whose magnitudes these
 * sums bound, so a relative perturbation rho of each rounded intermediate
 * (a different summation order, or a value rounded to the neighbouring
 * bfloat16) moves a result by at most about (rounding levels) rho times its
 * magnitude. Writes gmag (size of the parameters) and Omag (B x d).
 */
void oracle_mlp_grad_mag(int B, int D, int H, int d, const double *theta, const double *X, const double *T,
                         double *gmag, double *Omag)
{
    const double *W1 = theta, *b1 = W1 + (size_t)H * D, *W2 = b1 + H, *b2 = W2 + (size_t)H * H;
    const double *W3 = b2 + H, *b3 = W3 + (size_t)d * H;
    double *mW1 = gmag, *mb1 = mW1 + (size_t)H * D, *mW2 = mb1 + H, *mb2 = mW2 + (size_t)H * H;
    double *mW3 = mb2 + H, *mb3 = mW3 + (size_t)d * H;
    size_t np = (size_t)H * D + H + (size_t)H * H + H + (size_t)d * H + d;
    memset(gmag, 0, sizeof(double) * np);
    double *H1 = (double *)malloc(sizeof(double) * (size_t)H);
    double *A1 = (double *)malloc(sizeof(double) * (size_t)H);
    double *A2 = (double *)malloc(sizeof(double) * (size_t)H);
    double *G2 = (double *)malloc(sizeof(double) * (size_t)H);
    double *G1 = (double *)malloc(sizeof(double) * (size_t)H);
    double *G3 = (double *)malloc(sizeof(double) * (size_t)d);
    char *on1 = (char *)malloc((size_t)H);
    char *on2 = (char *)malloc((size_t)H);
    for (int b = 0; b < B; ++b) {
        const double *x = X + (size_t)b * D;
        /* the actual (rounded) pass, for the gates */
        for (int h = 0; h < H; ++h) {
            double z = b1[h], a = fabs(b1[h]);
            for (int f = 0; f < D; ++f) {
                z += W1[(size_t)h * D + f] * x[f];
                a += fabs(W1[(size_t)h * D + f]) * fabs(x[f]);
            }
            on1[h] = z > 0.0;
            H1[h] = oracle_bf16(z > 0.0 ? z : 0.0);
            A1[h] = on1[h] ? a : 0.0;
        }
        for (int h = 0; h < H; ++h) {
            double z = b2[h], a = fabs(b2[h]);
            for (int g = 0; g < H; ++g) {
                z += W2[(size_t)h * H + g] * H1[g];
                a += fabs(W2[(size_t)h * H + g]) * A1[g];
            }
            on2[h] = z > 0.0;
            A2[h] = on2[h] ? a : 0.0;
        }
        for (int c = 0; c < d; ++c) {
            double a = fabs(b3[c]);
            for (int g = 0; g < H; ++g) a += fabs(W3[(size_t)c * H + g]) * A2[g];
            Omag[(size_t)b * d + c] = a;
            G3[c] = 2.0 * (a + fabs(T[(size_t)b * d + c])) / ((double)B * d);
        }
        for (int c = 0; c < d; ++c) {
            for (int g = 0; g < H; ++g) mW3[(size_t)c * H + g] += G3[c] * A2[g];
            mb3[c] += G3[c];
        }
        for (int g = 0; g < H; ++g) {
            double s = 0.0;
            for (int c = 0; c < d; ++c) s += G3[c] * fabs(W3[(size_t)c * H + g]);
            G2[g] = on2[g] ? s : 0.0;
        }
        for (int h = 0; h < H; ++h) {
            for (int g = 0; g < H; ++g) mW2[(size_t)h * H + g] += G2[h] * A1[g];
            mb2[h] += G2[h];
        }
        for (int g = 0; g < H; ++g) {
            double s = 0.0;
            for (int h = 0; h < H; ++h) s += G2[h] * fabs(W2[(size_t)h * H + g]);
            G1[g] = on1[g] ? s : 0.0;
        }
        for (int h = 0; h < H; ++h) {
            for (int f = 0; f < D; ++f) mW1[(size_t)h * D + f] += G1[h] * fabs(x[f]);
            mb1[h] += G1[h];
        }
    }
    free(H1);
    free(A1);
    free(A2);
    free(G2);
    free(G1);
    free(G3);
    free(on1);
    free(on2);
}

/* Input standardisation of the placement MLP: per-feature mean and
 * population standard deviation over the N rows present when the network is
 * first used (1 where a feature is constant), summed in FP64. */
void oracle_mlp_stats(int64_t N, int D, const double *X, double *mean, double *std_out)
{
    for (int f = 0; f < D; ++f) {
        double s = 0.0, s2 = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            double v = X[i * D + f];
            s += v;
            s2 += v * v;
        }
        double m = s / (double)N, var = s2 / (double)N - m * m;
        mean[f] = m;
        std_out[f] = var > 0.0 ? sqrt(var) : 1.0;
    }
}

/* Network inputs of the rows idx[0..B): bfloat16 of (x - mean) / std. The
 * rounding to bfloat16 decides a code, so it is taken in the precision the
 * device computes the value in: mean and std as binary32, then one binary32
 * subtraction and one binary32 division, each correctly rounded. */
void oracle_mlp_inputs(int B, int D, const double *X, const int64_t *idx, const double *mean,
                       const double *std_in, double *out)
{
    for (int b = 0; b < B; ++b)
        for (int f = 0; f < D; ++f) {
            float x = (float)X[idx[b] * D + f];
            float v = (x - (float)mean[f]) / (float)std_in[f];
            out[(size_t)b * D + f] = oracle_bf16((double)v);
        }
}

/* Training targets of the rows idx[0..B): y / s with s the root mean square
 * of the B x d values (1 when they are all zero). Returns s. */
double oracle_mlp_targets(int B, int d, const double *Y, const int64_t *idx, double *out)
{
    double t = 0.0;
    for (int b = 0; b < B; ++b)
        for (int c = 0; c < d; ++c) t += Y[idx[b] * d + c] * Y[idx[b] * d + c];
    double ms = t / ((double)B * d);
    double sc = ms > 0.0 ? sqrt(ms) : 1.0;
    for (int b = 0; b < B; ++b)
        for (int c = 0; c < d; ++c) out[(size_t)b * d + c] = Y[idx[b] * d + c] / sc;
    return sc;
}

/* Forward pass only (placement): O = MLP(X) with the same roundings. */
void oracle_mlp_forward(int B, int D, int H, int d, const double *theta, const double *X, int round, double *O)
{
    double *T = (double *)calloc((size_t)B * d, sizeof(double));
    size_t np = (size_t)H * D + H + (size_t)H * H + H + (size_t)d * H + d;
    double *g = (double *)malloc(sizeof(double) * np);
    oracle_mlp_grad(B, D, H, d, theta, X, T, round, g, O);
    free(T);
    free(g);
}

/* Adam (Kingma & Ba 2015) with bias correction, step number `step` >= 1:
 * m = b1 m + (1 - b1) g; v = b2 v + (1 - b2) g^2;
 * theta -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps). */
void oracle_adam(int64_t n, double *theta, const double *g, double *m, double *v, int step, double lr,
                 double b1, double b2, double eps)
{
    double c1 = 1.0 - pow(b1, step), c2 = 1.0 - pow(b2, step);
    for (int64_t e = 0; e < n; ++e) {
        m[e] = b1 * m[e] + (1.0 - b1) * g[e];
        v[e] = b2 * v[e] + (1.0 - b2) * g[e] * g[e];
        theta[e] -= lr * (m[e] / c1) / (sqrt(v[e] / c2) + eps);
    }
}

/*
 * Forces of selected points only (same definitions as oracle_forces), for
 * checking a large state on a sample: A and R rows of pts[0..n) in A_out,
 * R_out (n x d). The reverse attraction of point i sums over every j with i
 * in N_HD(j), found by one scan of all lists.
 */
void oracle_forces_points(const oracle_state *st, uint32_t t, uint32_t neg_stream, double zhat,
                          const int64_t *pts, int64_t n, double *A_out, double *R_out)
{
    int64_t N = st->N;
    int d = st->d, kh = st->k_hd, kl = st->k_ld;
    double alpha = st->alpha;
    memset(A_out, 0, sizeof(double) * (size_t)(n * d));
    memset(R_out, 0, sizeof(double) * (size_t)(n * d));
    /* position of each sampled point in the output (or -1) */
    int64_t *slot = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    for (int64_t i = 0; i < N; ++i) slot[i] = -1;
    for (int64_t a = 0; a < n; ++a) slot[pts[a]] = a;
    /* attraction: out-edges of sampled points and in-edges from every point */
    for (int64_t j = 0; j < N; ++j) {
        for (int e = 0; e < kh; ++e) {
            int64_t i = st->hd_idx[j * kh + e];
            int64_t sj = slot[j], si = slot[i];
            if (sj < 0 && si < 0) continue;
            const double *yj = st->Y + j * d, *yi = st->Y + i * d;
            double r2 = sqdist(yj, yi, d);
            double coef = 4.0 * (st->P[j * kh + e] / (2.0 * (double)N)) * kernel_w_inv_alpha(r2, alpha);
            for (int c = 0; c < d; ++c) {
                double f = coef * (yj[c] - yi[c]); /* force of pair (j, i) on j */
                if (sj >= 0) A_out[sj * d + c] += f;
                if (si >= 0) A_out[si * d + c] -= f;
            }
        }
    }
    int32_t *S = (int32_t *)malloc(sizeof(int32_t) * (size_t)(kh + kl));
    for (int64_t a = 0; a < n; ++a) {
        int64_t i = pts[a];
        const double *yi = st->Y + i * d;
        int ns = 0;
        for (int e = 0; e < kh; ++e) S[ns++] = st->hd_idx[i * kh + e];
        for (int e = 0; e < kl; ++e) {
            int32_t j = st->ld_idx[i * kl + e];
            if (!contains(st->hd_idx + i * kh, kh, j)) S[ns++] = j;
        }
        for (int e = 0; e < ns; ++e) {
            const double *yj = st->Y + (int64_t)S[e] * d;
            double r2 = sqdist(yi, yj, d);
            double coef = 4.0 * (kernel_w(r2, alpha) / zhat) * kernel_w_inv_alpha(r2, alpha);
            for (int c = 0; c < d; ++c) R_out[a * d + c] += coef * (yi[c] - yj[c]);
        }
        double scale = (double)(N - 1) / (double)st->n_neg;
        for (int s = 0; s < st->n_neg; ++s) {
            uint32_t w4[4];
            draw4(st->seed, t, (uint32_t)i, neg_stream, (uint32_t)(s % 32), w4);
            int64_t j = map_other(negative_word(w4[1], w4[3], (uint32_t)(s / 32)), N, i);
            if (contains(S, ns, j)) continue;
            const double *yj = st->Y + j * d;
            double r2 = sqdist(yi, yj, d);
            double coef = scale * 4.0 * (kernel_w(r2, alpha) / zhat) * kernel_w_inv_alpha(r2, alpha);
            for (int c = 0; c < d; ++c) R_out[a * d + c] += coef * (yi[c] - yj[c]);
        }
    }
    free(S);
    free(slot);
}


/*
 * Recalibrate every point from its current HD list: list distances
 * recomputed from X, the list reordered by (d2, idx), beta and P from a cold
 * start at the state's perplexity (Eq. 1). Follows a change of perplexity or
 * of rows of X (drift); the lists themselves are kept.
 */
void oracle_recalibrate(oracle_state *st, double bisect_tol, int bisect_maxit)
{
    int kh = st->k_hd;
    for (int64_t i = 0; i < st->N; ++i) {
        sort_hd_list(st, i);
        oracle_bisect(st->hd_d2 + i * kh, kh, st->perplexity, 0.0, bisect_tol, bisect_maxit,
                      st->beta + i, st->P + i * kh);
    }
}

/* Replace the entries -1 of list row `row` (k entries, point n of N): slot e
 * draws j = map_other(w0, N, n) from counter (t, n, REMOVE, salt + e) and
 * steps to j + 1 (mod N, skipping n) while j is already in the row. */
static void fill_removed(oracle_state *st, int32_t *row, int k, int64_t n, int64_t N, uint32_t salt)
{
    for (int e = 0; e < k; ++e) {
        if (row[e] >= 0) continue;
        uint32_t w[4];
        draw4(st->seed, st->t, (uint32_t)n, STREAM_REMOVE, salt + (uint32_t)e, w);
        int64_t j = map_other(w[0], N, n);
        for (;;) {
            int taken = 0;
            for (int a = 0; a < k; ++a)
                if (row[a] == j) taken = 1;
            if (!taken) break;
            j = (j + 1) % N;
            if (j == n) j = (j + 1) % N;
        }
        row[e] = (int32_t)j;
    }
}

/*
 * Remove the points flagged in `removed` (N entries). The state's X must
 * already hold the kept rows, compacted in their original order; every
 * other array is compacted here in place, and st->N becomes the kept count
 * N'. Kept point o gets index n = its rank among the kept points. In every
 * kept point's HD and LD list, entries that point to a kept point are
 * renumbered, entries that pointed to a removed point are replaced by
 * fill_removed (HD slots salt 0, LD slots salt 1024). Then HD distances,
 * order, beta and P are recomputed for every point (oracle_recalibrate), A
 * and V of kept points are kept, Zhat is scaled by the ratio of ordered pair
 * counts and E = max(E, n_removed / N). Returns N'.
 */
int64_t oracle_remove(oracle_state *st, const uint8_t *removed, double bisect_tol, int bisect_maxit)
{
    int64_t N = st->N, Nk = 0;
    int d = st->d, kh = st->k_hd, kl = st->k_ld;
    int64_t *map = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    for (int64_t o = 0; o < N; ++o) map[o] = removed[o] ? -1 : Nk++;
    for (int64_t o = 0; o < N; ++o) {
        int64_t n = map[o];
        if (n < 0) continue;
        for (int c = 0; c < d; ++c) {
            st->Y[n * d + c] = st->Y[o * d + c];
            st->V[n * d + c] = st->V[o * d + c];
        }
        st->beta[n] = st->beta[o];
        for (int e = 0; e < kh; ++e) {
            int32_t j = st->hd_idx[o * kh + e];
            st->hd_idx[n * kh + e] = (int32_t)map[j];
        }
        for (int e = 0; e < kl; ++e) {
            int32_t j = st->ld_idx[o * kl + e];
            st->ld_idx[n * kl + e] = (int32_t)map[j];
        }
    }
    for (int64_t n = 0; n < Nk; ++n) {
        fill_removed(st, st->hd_idx + n * kh, kh, n, Nk, 0u);
        fill_removed(st, st->ld_idx + n * kl, kl, n, Nk, 1024u);
    }
    double nr = (double)(N - Nk);
    st->Zhat *= ((double)Nk * (double)(Nk - 1)) / ((double)N * (double)(N - 1));
    if (nr / (double)N > st->E) st->E = nr / (double)N;
    st->N = Nk;
    /* renumbering closes the refinement window of recent insertions */
    st->fresh_lo = Nk;
    st->fresh_until = st->t;
    oracle_recalibrate(st, bisect_tol, bisect_maxit);
    free(map);
    return Nk;
}


/*
 * Shrink (or grow) the embedding: Y and V scaled by `factor` (the paper's
 * "implosion", which makes gradients significant again after the layout has
 * spread), then Zhat re-estimated at the new Y with negatives from counter
 * (t, i, ZINIT, s), as for the first estimate.
 */
void oracle_scale(oracle_state *st, double factor)
{
    int64_t n = st->N * st->d;
    for (int64_t e = 0; e < n; ++e) {
        st->Y[e] *= factor;
        st->V[e] *= factor;
    }
    double *A = (double *)malloc(sizeof(double) * (size_t)n);
    double *R = (double *)malloc(sizeof(double) * (size_t)n);
    st->Zhat = oracle_forces(st, st->t, STREAM_ZINIT, 1.0, A, R, NULL);
    free(A);
    free(R);
}
