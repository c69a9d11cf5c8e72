/*
 * funcsne.h -- C ABI of the GB300 (sm_103a) FUnc-SNE iteration.
 *
 * FUnc-SNE (Lambert, Couplet, Verleysen, Lee, arXiv 2509.07681) embeds N
 * high-dimensional (HD) points x_i in R^D into a low-dimensional (LD) space
 * R^d by gradient descent on the variable-tail t-SNE objective (Eq. 4-5)
 * while it refines, at every iteration, approximate HD and LD neighbour sets
 * from neighbours of neighbours, cross-space proposals and random points
 * (Section 3). This library runs one such iteration per step on one GPU.
 *
 * Conventions for every entry point:
 *   - Return value: FUNCSNE_OK (0) or a negative FUNCSNE_E_* code. No C++
 *     exception crosses the ABI. funcsne_last_error() gives a message.
 *   - Array arguments are plain pointers to row-major data; each entry
 *     point accepts host memory or device memory of the current device,
 *     detected with cudaPointerGetAttributes. Data passed in is copied;
 *     the caller keeps ownership of every buffer it passes.
 *   - Work is enqueued on the handle's CUDA stream (funcsne_set_stream);
 *     calls that write caller buffers synchronise that stream first. That
 *     stream does not wait for other streams: device inputs written on
 *     another stream must be complete (or that stream passed to
 *     funcsne_set_stream) before the call.
 *   - Point indices are int32 (N < 2^31).
 */
#ifndef FUNCSNE_H
#define FUNCSNE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    FUNCSNE_OK = 0,
    FUNCSNE_E_ARG = -1,   /* invalid argument (size, range, NULL pointer)        */
    FUNCSNE_E_OOM = -2,   /* device allocation failed                            */
    FUNCSNE_E_CUDA = -3,  /* a CUDA runtime call failed                          */
    FUNCSNE_E_NAN = -4,   /* non-finite input data or embedding                   */
    FUNCSNE_E_RANGE = -5, /* a device-side index check failed                     */
    FUNCSNE_E_STATE = -6  /* call not valid in the handle's current state         */
};

/* HD storage precision (option "precision"). Distances are always
 * accumulated in FP32; reduced-precision rows are dequantised first, and
 * candidates that may enter a neighbour set are re-ranked from the FP32
 * master rows, so neighbour sets equal those of FUNCSNE_FP32. */
enum { FUNCSNE_FP32 = 0, FUNCSNE_BF16 = 1, FUNCSNE_FP8 = 2 };

/* Neighbour spaces for funcsne_get_knn. */
enum { FUNCSNE_SPACE_HD = 0, FUNCSNE_SPACE_LD = 1 };

/* Placement of inserted points (funcsne_insert). */
enum { FUNCSNE_PLACE_MEAN = 0, FUNCSNE_PLACE_SURROGATE = 1 };

typedef struct funcsne funcsne_t;

/* Snapshot of the per-point state, for testing and checkpointing. Every
 * pointer may be NULL (field skipped) and may be host or device memory. */
typedef struct {
    float *Y;        /* N x d embedding                                        */
    float *V;        /* N x d momentum                                          */
    int32_t *hd_idx; /* N x k_hd HD neighbour indices, ordered by (d2, index)   */
    float *hd_d2;    /* N x k_hd squared HD distances (FP32, exact rows)         */
    int32_t *ld_idx; /* N x k_ld LD neighbour indices                           */
    float *beta;     /* N bandwidths beta_i = 1 / (2 sigma_i^2)  (Eq. 1)         */
    float *P;        /* N x k_hd conditional affinities p_{j|i}, aligned with hd_idx */
    double Zhat;     /* running estimate of sum_{k != l} w_kl (Eq. 4)           */
    double E;        /* smoothed fraction of points with new HD neighbours       */
    uint32_t t;      /* iteration counter                                        */
    int64_t fresh_lo;     /* insertion window (option "fresh_iters"): points     */
    uint32_t fresh_until; /* fresh_lo .. N-1 refine while t < fresh_until;      */
                          /* fresh_lo = N (and any fresh_until) means none      */
} funcsne_state_t;

typedef struct {
    int64_t N;
    uint32_t t;
    double E;              /* E[N_new / N] after the last step (Section 3)        */
    double Zhat;           /* normalisation estimate used by the next step         */
    double last_Z;         /* Z_t estimated by the last step                        */
    int64_t last_n_new;    /* points whose HD set changed in the last step          */
    int32_t last_coin;     /* 1 if the last step refined the HD sets               */
    int32_t precision;     /* FUNCSNE_FP32 / _BF16 / _FP8                           */
    uint32_t error_word;   /* device error bits (0 = none)                          */
    int64_t cand_scored;   /* HD candidates scored (cumulative)                      */
    int64_t cand_reranked; /* of which re-ranked from FP32 rows (cumulative)         */
    int64_t mlp_steps;     /* training steps of the placement MLP                    */
    double mlp_loss;       /* its loss on the last training batch                    */
    int64_t n_refined;     /* steps that refined the HD sets (cumulative)           */
} funcsne_stats_t;

/* One training step of the placement MLP with its intermediate values, for
 * testing. Each pointer may be NULL (skipped) and may be host or device
 * memory. B = option "mlp_batch", H = "mlp_hidden", n_params =
 * H D + H + H H + H + d H + d (layout W1 b1 W2 b2 W3 b3, row-major). */
typedef struct {
    int32_t *batch_idx;   /* B point indices of the batch                       */
    float *xhat;          /* B x D normalised inputs (bfloat16 values)           */
    float *target;        /* B x d scaled targets y / s                          */
    float *output;        /* B x d network outputs                               */
    float *theta_before;  /* n_params FP32 parameters before the step            */
    float *weights_bf16;  /* n_params bfloat16 copy the step used (as float)     */
    float *grad;          /* n_params gradient                                    */
    float *theta_after;   /* n_params FP32 parameters after the Adam update       */
    double loss;          /* mean squared error of the batch                      */
    float scale;          /* s = RMS of the batch's y                             */
    int32_t step;         /* Adam step number of this step (1 = first)            */
    int64_t n_params;
} funcsne_mlp_debug_t;

/*
 * funcsne_create -- allocate a handle and initialise the method's state
 * (Section 3: optimisation starts right after the initial allocations).
 *   X          N x D row-major FP32 data (host or device), copied.
 *   N, D       number of points (k_hd < N, k_ld < N) and HD dimension (D >= 1).
 *   d          LD dimension, 1 <= d <= 32 (Section 3: arbitrary LD dimension).
 *   k_hd       HD neighbours per point, 2 <= k_hd <= 64.
 *   k_ld       LD neighbours per point, 1 <= k_ld <= 32.
 *   n_neg      negative samples per point and step, 1 <= n_neg <= 1024.
 *   alpha      tail parameter of Eq. 4 (alpha > 0; 1 = t-SNE).
 *   perplexity target perplexity of Eq. 1, 1 < perplexity < k_hd + 1.
 *   seed       key of every Philox4x32-10 stream the method draws.
 *   out        receives the handle (owned by the caller; funcsne_destroy).
 * Initial state: k distinct random HD and LD neighbours per point, Y0 = a
 * random linear projection of the centred data scaled to std 1e-4 per LD
 * dimension, V = 0, bandwidths calibrated from a cold start, E = 1,
 * Zhat = the estimate of Z at Y0.
 * Errors: FUNCSNE_E_ARG (sizes, ranges, NULL), FUNCSNE_E_NAN (non-finite X),
 * FUNCSNE_E_OOM, FUNCSNE_E_CUDA. On error *out is NULL.
 */
int funcsne_create(const float *X, int64_t N, int32_t D, int32_t d, int32_t k_hd,
                   int32_t k_ld, int32_t n_neg, float alpha, float perplexity, uint64_t seed,
                   funcsne_t **out);

/*
 * funcsne_set_option / funcsne_get_option -- numeric options by name:
 *   "lr"             learning rate (default max(N/12, 200))
 *   "momentum"       momentum of the update (default 0.8)
 *   "att_ratio"      scale of the attractive force (Section 3; default 1)
 *   "rep_ratio"      scale of the repulsive force (Section 3; default 1)
 *   "exaggeration"   extra attraction factor while t < "exag_iters" (default 1)
 *   "exag_iters"     iterations with exaggeration (default 0)
 *   "hd_mode"        0: refine the HD sets with probability 0.05 + 0.95 E
 *                    (Section 3); 1: every iteration; 2: never
 *   "coin_floor"     p0 of the refinement probability p0 + (1 - p0) E in
 *                    [0, 1] (default 0.05, the paper's value)
 *   "gamma_e"        smoothing rate in (0, 1] of E, the running fraction of
 *                    points that found new HD neighbours:
 *                    E <- (1 - gamma_e) E + gamma_e N_new / N after each
 *                    refinement (default 0.1; the paper gives none)
 *   "gamma_z"        smoothing rate in (0, 1] of the normalisation estimate:
 *                    Zhat <- (1 - gamma_z) Zhat + gamma_z Z_t (default 0.1)
 *   "precision"      FUNCSNE_FP32 / FUNCSNE_BF16 / FUNCSNE_FP8 HD storage
 *   "alpha"          tail parameter (may change between steps)
 *   "perplexity"     target perplexity in (1, k_hd + 1); a change recomputes
 *                    every HD list's distances and order and recalibrates
 *                    every beta and P from a cold start (Eq. 1)
 *   "concurrent"     1: the HD and LD refinements (which only read the state
 *                    of the iteration) run side by side (default 0)
 *   "forces_cw"      floats of an LD row each lane reads in the forces
 *                    kernel: 4, 8 (default) or 16 (a tuning knob; used when
 *                    "forces_pair" is 0 or rows are narrower than 8 floats)
 *   "forces_pair"    1 (default): LD rows of 8 floats (d = 5 ... 8) are
 *                    read by two lanes with one 16-byte load each, two rows
 *                    per lane and pass; 0 (and every other row width): the
 *                    "forces_cw" split
 *   "ld_pair"        1 (default): the LD refinement reads rows of 8 or more
 *                    floats the same way; 0: two lanes per row
 *   "hd_prefetch"    1 (default): the HD refinement loads the next point's
 *                    lists and copies its own row into a second shared-memory
 *                    buffer while the current point is scored, where two
 *                    lanes read a gathered row (rows up to 224 bytes) and the
 *                    two buffers leave room for four blocks per SM
 *                    (read-only "hd_prefetch_used" tells); 0: off
 *   "jump_iters"     jump start (Section 3): during the first jump_iters
 *                    iterations no gradient is applied; instead, at the start
 *                    of each of "jump_parts" (default 2) equal parts, Y is
 *                    replaced by a random linear projection of the data
 *                    (Philox counter (part + 1, f, 8, c), std 1e-4 per
 *                    dimension) while both neighbour sets keep refining
 *                    (default 0: off)
 *   "insert_rounds"  neighbour-of-neighbour rounds that build an inserted
 *                    point's HD list (0..256, default 64)
 *   "fresh_iters"    iterations after an insertion during which the inserted
 *                    points refine their HD lists in every iteration, also
 *                    when the coin does not fire (an addition for points
 *                    added on the fly; E is updated only by the coin's
 *                    iterations). An insertion inside an open window extends
 *                    it and keeps the earlier points in it; a removal closes
 *                    it. 0 (default): off
 *   "hd_lanes"       lanes that read one gathered HD row in the refinement:
 *                    1, 2, 4 or 8, or 0 (default) to choose from the row
 *                    bytes. A tuning knob; it fixes the FP32 summation order,
 *                    so results depend on it (bit for bit). Read-only
 *                    "hd_lanes_used" gives the lanes in use
 *   "surrogate"      1: train the placement MLP inside funcsne_step, one
 *                    step before every "mlp_every"-th iteration (default 0)
 *   "mlp_every"      iterations between training steps (default 10)
 *   "mlp_lr"         Adam learning rate (default 1e-3)
 *   "mlp_batch"      training batch size B (default 4096; before first use)
 *   "mlp_hidden"     hidden width H (default 256; before first use)
 * Unknown keys or out-of-range values: FUNCSNE_E_ARG.
 */
int funcsne_set_option(funcsne_t *h, const char *key, double value);
int funcsne_get_option(const funcsne_t *h, const char *key, double *value);

/* Use the given cudaStream_t (NULL = the handle's own stream) for all work. */
int funcsne_set_stream(funcsne_t *h, void *stream);

/*
 * funcsne_step -- enqueue n_iters iterations (Section 3 / Eq. 5-6):
 *   1. with probability 0.05 + 0.95 E (or always / never, option hd_mode),
 *      refine every HD set from 32 candidates (neighbours of HD neighbours,
 *      LD neighbours and their neighbours, random points) by a top-k_hd
 *      merge on (d2, index); flag points whose set changed and recalibrate
 *      their bandwidth by bisection from the previous value;
 *   2. refine every LD set from 32 candidates (neighbours of LD neighbours,
 *      HD neighbours, random points) at the current embedding;
 *   3. attraction over the HD sets (both directions of p_ij), repulsion over
 *      the HD and LD sets plus n_neg Philox negatives, normalised by Zhat;
 *   4. momentum update of Y; Zhat and E smoothed; t += 1.
 * Asynchronous on the handle's stream. Errors surface at funcsne_sync.
 */
int funcsne_step(funcsne_t *h, int32_t n_iters);

/* Wait for the handle's stream; report device error words (FUNCSNE_E_RANGE,
 * FUNCSNE_E_NAN) and CUDA errors. */
int funcsne_sync(funcsne_t *h);

/*
 * funcsne_insert -- append n_new points (Section 3: the algorithm admits new
 * points without a pre-computation phase). X_new is n_new x D FP32 (host or
 * device), copied. Each new point gets k_hd HD neighbours from random
 * candidates refined by "insert_rounds" (default 64) neighbour-of-neighbour
 * rounds against the existing points, its LD position by `placement`
 * (FUNCSNE_PLACE_MEAN: mean of its HD neighbours' positions;
 * FUNCSNE_PLACE_SURROGATE: the online MLP,
 * falling back to the mean while the MLP is untrained), and LD neighbours
 * seeded from its HD neighbours. *first_id receives the index of the first
 * new point (ids are contiguous). Errors: FUNCSNE_E_ARG, FUNCSNE_E_OOM.
 */
int funcsne_insert(funcsne_t *h, const float *X_new, int64_t n_new, int32_t placement,
                   int64_t *first_id);

/*
 * funcsne_update_points -- replace the HD rows of n existing points (drift;
 * Section 3 lets the data change while the method runs). ids: n distinct
 * point ids in [0, N) (host or device int64); X_rows: n x D FP32 (host or
 * device), copied. Every point's HD list then has its distances recomputed,
 * is reordered by (d2, idx), and its beta and P are recalibrated from a cold
 * start (Eq. 1); the lists themselves, Y and V are kept, and later
 * iterations refine the neighbourhoods. Errors: FUNCSNE_E_ARG (ids out of
 * range or repeated), FUNCSNE_E_NAN (non-finite rows: nothing changes),
 * FUNCSNE_E_OOM, FUNCSNE_E_CUDA.
 */
int funcsne_update_points(funcsne_t *h, const int64_t *ids, int64_t n, const float *X_rows);

/*
 * funcsne_remove -- remove n points (Section 3: points may leave while the
 * method runs). ids: n distinct ids in [0, N) (host or device int64). The
 * kept points keep their order and are renumbered 0 .. N - n - 1. In every
 * HD and LD list, entries that pointed to a removed point are replaced, in
 * slot order, by j = a uniform other point from Philox counter
 * (t, i, 11, salt + slot) (salt 0 for HD, 1024 for LD), stepped to j + 1
 * while already listed; then every HD list is re-scored, reordered and
 * recalibrated as in funcsne_update_points. Zhat is scaled by the ratio of
 * ordered pair counts and E becomes max(E, n / N). Capacity is kept.
 * Errors: FUNCSNE_E_ARG (ids out of range or repeated, or fewer than
 * max(k_hd, k_ld) + 1 points would remain), FUNCSNE_E_OOM, FUNCSNE_E_CUDA.
 */
int funcsne_remove(funcsne_t *h, const int64_t *ids, int64_t n);

/*
 * Placement MLP (an addition to the method; the paper has no learned part):
 * a D-H-H-d ReLU network with bfloat16 weights and FP32 accumulation,
 * trained by Adam (lr "mlp_lr", beta 0.9 / 0.999, eps 1e-8) to map the
 * normalised x_i of B points drawn by Philox to y_i / s (s = RMS of the
 * batch's y). Inputs are normalised by the per-feature mean and standard
 * deviation of the points present at its first use. It places points
 * inserted with FUNCSNE_PLACE_SURROGATE at s MLP(x).
 * funcsne_mlp_train runs n_steps training steps now; funcsne_mlp_predict
 * writes s MLP(x) for the n rows of X (n x D, host or device) into Y_out
 * (n x d); funcsne_mlp_debug_step runs one step and exports its values.
 */
int funcsne_mlp_train(funcsne_t *h, int32_t n_steps);
int funcsne_mlp_predict(const funcsne_t *h, const float *X, int64_t n, float *Y_out);
int funcsne_mlp_debug_step(funcsne_t *h, funcsne_mlp_debug_t *out);

/* Copy the first min(N, cap_rows) rows of the N x d embedding into Y_out. */
int funcsne_get_embedding(const funcsne_t *h, float *Y_out, int64_t cap_rows);

/*
 * funcsne_get_embedding_async -- read the embedding out without waiting, for
 * a viewer that shows each iteration while the next ones run (Section 3:
 * the method suits interactive visualisation). The embedding as left by the
 * steps queued so far is snapshotted on the device (stream-ordered on the
 * handle's stream), then copied to the first min(N, cap_rows) x d entries
 * of Y_out on an internal stream, so steps queued afterwards run during the
 * copy. Y_out (host or device) must stay valid and unread until
 * funcsne_wait_embedding or funcsne_sync returns; with pageable host memory
 * the call itself waits for the copy (pinned memory overlaps). One snapshot
 * buffer: a second call waits on the device for the first copy to finish
 * before it overwrites the snapshot. Errors: FUNCSNE_E_ARG, FUNCSNE_E_OOM,
 * FUNCSNE_E_CUDA.
 */
int funcsne_get_embedding_async(funcsne_t *h, float *Y_out, int64_t cap_rows);

/* Wait until the copy of the last funcsne_get_embedding_async has landed. */
int funcsne_wait_embedding(funcsne_t *h);

/*
 * funcsne_scale_embedding -- multiply Y and V by factor (> 0), then
 * re-estimate Zhat at the scaled embedding (negatives from Philox counter
 * (t, i, 9, s)). Section 3's "implosion": a layout that keeps spreading makes
 * the gradients small, and shrinking it makes them significant again.
 * Errors: FUNCSNE_E_ARG, FUNCSNE_E_OOM, FUNCSNE_E_CUDA.
 */
int funcsne_scale_embedding(funcsne_t *h, float factor);

/* Copy the first min(N, cap_rows) rows of the N x D HD data (FP32, as held
 * after insertions, drift and removals) into X_out (host or device). With
 * funcsne_export_state this is a complete checkpoint of the iteration. */
int funcsne_get_data(const funcsne_t *h, float *X_out, int64_t cap_rows);

/* Copy the current neighbour lists of `space` (FUNCSNE_SPACE_HD: N x k_hd,
 * FUNCSNE_SPACE_LD: N x k_ld) into idx and, when d2 is non-NULL, their
 * squared distances (LD distances at the current embedding). */
int funcsne_get_knn(const funcsne_t *h, int32_t space, int32_t *idx, float *d2);

int funcsne_get_stats(const funcsne_t *h, funcsne_stats_t *stats);

/* Snapshot / restore the per-point state (see funcsne_state_t). On import,
 * HD distances are recomputed from X and each HD list (with its P row) is
 * ordered by (d2, index); hd_d2 is ignored. Lists must hold distinct
 * indices other than the point itself (FUNCSNE_E_ARG otherwise). */
int funcsne_export_state(const funcsne_t *h, funcsne_state_t *st);
int funcsne_import_state(funcsne_t *h, const funcsne_state_t *st);

/* Run one iteration like funcsne_step and also copy the forces of step 3
 * before the update: att (N x d) = sum over HD pairs of
 * 4 p_ij w^{1/alpha} (y_i - y_j), rep (N x d) = the estimated
 * 4 sum_j q_ij w^{1/alpha} (y_i - y_j), so that dL/dy = att - rep (Eq. 5). */
int funcsne_debug_step(funcsne_t *h, float *att, float *rep);

/* Run n_iters iterations like funcsne_step but with direct kernel launches
 * and CUDA events between the kernels on the handle's stream; waits for
 * the stream and writes into ms_per_kernel[0..3] the summed device time
 * (milliseconds) of the HD refinement, LD refinement, forces and update
 * kernels. For measurement. */
int funcsne_profile_step(funcsne_t *h, int32_t n_iters, double *ms_per_kernel);

/* Exercise the bounded device wait on the handle's stream: a kernel polls
 * an mbarrier that nothing arrives on, gives up after `polls` polls
 * (1 .. 2^24) and sets the device error bit that the tensor-core kernels
 * set when a wait runs out. The next funcsne_sync then returns
 * FUNCSNE_E_CUDA ("a device wait timed out") and so do later ones on this
 * handle; the CUDA context stays usable. For testing failure detection.
 * Errors: FUNCSNE_E_ARG. */
int funcsne_debug_bounded_wait(funcsne_t *h, uint32_t polls);

/* Copy into E_out (host or device, min(cap_rows, N) floats) each row's
 * stored bound E_i >= ||x_i - x~_i|| on the error of its BF16 or FP8 copy
 * x~_i, the bound the distance band of the reduced-precision HD refinement
 * uses (E^2 summed from upward-rounded FP32 squares of the element errors,
 * then an upward-rounded square root). For testing.
 * Errors: FUNCSNE_E_ARG (NULL), FUNCSNE_E_STATE (FP32 rows: no copy). */
int funcsne_debug_row_bounds(const funcsne_t *h, float *E_out, int64_t cap_rows);

/* Allocation-failure injection, for testing failure detection on the host:
 * after `after` more successful device allocations of the library (any
 * handle), the next one fails as if the device were out of memory, once;
 * the call that made it returns FUNCSNE_E_OOM and releases what it had
 * allocated. after < 0 switches the injection off. Process-wide, not
 * thread-safe against concurrent calls. Always returns FUNCSNE_OK. */
int funcsne_debug_fail_alloc(int64_t after);

/* Exact k nearest HD neighbours (FP32 distances, ties by index) of the n_q
 * query points `queries` (int32, host or device), by brute force over all
 * points: for measuring neighbour recall. idx: n_q x k, d2: n_q x k or NULL. */
int funcsne_exact_knn(const funcsne_t *h, const int32_t *queries, int64_t n_q, int32_t k,
                      int32_t *idx, float *d2);

/*
 * funcsne_exact_knn_noalloc -- the brute-force exact KNN of funcsne_exact_knn
 * for callers that cannot allocate device memory at the time of the call
 * (for example code running under another framework's caching allocator,
 * or a latency-critical path that must not incur the implicit
 * synchronisation of cudaMalloc). The paper has no counterpart; this is a
 * deployment convenience of this library. It allocates nothing: the
 * kernels' scratch (query indices and partial top-k lists) lives in a 4 MiB
 * file-scope device array that every GPU loading the library keeps until
 * the process exits. No handle is needed.
 *   X        device pointer, N rows of D FP32 features with row pitch ldx
 *            floats (ldx % 4 == 0, ldx >= D rounded up to 4, ldx <= 4096),
 *            16-byte aligned; columns D .. ceil(D/4)*4 - 1 must be zero.
 *   queries  HOST array of n_q point indices in [0, N). They are checked
 *            on the host before return, then copied to the device with
 *            cudaMemcpyAsync on `stream`: from pageable memory the copy has
 *            finished when the call returns; from page-locked (pinned)
 *            memory it runs when the stream reaches it, so such a buffer
 *            must stay unchanged until then.
 *   k        neighbours per query, 1 <= k <= min(64, N - 1).
 *   idx, d2  DEVICE outputs, n_q x k int32 and FP32 (d2 may be NULL); ordered
 *            by (d2, index), the query point itself excluded.
 *   stream   cudaStream_t to run on (NULL = legacy default stream); the
 *            call is asynchronous on it.
 * Limits: the scratch holds n_q x (4 + 256 x ceil(k/32)) bytes plus
 * alignment, so n_q is at most about 16,000 for k <= 32 and about 8,000 for
 * k <= 64; larger n_q returns FUNCSNE_E_ARG (split the queries).
 * The first call on each device looks up the array's device address with
 * that device current; make that first call before any stream capture.
 * All calls share the array: calls that overlap on the GPU (other streams
 * or other host threads) race on it and must be serialised by the caller.
 * Errors: FUNCSNE_E_ARG (message via funcsne_last_error(NULL)),
 * FUNCSNE_E_CUDA.
 */
int funcsne_exact_knn_noalloc(const float *X, int64_t N, int32_t D, int32_t ldx,
                              const int32_t *queries, int64_t n_q, int32_t k, int32_t *idx,
                              float *d2, void *stream);

/* Message for the last error on this handle (or the last create failure
 * when h is NULL). Valid until the next call on the handle. */
const char *funcsne_last_error(const funcsne_t *h);

/* Release the handle and its device memory (NULL-safe). */
void funcsne_destroy(funcsne_t *h);

#ifdef __cplusplus
}
#endif

#endif /* FUNCSNE_H */
