/*
 * recon.h -- C ABI of librecon, the GB300 (sm_103a) hot path of subquadratic
 * network reconstruction (T. P. Peixoto, "Scalable network reconstruction in
 * subquadratic time", arXiv:2401.01404).
 *
 * The library reconstructs a sparse symmetric coupling matrix W from samples
 * X by maximising a pseudo-likelihood with a Laplace (L1) prior (App. A),
 * using greedy coordinate descent (Algorithm 2): each iteration finds the
 * m = round(kappa*N) pairs (i,j) whose single-coupling update gains the most
 * (FindBest, Algorithm 3, over an NNDescent k-nearest-neighbour search,
 * Algorithm 4) and updates only those.
 *
 * Conventions shared by every call:
 *  - Pairs are 0-based int32 node ids, stored as consecutive (i, j) entries.
 *    Outputs are canonical (i < j).  Inputs may be in either order.
 *  - d(i,j) is returned as -gain, where gain = max_w pi(W_ij <- w) - pi(W)
 *    >= 0 is the objective increase of the best update of that coupling.  The
 *    paper's d(i,j) = -max_w pi(W) (Algorithm 2) differs from it by the
 *    constant pi(W), so both rank pairs identically; the constant (about
 *    N*M*log 2 in magnitude) would leave no float resolution for the ranking.
 *  - All work is ordered on the CUDA stream given to recon_init.  A call that
 *    returns host outputs has synchronised that stream; a call with device
 *    outputs only has enqueued its work and returns without waiting, except
 *    where stated.  Calls on one context must not overlap in host threads.
 *  - A pointer flagged *_is_device != 0 is a device pointer on the context's
 *    device; otherwise it is an ordinary host pointer.
 *  - Every call returns a recon_status; nothing is thrown across the ABI.  On
 *    failure, recon_last_error() describes the cause.  RECON_ECUDA and
 *    RECON_ETIMEOUT leave the context unusable (RECON_ESTATE afterwards)
 *    until it is destroyed.  There is no CPU fallback: without a usable GPU,
 *    recon_init fails.
 */
#ifndef RECON_H
#define RECON_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct recon_ctx recon_ctx; /* opaque, owned by the library */

typedef enum {
    RECON_OK = 0,
    RECON_EINVAL = 1,       /* invalid argument; the message names it */
    RECON_ENOMEM = 2,       /* device or host allocation failed */
    RECON_ECUDA = 3,        /* a CUDA call failed */
    RECON_ETIMEOUT = 4,     /* a bounded device-side wait ran out */
    RECON_ESTATE = 5,       /* the context was left unusable by an earlier error */
    RECON_EUNSUPPORTED = 6  /* the option combination is not supported */
} recon_status;

typedef enum { RECON_ISING = 0, RECON_GAUSSIAN = 1 } recon_model;

typedef enum {
    RECON_X_INT8 = 0, /* Ising spins, every value -1 or +1 */
    RECON_X_FP32 = 1  /* Gaussian samples, finite floats */
} recon_xtype;

typedef enum {
    RECON_KNN_NNDESCENT = 0,  /* FindKNN by NNDescent (Algorithm 4) at every level */
    RECON_KNN_EXHAUSTIVE = 1, /* FindKNN by scoring every pair of the level's node set */
    RECON_KNN_AUTO = 2,       /* exhaustive where it costs fewer pair evaluations */
    RECON_KNN_SCREEN = 3      /* Algorithm 3's exhaustive base case over all nodes, computed
                                 exactly: the tensor-core gradient screen (App. B's gradient
                                 as distance) keeps every pair that can have a nonzero gain,
                                 and only those, plus the stored couplings, are scored */
} recon_knn_mode;

typedef enum {
    RECON_SEED_RANDOM = 0, /* random k-out initial lists (Algorithm 4) */
    RECON_SEED_SCREEN = 1, /* lists seeded from the dense tensor-core gradient screen */
    RECON_SEED_LEARNED = 2 /* lists seeded from the learned sketch embedding */
} recon_seed_mode;

/* The distance the search ranks pairs by (App. B, "Gradient as distance").
 *   GAIN      d(i,j) = -(max_w pi(W_ij <- w) - pi(W)), the exact gain of Algorithm 2.
 *   GRADIENT  d(i,j) = -|d log pi / d W_ij| at the current W: the smooth part's
 *             derivative D at W_ij, and D - lambda sign(W_ij) for a stored coupling
 *             (a central difference of the penalty at W_ij = 0 is zero).  One pass
 *             over the samples, no 1-D solve; recon_score returns it (w_out = the
 *             current coupling), and the coordinate updates still solve each pair
 *             exactly.  Not with RECON_KNN_SCREEN (whose survivors are the pairs with
 *             |D| > lambda only): recon_init returns RECON_EUNSUPPORTED. */
typedef enum { RECON_DIST_GAIN = 0, RECON_DIST_GRADIENT = 1 } recon_distance;

typedef struct {
    double lambda;        /* Laplace prior penalty (App. A), >= 0 */
    uint64_t seed;        /* seed of every random choice of the search */
    double eps_knn;       /* NNDescent stops when Delta/(k|S|) < eps_knn (Algorithm 4) */
    int32_t max_knn_iters;/* NNDescent iteration cap; 0 means 2*ceil(log_{2k}|S|)+2 */
    float w_clamp;        /* couplings are kept within |W_ij| <= w_clamp (0: model default) */
    float h_clamp;        /* Ising fields are kept within |h_i| <= h_clamp */
    int32_t knn_mode;     /* recon_knn_mode */
    int32_t seed_mode;    /* recon_seed_mode, for the first FindBest level */
    int32_t screen_c;     /* per-node candidates kept by the screen / learned seeding */
    int32_t timing;       /* nonzero: time every pair-scoring launch with CUDA events
                             on the context's stream (see recon_stats.score_ms) */
    int32_t no_graphs;    /* nonzero: enqueue NNDescent iterations launch by launch instead of
                             replaying one captured CUDA graph per iteration */
    float learned_frac;   /* RECON_SEED_LEARNED: share of each initial list taken from the
                             proposal's best seeds, in (0, 1]; the rest are random ids
                             (0 selects the default 0.5) */
    int32_t distance;     /* recon_distance: the d(i, j) that the search ranks pairs by */
    int32_t screen_fp8;   /* nonzero (Ising only): the tensor-core screen reads E4M3 operands,
                             twice the bf16 rate; its margin (each node's actual rounding
                             error of its residuals, plus an accumulation allowance) widens
                             with the coarser rounding, so the result is still exact, with
                             more survivors to score.
                             RECON_GAUSSIAN: recon_init returns RECON_EUNSUPPORTED */
    int32_t screen_no_rank1; /* nonzero: at the empty network (no stored coupling, where every
                             sample of a node has the same field) the screen still uses the
                             general form above; by default it computes the spin product
                             X X^T in E4M3 (exact, K = M) plus a rank-two correction */
    /* A split search: with shard_count > 1 this context's screen covers only shard
     * shard_index of its work items (every shard_count-th 128 x 256 half of a 256 x 256
     * super-tile of the pair matrix; with screen_pair, every shard_count-th super-tile),
     * so that shard_count processes (one GPU each) share one search.  Each
     * returns the m best pairs of its shard (stored couplings included), and
     * recon_select_best over the union of the shards' results gives the unsharded
     * answer exactly.  Only with RECON_KNN_SCREEN (else RECON_EUNSUPPORTED);
     * recon_gcd_step refuses a sharded context (merge before updating); 0 or 1:
     * no sharding. */
    int32_t shard_index;
    int32_t shard_count;
    int32_t screen_pair;  /* nonzero: the screen runs in the CTA-pair form (tcgen05
                             cta_group::2; clusters of two CTAs, one M = 256 MMA per
                             256 x 256 super-tile, each SM holding half of each operand
                             tile) instead of the default one CTA per 128 x 256 unit.
                             Both give the same survivors; the pair form moves a third
                             less operand data but measures 5-7 % slower, its
                             accumulator handoff crossing the two SMs. */
} recon_options;

typedef struct {
    int64_t pair_evals;       /* pairs scored since init (each counts once per score) */
    int64_t newton_passes;    /* sample passes beyond the first, summed over pairs */
    int64_t knn_iters;        /* NNDescent iterations run by the last recon_best_pairs */
    int32_t levels;           /* FindBest KNN levels of the last recon_best_pairs */
    int32_t level_k[16];      /* k used at each level */
    int64_t level_size[17];   /* |S_t| at each level (the last one is exhaustive) */
    int64_t nnz;              /* stored couplings (including ones set back to zero) */
    int64_t samples;          /* M */
    int64_t kernel_launches;  /* kernels this context has launched */
    int64_t score_launches;   /* pair-scoring launches timed (options.timing) */
    int64_t score_pairs;      /* pairs those launches scored */
    double score_ms;          /* their summed device time, from CUDA events */
    int64_t screen_launches;  /* tensor-core screen launches timed (options.timing) */
    double screen_ms;         /* their summed device time */
    double screen_flop;       /* their algorithmic work: 2 x (128 x 128 tiles) x K per launch */
    int64_t screen_survivors; /* pairs the screen passed on, summed */
    int64_t seeded_nodes;     /* nodes whose first list held learned seeds (last call) */
    int64_t tuned_threads;    /* block width the autotuner picked for the segmented scorer (0: not yet) */
    int64_t dropped_offers;   /* NNDescent second neighbours past the per-node cap, and offers past
                                 a full offer buffer, skipped for an iteration */
    int64_t screen_rank1;     /* screen launches in the rank-one form of the empty network */
    int64_t device_bytes;     /* device memory this context has requested since init (every
                                 allocation counted; frees are not subtracted) */
    int64_t nnd_graph_loops;  /* NNDescent runs whose iterations went to the GPU as one graph
                                 launch (a conditional WHILE node with the stopping test on the
                                 device) rather than one launch and one host test per iteration
                                 (options.timing, which times each iteration, uses the latter) */
} recon_stats;

/* Fills *opt with the defaults: lambda = 0 (set it), seed = 1,
 * eps_knn = 1e-3, max_knn_iters = 0, w_clamp = 0 (the model's default: 5 for
 * the Ising model, whose float solver supports |W_ij| <= 8; no clamp for the
 * Gaussian model), h_clamp = 10, knn_mode = RECON_KNN_NNDESCENT,
 * seed_mode = RECON_SEED_RANDOM, screen_c = 0, timing = 0. */
void recon_default_options(recon_options *opt);

/* recon_init -- Sec. II's reconstruction problem for data X and the model's
 * pseudo-likelihood (App. A), starting from the empty network W = 0 (Sec. II).
 *   X        : M x N samples, sample-major: X[m*N + i] is node i in sample m.
 *              int8 spins (-1/+1) for RECON_ISING, float for RECON_GAUSSIAN.
 *              Read during the call only; the caller keeps ownership and may
 *              free it when the call returns.
 *   x_is_device: X is a device pointer (else host).
 *   opt      : may be NULL for the defaults; copied.
 *   stream   : a cudaStream_t (NULL = the legacy default stream).
 * The library copies X into its own node-major device layout, fits the
 * per-node parameters at W = 0 (Ising fields h_i = atanh(mean x_i) clamped to
 * h_clamp; Gaussian theta_i^2 = mean x_i^2) and the per-sample fields.
 * Errors: RECON_EINVAL for N < 2, M < 1, lambda < 0 or not finite, a spin
 * not in {-1,+1}, a non-finite sample, an unknown model or type;
 * RECON_ENOMEM; RECON_ECUDA (also when no CUDA device is usable).  On error
 * *out is NULL. Synchronous. */
recon_status recon_init(recon_ctx **out, const void *X, int64_t M, int64_t N, int32_t x_type,
                        int32_t x_is_device, int32_t model, const recon_options *opt, void *stream);

/* recon_objective -- log pi(W, theta) up to its constant: the log
 * pseudo-likelihood summed over samples and nodes plus the Laplace log-prior
 * -lambda sum_{i<j} |W_ij| (App. A).  Per-term float, double accumulation.
 * Synchronous. */
recon_status recon_objective(recon_ctx *ctx, double *out);

/* recon_score -- d(i,j) = -gain for P pairs at the current (W, theta)
 * (Algorithm 2's distance; each gain is the exact optimum of the
 * single-coupling problem under the L1 prior, solved to float precision).
 *   pairs : P x 2 int32; i != j, both in [0, N).
 *   d_out : P floats.  w_out: P floats (the maximising W_ij), may be NULL.
 *   io_is_device: pairs, d_out and w_out are all device pointers (else all host).
 * Errors: RECON_EINVAL for a bad id or P < 0.  P = 0 is a no-op. */
recon_status recon_score(recon_ctx *ctx, const int32_t *pairs, int64_t P, float *d_out, float *w_out,
                         int32_t io_is_device);

/* recon_best_pairs -- FindBest(m, {0..N-1}, d) of Algorithm 3 with
 * m = round(kappa*N) (half up), over FindKNN by NNDescent (Algorithm 4) or
 * exhaustive scoring (opt.knn_mode).  At each level k_t = max(k,
 * ceil(4m/|S_t|)) (at most |S_t|-1); the recursion ends with an exhaustive
 * search once |S_t|^2 <= 4m.
 *   pairs : cap x 2 int32, written with min(m, found) canonical pairs in
 *           ascending d (ties by (i, j)).  d: cap floats (may be NULL).
 *   *m_out: the number written; when cap < m it is set to m and nothing is
 *           written (RECON_EINVAL).
 * Errors besides RECON_EINVAL: RECON_ENOMEM (a search buffer or the device),
 * RECON_ETIMEOUT when a bounded wait of the pair scorer (its staged row
 * copies) or of the tensor-core screen ran out.
 * Synchronous. */
recon_status recon_best_pairs(recon_ctx *ctx, int32_t k, double kappa, int32_t *pairs, float *d,
                              int64_t cap, int64_t *m_out, int32_t out_is_device);

/* recon_select_best -- the m best of P scored pairs, unique and ordered by
 * (d, i, j): the last step of Algorithm 3 (the best m of the pairs its levels
 * collected), here the merge of the shards of a split search (see
 * recon_options.shard_count).  Duplicate pairs must carry the same d (as the
 * same pair scored at the same state does) and are kept once.
 *   pairs : P x 2 int32, i != j, both in [0, N) (either order); d: P floats.
 *   out_pairs : cap x 2 int32 (canonical i < j), out_d: cap floats (may be NULL);
 *   *count_out = min(m, unique pairs); when cap < that, nothing is written and
 *   RECON_EINVAL is returned.  io_is_device: all four arrays on the device (else
 *   host).  Synchronous. */
recon_status recon_select_best(recon_ctx *ctx, const int32_t *pairs, const float *d, int64_t P, int64_t m,
                               int32_t *out_pairs, float *out_d, int64_t cap, int64_t *count_out,
                               int32_t io_is_device);

/* recon_score_noalloc -- recon_score for host pair lists that performs no
 * device allocation (the paper has no counterpart: this is a deployment
 * variant).  Meant for callers that may not allocate device memory while they
 * run: a process sharing the GPU with PyTorch or JAX, whose caching allocators
 * hold most of the memory, or a serving loop that forbids allocation after
 * start-up.  recon_score stages host pairs and results in buffers it grows with
 * cudaMalloc/cudaFree (and cudaFree waits for the whole device); this call
 * stages them in one array of 1 MiB that the library reserves statically in
 * device memory on every GPU that loads it, for the life of the process.
 *   pairs : P x 2 int32 host array; d_out (and w_out, may be NULL): P floats on
 *           the host.  Same values as recon_score on the same pairs.
 *   P     : at most 65536 per call; larger P returns RECON_EINVAL (split the
 *           list into several calls).
 * The first call on a device looks up the array's device address (once per
 * device); make that first call before any stream capture.  All calls share
 * the array and it keeps the last call's contents; each call clears the words
 * it needs zeroed.  Calls that overlap on the GPU (several host threads or
 * streams) race on the array.  Synchronous. */
recon_status recon_score_noalloc(recon_ctx *ctx, const int32_t *pairs, int64_t P, float *d_out, float *w_out);

/* recon_set_list_lengths -- per-node list lengths for the first FindBest level
 * (Algorithm 3 uses one k for all nodes; a per-node k_i in [1, 64] lets the
 * search spend its effort unevenly, and the level then uses max(k_i, ceil(4m/N))
 * for node i, which keeps the level's guarantees).  n = N lengths (host), or
 * n = 0 to return to the uniform k of recon_best_pairs.  Takes effect with
 * RECON_KNN_NNDESCENT (and AUTO, which then searches by NNDescent). */
recon_status recon_set_list_lengths(recon_ctx *ctx, const int32_t *k, int64_t n);

/* recon_knn_graph -- the k-NN graph that the first level of the last FindBest
 * search built (Algorithm 3, first level; Algorithm 4's lists at the end of the
 * search): row i holds the best list of node i, ascending in d(i, j) = -gain
 * (ties in the search's internal order), k_i entries then padding (id -1,
 * d +inf).  Host buffers ids and d (either may be NULL) of cap >= N k entries,
 * row-major [N x k], node ids global.  *k_out = the row stride k (max k_i),
 * *n_out = N; both 0 when the last search built no lists (the screen, a level
 * small enough for the exhaustive base case, or no search yet).  ids = d = NULL
 * queries the sizes.  EINVAL if cap < N k. Synchronous. */
recon_status recon_knn_graph(recon_ctx *ctx, int32_t *ids, float *d, int64_t cap, int32_t *k_out, int64_t *n_out);

/* recon_row_best -- every pair {i, j} with i in rows, j != i and d(i, j) < d_cut,
 * scored exactly at the current state (as recon_score) against all N columns of
 * each row: Algorithm 3's exhaustive scoring restricted to a node subset, the
 * ground truth of a subsample (rows on the host, duplicates allowed, each in
 * [0, N)).  The pairs are canonical (i < j), unique, in ascending (d, i, j);
 * the first min(count, cap) are written to the host buffers pairs [cap x 2] and
 * d [cap] (d may be NULL); *count_out = the number found.  Costs N scores per
 * row.  EINVAL on a bad row, a NaN cut, or cap > 0 with pairs NULL. Synchronous. */
recon_status recon_row_best(recon_ctx *ctx, const int32_t *rows, int64_t nrows, float d_cut, int32_t *pairs, float *d,
                            int64_t cap, int64_t *count_out);

/* recon_exhaustive_best -- the m best pairs over all N(N-1)/2 pairs, exact
 * (Algorithm 3's exhaustive base case applied to the whole node set); the
 * ground truth that recall is measured against.  Arguments as in
 * recon_best_pairs, with m given directly. Synchronous. */
recon_status recon_exhaustive_best(recon_ctx *ctx, int64_t m, int32_t *pairs, float *d, int64_t cap,
                                   int64_t *m_out, int32_t out_is_device);

/* recon_cd_sweep -- the update loop of Algorithm 2: each pair's coupling is
 * set to its maximiser in turn, in the given order, with the per-sample fields
 * of both endpoints refreshed (App. A's tracked sums).  Pairs that share no
 * node are updated concurrently (App. B); the result equals the sequential
 * loop in the given order.  Duplicate pairs are allowed and are applied twice.
 *   pairs_is_device: pairs is a device pointer (else host).
 *   delta_out: sum |W_ij' - W_ij| (may be NULL).  Synchronous. */
recon_status recon_cd_sweep(recon_ctx *ctx, const int32_t *pairs, int64_t P, int32_t pairs_is_device,
                            double *delta_out);

/* recon_field_sweep -- optimises every per-node parameter theta_i (Ising
 * field h_i; Gaussian theta_i^2 = 1/W_ii) at fixed couplings, the update that
 * App. A performs alongside W.  delta_out: sum |theta_i' - theta_i| (may be
 * NULL). Synchronous. */
recon_status recon_field_sweep(recon_ctx *ctx, double *delta_out);

/* recon_gcd_step -- one iteration of Algorithm 2: recon_best_pairs(k, kappa),
 * recon_cd_sweep over them in ascending d, then recon_field_sweep.
 * delta_out: Delta of the iteration (couplings + per-node parameters);
 * objective_out: the objective afterwards; m_out: pairs updated.  Any of the
 * three may be NULL. Synchronous. */
recon_status recon_gcd_step(recon_ctx *ctx, int32_t k, double kappa, double *delta_out,
                            double *objective_out, int64_t *m_out);

/* ---- learned proposal (Ising) --------------------------------------------
 * The paper starts NNDescent from random k-out lists (Algorithm 4) and relies
 * on that randomness to reach every pair eventually (Sec. III).  The learned
 * proposal only changes where the first FindBest level's lists start: each
 * node's sketch s_i = Omega^T x_i / sqrt(M) (Omega: 64 random +-1 columns) goes
 * through an MLP 64 -> 128 (ReLU) -> 32 into an embedding e_i, and the pairs
 * with the largest |<e_i, e_j>| seed the lists; every seed is scored exactly
 * before it can stay.  Random seeding is the default and the fallback (an
 * untrained context seeds at random even with RECON_SEED_LEARNED). */

typedef struct {
    int32_t steps;          /* full-batch Adam steps (Kingma and Ba, 2015) */
    float lr;               /* learning rate */
    uint64_t seed;          /* initial weights (on the first use) and the sketch */
    int64_t n_pairs;        /* > 0: train on these host pairs ... */
    const int32_t *pairs;   /* ... n_pairs x 2 */
    const float *targets;   /* their targets; NULL: tau = sign(w*) sqrt(2 gain) from
                               the exact scorer, so that tau^2 / 2 is the gain */
    int64_t n_best;         /* n_pairs == 0: train on the n_best exact best pairs (tensor-core
                               screen, default N) ... */
    int64_t n_random;       /* ... and n_random uniform random pairs (default 8N) */
    int32_t fixed_sketch;   /* nonzero: train on the context's own sketches; by default Omega
                               is drawn afresh at every step, so that the network learns a
                               function of sketch similarity that carries to other data,
                               rather than the nodes of its training data */
    int32_t reserved[7];
} recon_train_opts;

/* Parameters: W1 [128 x 64] | b1 [128] | W2 [32 x 128] | b2 [32], row-major, FP32
 * (the forward pass uses their BF16 rounding with FP32 accumulation). */
int64_t recon_proposal_param_count(void);
void recon_default_train_opts(recon_train_opts *opts);

/* recon_proposal_train -- trains the proposal on exact pair scores of this
 * context's data (loss mean (<e_i,e_j> - tau_ij)^2).  loss_out: steps floats
 * (host), the loss before each step, may be NULL.  Synchronous. */
recon_status recon_proposal_train(recon_ctx *ctx, const recon_train_opts *opts, float *loss_out);

/* recon_proposal_weights -- copies the parameters out (get_out) and/or in
 * (set_in, which also restarts Adam and makes the proposal usable for seeding);
 * host arrays of recon_proposal_param_count() floats.  Weights trained on one
 * context can be set into another (for example a smaller run's). Synchronous. */
recon_status recon_proposal_weights(recon_ctx *ctx, float *get_out, const float *set_in, int64_t count);

/* recon_proposal_embed -- sketches (N x 64) and embeddings (N x 32) of every
 * node under the current weights; host arrays, either may be NULL. */
recon_status recon_proposal_embed(recon_ctx *ctx, float *sketch_out, float *embed_out);

/* recon_proposal_grad -- loss and its gradient (recon_proposal_param_count()
 * floats, host) for the given host pairs and targets, without a step. */
recon_status recon_proposal_grad(recon_ctx *ctx, const int32_t *pairs, const float *targets, int64_t P,
                                 float *grad_out, double *loss_out);

/* recon_get_model -- the current couplings and per-node parameters.
 *   ij: cap x 2 int32, w: cap floats; receive the stored couplings (i < j),
 *   including ones that an update set back to zero; *nnz gets their count
 *   (when cap < count nothing is written and RECON_EINVAL is returned).
 *   fields: N floats (Ising h_i; Gaussian theta_i^2), may be NULL.
 * Host pointers. Synchronous. */
recon_status recon_get_model(recon_ctx *ctx, int32_t *ij, float *w, int64_t cap, int64_t *nnz,
                             float *fields);

/* recon_set_model -- replaces the state: couplings W (nnz entries, i != j,
 * each unordered pair at most once) and per-node parameters (N floats, may be
 * NULL to keep them), then recomputes the per-sample fields from scratch.
 * Host pointers. Synchronous. */
recon_status recon_set_model(recon_ctx *ctx, const int32_t *ij, const float *w, int64_t nnz,
                             const float *fields);

/* recon_get_stats -- counters (see recon_stats). Host pointer. */
recon_status recon_get_stats(recon_ctx *ctx, recon_stats *out);

/* recon_save / recon_load -- checkpoint of the whole state (options, samples,
 * couplings, per-node parameters, counters) in a versioned binary file;
 * recon_load rebuilds the per-sample fields, so a loaded context continues
 * exactly as the saved one would. */
recon_status recon_save(recon_ctx *ctx, const char *path);
recon_status recon_load(recon_ctx **out, const char *path, void *stream);

/* ---- device ceilings ------------------------------------------------------
 * The paper has no counterpart: these are the arithmetic and on-chip bandwidth
 * ceilings that the kernels' rooflines are stated against, measured on the
 * device by short fixed-work kernels timed with CUDA events (eight independent
 * dependency chains per thread, 8 CTAs of 256 threads per SM). */
typedef struct {
    int32_t sm_count;        /* streaming multiprocessors */
    double sm_clock_mhz;     /* the device's reported maximum SM clock */
    int64_t l2_bytes;        /* L2 cache size */
    double fp32_tflops;      /* FP32 fused multiply-add, 2 flops each */
    double fp64_tflops;      /* FP64 fused multiply-add, 2 flops each */
    double mufu_rcp_gops;    /* rcp.approx.ftz.f32 per second (10^9; with one FP32 add each) */
    double mufu_ex2_gops;    /* ex2.approx.ftz.f32 per second */
    double mufu_lg2_gops;    /* lg2.approx.ftz.f32 per second (with one FP32 add each) */
    double mufu_tanh_gops;   /* tanh.approx.f32 per second */
    double l2_read_gbs;      /* 16-byte loads from an L2-resident buffer into the SMs, GB/s */
    double l2_buffer_bytes;  /* size of that buffer (a quarter of L2) */
} recon_peaks;

/* recon_device_peaks -- measures the ceilings above on CUDA device `device`
 * (which becomes the calling thread's current device).  Allocates a quarter of
 * the L2 size of device memory for the call and frees it; changes no device
 * setting.  Takes a few milliseconds.  RECON_ECUDA if a CUDA call fails;
 * RECON_EINVAL for out == NULL.  Synchronous. */
recon_status recon_device_peaks(int32_t device, recon_peaks *out);

/* recon_last_error -- message of the last failed call on ctx (or of the last
 * failed recon_init / recon_load in this thread when ctx is NULL). */
const char *recon_last_error(const recon_ctx *ctx);

/* recon_destroy -- frees every resource of ctx; NULL is a no-op. */
void recon_destroy(recon_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* RECON_H */
