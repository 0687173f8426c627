// common.cuh -- internal declarations of librecon (not part of the ABI).
//
// Device layout (node-major, sized for HBM residency):
//   Ising:    xbits  uint32 [N x Mw]  bit l of word c is sample 32c+l; 1 <=> x = -1
//             phi    float  [N x Mp]  per-sample local field h_i + sum_j W_ij x_j
//             t      float  [N x Mp]  tanh(phi); padding samples hold t = 1
//             h, H   float  [N]       fields; H_i = sum_m (1 - t_i^2)
//             T      float  [N]       sum of t_i over the Mp samples (padding t = 1)
//   Gaussian: xg     float  [N x Mp]  samples (padding 0)
//             e      float  [N x Mp]  residual x + s2 * mu
//             mu     float  [N x Mp]  neighbour sums sum_j W_ij x_j
//             s2, Q  float  [N]       theta_i^2 = 1/W_ii; Q_i = sum_m x_i^2
//   W: open-addressing hash table of the stored couplings, key (i << 32 | j), i < j.
// Mp = M rounded up to a multiple of 32; Mw = Mp / 32.  Padding samples
// (m >= M) have x = +1 and t = 1 for the Ising model, which makes every
// per-sample term of the pair problem vanish exactly; kernels that touch phi
// mask them instead.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <string>
#include <vector>

#include "recon.h"

#define RECON_EMPTY_KEY 0xFFFFFFFFFFFFFFFFull

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------

// SplitMix64 finaliser (Steele, Lea and Flood, OOPSLA 2014): counter-based
// stream for the random choices of the search, and the hash of the tables.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__host__ __device__ __forceinline__ uint64_t pair_key(int a, int b) {
    uint32_t lo = (uint32_t)(a < b ? a : b), hi = (uint32_t)(a < b ? b : a);
    return ((uint64_t)lo << 32) | hi;
}

// Order-preserving map float -> uint32 (ascending floats -> ascending ints).
__host__ __device__ __forceinline__ uint32_t float_key(float f) {
    uint32_t u;
#ifdef __CUDA_ARCH__
    u = __float_as_uint(f);
#else
    memcpy(&u, &f, 4);
#endif
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Hardware reciprocal (rcp.approx, about 1 ulp).
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ---------------------------------------------------------------------------
// coupling table
// ---------------------------------------------------------------------------
struct WTable {
    unsigned long long *keys;  // RECON_EMPTY_KEY when free
    float *vals;
    uint64_t mask;             // capacity - 1 (capacity a power of two)
};

__device__ __forceinline__ float wt_lookup(const WTable &T, uint64_t key) {
    uint64_t s = mix64(key) & T.mask;
    for (uint64_t probe = 0; probe <= T.mask; ++probe) {
        unsigned long long k = T.keys[s];
        if (k == key) return T.vals[s];
        if (k == RECON_EMPTY_KEY) return 0.f;
        s = (s + 1) & T.mask;
    }
    return 0.f;
}

__device__ __forceinline__ bool wt_contains(const WTable &T, uint64_t key) {
    uint64_t s = mix64(key) & T.mask;
    for (uint64_t probe = 0; probe <= T.mask; ++probe) {
        unsigned long long k = T.keys[s];
        if (k == key) return true;
        if (k == RECON_EMPTY_KEY) return false;
        s = (s + 1) & T.mask;
    }
    return false;
}

// Inserts or overwrites; returns false when the table is full.
__device__ __forceinline__ bool wt_upsert(const WTable &T, uint64_t key, float v) {
    uint64_t s = mix64(key) & T.mask;
    for (uint64_t probe = 0; probe <= T.mask; ++probe) {
        unsigned long long k = T.keys[s];
        if (k == key) { T.vals[s] = v; return true; }
        if (k == RECON_EMPTY_KEY) {
            unsigned long long prev = atomicCAS(&T.keys[s], RECON_EMPTY_KEY, (unsigned long long)key);
            if (prev == RECON_EMPTY_KEY || prev == key) { T.vals[s] = v; return true; }
        }
        s = (s + 1) & T.mask;
    }
    return false;
}

// Set insertion; returns 1 if the key was new, 0 if present, -1 if full.
__device__ __forceinline__ int set_insert(unsigned long long *keys, uint64_t mask, uint64_t key) {
    uint64_t s = mix64(key) & mask;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
        unsigned long long k = keys[s];
        if (k == key) return 0;
        if (k == RECON_EMPTY_KEY) {
            unsigned long long prev = atomicCAS(&keys[s], RECON_EMPTY_KEY, (unsigned long long)key);
            if (prev == RECON_EMPTY_KEY) return 1;
            if (prev == key) return 0;
        }
        s = (s + 1) & mask;
    }
    return -1;
}
__device__ __forceinline__ bool set_contains(const unsigned long long *keys, uint64_t mask, uint64_t key) {
    uint64_t s = mix64(key) & mask;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
        unsigned long long k = keys[s];
        if (k == key) return true;
        if (k == RECON_EMPTY_KEY) return false;
        s = (s + 1) & mask;
    }
    return false;
}

// ---------------------------------------------------------------------------
// device-resident counters
// ---------------------------------------------------------------------------
enum {
    CNT_PAIR_EVALS = 0,
    CNT_NEWTON = 1,
    CNT_ERR = 2,       // bit flags, see ERR_*
    CNT_SCRATCH0 = 3,  // per-call scratch counters
    CNT_SCRATCH1 = 4,
    CNT_SCRATCH2 = 5,
    CNT_SCRATCH3 = 6,
    CNT_N = 16
};
enum { ERR_BAD_SPIN = 1, ERR_TABLE_FULL = 2, ERR_BAD_VALUE = 4, ERR_OVERFLOW = 8, ERR_TIMEOUT = 16 };

// ---------------------------------------------------------------------------
// model views passed to kernels
// ---------------------------------------------------------------------------
// shared-memory barriers and bulk copies (the tensor-core screen and the
// staged pair scorer)
__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *b, uint32_t par) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(par)
        : "memory");
    return ok != 0;
}
// one contiguous global -> shared copy (16-byte aligned ends), its bytes
// counted on the mbarrier
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     su32(dst)),
                 "l"(src), "r"(bytes), "r"(su32(bar))
                 : "memory");
}

struct IsingView {
    const uint32_t *xbits;
    float *phi, *t, *h, *H;
    // T_i = sum of t over all Mp samples (padding included, t = 1 there), kept with H
    // wherever t changes; the pass at delta = 0 of the pair scorer takes sum_m t_j from it
    float *T;
    int N, M, Mp, Mw;
    // the same bits transposed per node (32 words): word l holds, at bit c, the
    // spin of sample 32 c + l (the sample lane l handles in word c)
    const uint32_t *xT;
};

struct GaussView {
    const float *xg;
    float *e, *mu, *s2, *Q;
    int N, M, Mp;
};

struct ScoreParams {
    float lambda, w_clamp, h_clamp;
    int grad_only;  // score by |d log pi / dW_ij| instead of the exact gain
    int stall;      // fault injection: the segmented scorer issues no row copies
};

// |d log pi / dW_ij| from the smooth part's derivative D at the current W_ij = W0
// (the penalty contributes lambda sign(W0); nothing at W0 = 0)
__device__ __forceinline__ float grad_dist(float D, float W0, float lambda) {
    return fabsf(W0 == 0.f ? D : D - (W0 > 0.f ? lambda : -lambda));
}

// ---------------------------------------------------------------------------
// growable device buffer
// ---------------------------------------------------------------------------
struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct SearchBufs;  // defined in search.cuh
struct Proposal;    // defined in proposal.cuh

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct recon_ctx {
    int model = 0, device = 0, num_sms = 0;
    int64_t N = 0, M = 0, Mp = 0, Mw = 0;
    recon_options opt{};
    cudaStream_t stream = nullptr;
    cudaStream_t gstream = nullptr;  // private stream of the captured NNDescent iterations

    // Ising
    uint32_t *xbits = nullptr;
    uint32_t *xbitsT = nullptr;  // N x 32 words, see IsingView::xT
    float *phi = nullptr, *t = nullptr, *h = nullptr, *H = nullptr, *T = nullptr;
    // Gaussian
    float *xg = nullptr, *e = nullptr, *mu = nullptr, *s2 = nullptr, *Q = nullptr;
    // per-node list lengths of the first FindBest level (empty: uniform k)
    std::vector<int32_t> klen_host;

    WTable W{};
    uint64_t w_cap = 0;

    unsigned long long *cnt = nullptr;  // device counters [CNT_N]
    unsigned long long *cnt_host = nullptr;  // pinned mirror

    std::vector<DBuf> bufs;  // scratch by slot
    SearchBufs *sb = nullptr;
    Proposal *prop = nullptr;  // learned proposal, created by recon_proposal_train

    recon_stats stats{};
    uint64_t stats_calls = 0;  // best-pairs calls so far (seeds each call's random choices)
    int tuned_threads = 0;     // block width of the segmented scorer, picked by the autotuner
    int64_t graph_launches_per_iter = 0;  // kernels in one captured NNDescent iteration
    // the captured NNDescent iteration, kept while everything it was captured
    // with (sizes, buffers, views, parameters) stays the same
    cudaGraphExec_t nnd_exec = nullptr;
    std::vector<uint8_t> nnd_sig;
    // all of a FindBest level's NNDescent iterations as one graph: a WHILE node
    // whose body is one iteration plus the device-side stopping test
    cudaGraphExec_t nnd_loop_exec = nullptr;
    std::vector<uint8_t> nnd_loop_sig;
    bool nnd_loop_broken = false;  // the conditional graph could not be built: iterate from the host
    cudaEvent_t nnd_ea = nullptr, nnd_eb = nullptr;  // scoring launch inside the iteration (timing)
    std::string err;
    bool broken = false;

    // per-launch CUDA events of the pair-scoring kernel (options.timing)
    struct TimedLaunch {
        cudaEvent_t a, b;
        int64_t pairs;
    };
    std::vector<TimedLaunch> timed;
    std::vector<cudaEvent_t> event_pool;

    IsingView iv() const {
        return IsingView{xbits, phi, t, h, H, T, (int)N, (int)M, (int)Mp, (int)Mw, xbitsT};
    }
    GaussView gv() const { return GaussView{xg, e, mu, s2, Q, (int)N, (int)M, (int)Mp}; }
    bool force_exact = false;  // exact gains even in gradient-distance mode (proposal targets)
    // host-side fault injection (tests): a cap on the device bytes the context
    // may request (RECON_FAULT_ALLOC_LIMIT), and a screen or a segmented scorer
    // whose loads are never issued, so that its bounded waits run out
    // (RECON_FAULT_SCREEN_STALL, RECON_FAULT_SCORE_STALL)
    uint64_t alloc_limit = 0, alloc_total = 0;
    // Newton passes counted by calls that keep their counters outside c->cnt
    // (recon_score_noalloc's static words)
    int64_t newton_extra = 0;
    bool fault_screen_stall = false, fault_score_stall = false;
    bool findbest_sorts = false;  // FindBest without its one-CTA small-level paths
    ScoreParams sp() const {
        return ScoreParams{(float)opt.lambda, opt.w_clamp, opt.h_clamp,
                           opt.distance == RECON_DIST_GRADIENT && !force_exact ? 1 : 0, fault_score_stall ? 1 : 0};
    }
};

// the context whose API call is running on this thread (for launch counting)
extern thread_local recon_ctx *tl_ctx;
// cudaMalloc under the current context's allocation cap (if one is set)
cudaError_t recon_malloc(void **p, size_t bytes);
inline void note_launch() {
    if (tl_ctx) tl_ctx->stats.kernel_launches++;
}

// scratch slots
enum {
    BUF_PAIRS = 0, BUF_GAIN, BUF_WST, BUF_BATCH, BUF_ORDER, BUF_OFF, BUF_FIRST, BUF_DELTA, BUF_TMP0,
    BUF_TMP1, BUF_TMP2, BUF_TMP3, BUF_SORT0, BUF_SORT1, BUF_SORT2, BUF_SORT3, BUF_SORT4, BUF_NSLOTS
};

// returns false on allocation failure (message set)
bool ensure_buf(recon_ctx *c, int slot, size_t bytes);
template <class T>
static inline T *buf(recon_ctx *c, int slot) {
    return (T *)c->bufs[slot].p;
}

// ---------------------------------------------------------------------------
// launchers (each returns cudaGetLastError())
// ---------------------------------------------------------------------------
// ising.cu
cudaError_t launch_ising_transpose_bits(IsingView v, uint32_t *xT, cudaStream_t s);
cudaError_t ising_score_seg_setup();
cudaError_t launch_ising_pack(const int8_t *X_sm, int64_t M, int64_t N, int Mw, uint32_t *xbits,
                              unsigned long long *cnt, cudaStream_t s);
cudaError_t launch_ising_init_fields(IsingView v, float h_clamp, cudaStream_t s);
cudaError_t launch_ising_phi_from_csr(IsingView v, const int64_t *off, const int32_t *nbr,
                                      const float *w, cudaStream_t s);
cudaError_t launch_ising_objective(IsingView v, double *partials, int nblocks, cudaStream_t s);
cudaError_t launch_ising_score(IsingView v, WTable W, ScoreParams p, const int32_t *pairs, int64_t P,
                               const int32_t *gid, float *d_out, float *w_out,
                               unsigned long long *cnt, cudaStream_t s);
cudaError_t launch_ising_score_seg(IsingView v, WTable W, ScoreParams p, const int32_t *seg_node,
                                   const int64_t *seg_start, const int32_t *seg_count, const int32_t *seg_vbase,
                                   int64_t nseg, const int32_t *cand, const int32_t *gid, float *d_out,
                                   unsigned long long *cnt, int threads, cudaStream_t s);
cudaError_t launch_ising_update(IsingView v, WTable W, ScoreParams p, const int32_t *pairs,
                                const int32_t *order, int64_t begin, int64_t end, double *delta,
                                unsigned long long *cnt, cudaStream_t s);
cudaError_t launch_ising_field_sweep(IsingView v, ScoreParams p, double *delta, cudaStream_t s);
cudaError_t launch_ising_unpack(IsingView v, int8_t *X_sm, cudaStream_t s);
int ising_max_words();

// gauss.cu
cudaError_t launch_gauss_pack(const float *X_sm, int64_t M, int64_t N, int Mp, float *xg,
                              unsigned long long *cnt, cudaStream_t s);
cudaError_t launch_gauss_init(GaussView v, cudaStream_t s);
cudaError_t launch_gauss_mu_from_csr(GaussView v, const int64_t *off, const int32_t *nbr,
                                     const float *w, cudaStream_t s);
cudaError_t launch_gauss_objective(GaussView v, double *partials, int nblocks, cudaStream_t s);
cudaError_t launch_gauss_score(GaussView v, WTable W, ScoreParams p, const int32_t *pairs, int64_t P,
                               const int32_t *gid, float *d_out, float *w_out,
                               unsigned long long *cnt, cudaStream_t s);
cudaError_t launch_gauss_score_seg(GaussView v, WTable W, ScoreParams p, const int32_t *seg_node,
                                   const int64_t *seg_start, const int32_t *seg_count, const int32_t *seg_vbase,
                                   int64_t nseg, const int32_t *cand, const int32_t *gid, float *d_out, int threads,
                                   cudaStream_t s);
cudaError_t launch_gauss_update(GaussView v, WTable W, ScoreParams p, const int32_t *pairs,
                                const int32_t *order, int64_t begin, int64_t end, double *delta,
                                unsigned long long *cnt, cudaStream_t s);
cudaError_t launch_gauss_diag_sweep(GaussView v, double *delta, cudaStream_t s);
cudaError_t launch_gauss_unpack(GaussView v, float *X_sm, cudaStream_t s);

// util.cu
cudaError_t launch_penalty(WTable W, double *out, cudaStream_t s);
cudaError_t launch_sum_doubles(const double *in, int64_t n, double *out, cudaStream_t s);
int64_t layer_tmp_elems(int64_t P);
cudaError_t launch_layer_frontier(const int32_t *pairs, int64_t P, int N, unsigned long long *keys,
                                  unsigned long long *keys_alt, uint32_t *vals, uint32_t *vals_alt, int64_t *tmp,
                                  int32_t *succ, int32_t *indeg, int32_t *fa, int32_t *fb, int *batch, int *order,
                                  int *boff, int *nb, cudaStream_t s);
cudaError_t launch_ising_update_rounds(IsingView v, WTable W, ScoreParams p, const int32_t *pairs,
                                       const int32_t *order, const int32_t *off, int b0, int b1, double *delta,
                                       unsigned long long *cnt, cudaStream_t s);
cudaError_t launch_gauss_update_rounds(GaussView v, WTable W, ScoreParams p, const int32_t *pairs,
                                       const int32_t *order, const int32_t *off, int b0, int b1, double *delta,
                                       unsigned long long *cnt, cudaStream_t s);
cudaError_t launch_fill_u64(unsigned long long *p, unsigned long long v, int64_t n, cudaStream_t s);
cudaError_t launch_fill_i32(int32_t *p, int32_t v, int64_t n, cudaStream_t s);
cudaError_t launch_table_count(WTable W, unsigned long long *out, cudaStream_t s);
cudaError_t launch_table_dump(WTable W, int32_t *ij, float *w, unsigned long long *cursor,
                              cudaStream_t s);
cudaError_t launch_table_rehash(WTable from, WTable to, cudaStream_t s);
cudaError_t launch_table_insert(WTable T, const int32_t *ij, const float *w, int64_t n, unsigned long long *cnt,
                                cudaStream_t s);
cudaError_t launch_check_pairs(const int32_t *pairs, int64_t P, int n, unsigned long long *cnt, cudaStream_t s);
// exclusive scan of n int64 counts (tmp holds >= scan_tmp_elems(n) int64)
int64_t scan_tmp_elems(int64_t n);
cudaError_t launch_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s);
// stable LSD radix sort of (key, value) by key bits [bit0, bit1); ping-pong buffers
int64_t radix_tmp_elems(int64_t n);
cudaError_t radix_sort_u64(unsigned long long *keys, uint32_t *vals, unsigned long long *keys_alt,
                           uint32_t *vals_alt, int64_t n, int bit0, int bit1, int64_t *tmp,
                           bool *result_in_alt, cudaStream_t s);

// screen.cu
// operands: bf16 rows of K = 2 Mp, or (Ising, fp8) E4M3 rows padded to a multiple of 128
int screen_k(recon_ctx *c, bool fp8);
cudaError_t launch_screen_prep(recon_ctx *c, void *A, void *B, float *l1, bool fp8);
float screen_rel_err(int model, int Mp, bool fp8);
float screen_acc_err(recon_ctx *c, bool fp8);
cudaError_t launch_screen(recon_ctx *c, const void *A, const void *B, const float *l1, int32_t *out, int64_t cap,
                          unsigned long long *count, float margin_scale, double *flop_out, bool fp8);
// general form: operands of K columns (a multiple of 64 bf16 or 128 fp8), of which the first
// k_valid are nonzero; threshold `thr` on |G_ij|, margin rel * (l_i + l_j) (or l_i l_j) + abs_margin
// when l1 is given, stored couplings skipped when skip_stored
// r1 != NULL: the rank-one form at the empty network (A = B the E4M3 spin rows, r1 the
// per-node (s_i, tau_i); keep |2 S_ij - tau_j s_i - tau_i s_j| > thr - abs_margin);
// use_shard: cover only the context's shard of the units (options.shard_index / shard_count)
cudaError_t launch_screen_ex(recon_ctx *c, const void *A, const void *B, int K, float thr, const float *l1,
                             float rel, int product_margin, bool skip_stored, int32_t *out, int64_t cap,
                             unsigned long long *count, double *flop_out, bool fp8, float abs_margin,
                             int k_valid, const float2 *r1, bool use_shard);
int screen_k_rank1(recon_ctx *c);
float screen_rank1_margin(recon_ctx *c);
cudaError_t launch_screen_prep_rank1(recon_ctx *c, void *A, float2 *r1, unsigned long long *flag);

// host helpers (api.cu)
recon_status set_err(recon_ctx *c, recon_status st, const char *fmt, ...);
recon_status cuda_fail(recon_ctx *c, cudaError_t e, const char *where);
