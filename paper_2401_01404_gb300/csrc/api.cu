// api.cu -- the C ABI of librecon (declared in include/recon.h): argument
// checking, device state, and the host orchestration of the kernels.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "common.cuh"
#include "proposal.cuh"
#include "search.cuh"

static thread_local std::string g_err;  // errors without a context
thread_local recon_ctx *tl_ctx = nullptr;

cudaError_t recon_malloc(void **p, size_t bytes) {
    recon_ctx *c = tl_ctx;
    if (c && c->alloc_limit && c->alloc_total + bytes > c->alloc_limit) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess && c) c->alloc_total += bytes;
    return e;
}

recon_status set_err(recon_ctx *c, recon_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) {
        c->err = buf;
        if (st == RECON_ECUDA || st == RECON_ETIMEOUT) c->broken = true;
    } else
        g_err = buf;
    return st;
}

recon_status cuda_fail(recon_ctx *c, cudaError_t e, const char *where) {
    return set_err(c, RECON_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call)                                                \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);  \
    } while (0)

#define LIVE(c)                                                                                     \
    do {                                                                                            \
        if (!(c)) return set_err(nullptr, RECON_EINVAL, "null context");                            \
        tl_ctx = (c);                                                                               \
        if ((c)->broken) return set_err((c), RECON_ESTATE, "context unusable after an earlier error: %s", \
                                        (c)->err.c_str());                                          \
    } while (0)

bool ensure_buf(recon_ctx *c, int slot, size_t bytes) {
    DBuf &b = c->bufs[slot];
    if (b.bytes >= bytes) return true;
    if (b.p) {
        cudaStreamSynchronize(c->stream);
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    size_t want = std::max<size_t>(bytes, 256);
    want += want / 4;
    if (recon_malloc(&b.p, want) != cudaSuccess) {
        cudaGetLastError();
        set_err(c, RECON_ENOMEM, "device allocation of %zu bytes failed", want);
        return false;
    }
    b.bytes = want;
    return true;
}

#define ENSURE(slot, bytes)                                    \
    do {                                                       \
        if (!ensure_buf(c, (slot), (bytes))) return RECON_ENOMEM; \
    } while (0)

static float effective_wclamp(int model, float w) {
    if (w > 0) return w;
    return model == RECON_ISING ? 5.0f : FLT_MAX;
}

extern "C" void recon_default_options(recon_options *o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->lambda = 0.0;
    o->seed = 1;
    o->eps_knn = 1e-3;
    o->max_knn_iters = 0;
    o->w_clamp = 0.f;  // model default: 5 for Ising, none for Gaussian
    o->h_clamp = 10.f;
    o->knn_mode = RECON_KNN_NNDESCENT;
    o->seed_mode = RECON_SEED_RANDOM;
    o->screen_c = 0;
    o->learned_frac = 0.5f;
}

static recon_status read_err_flags(recon_ctx *c, unsigned long long *flags) {
    CK(cudaMemcpyAsync(c->cnt_host + CNT_ERR, c->cnt + CNT_ERR, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *flags = c->cnt_host[CNT_ERR];
    if (*flags) CK(cudaMemsetAsync(c->cnt + CNT_ERR, 0, sizeof(unsigned long long), c->stream));
    return RECON_OK;
}

static recon_status alloc_table(recon_ctx *c, uint64_t cap) {
    WTable T{};
    if (recon_malloc((void **)&T.keys, sizeof(unsigned long long) * cap) != cudaSuccess ||
        recon_malloc((void **)&T.vals, sizeof(float) * cap) != cudaSuccess) {
        cudaGetLastError();
        if (T.keys) cudaFree(T.keys);
        return set_err(c, RECON_ENOMEM, "coupling table of %llu slots", (unsigned long long)cap);
    }
    T.mask = cap - 1;
    CK(launch_fill_u64(T.keys, RECON_EMPTY_KEY, (int64_t)cap, c->stream));
    if (c->W.keys) {
        CK(launch_table_rehash(c->W, T, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        cudaFree(c->W.keys);
        cudaFree(c->W.vals);
    }
    c->W = T;
    c->w_cap = cap;
    return RECON_OK;
}

static recon_status table_count(recon_ctx *c, int64_t *n) {
    CK(cudaMemsetAsync(c->cnt + CNT_SCRATCH0, 0, sizeof(unsigned long long), c->stream));
    CK(launch_table_count(c->W, c->cnt + CNT_SCRATCH0, c->stream));
    CK(cudaMemcpyAsync(c->cnt_host + CNT_SCRATCH0, c->cnt + CNT_SCRATCH0, sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *n = (int64_t)c->cnt_host[CNT_SCRATCH0];
    return RECON_OK;
}

// keep the load factor of the coupling table below one half with `extra` more keys
static recon_status table_reserve(recon_ctx *c, int64_t extra) {
    int64_t n = 0;
    recon_status st = table_count(c, &n);
    if (st != RECON_OK) return st;
    c->stats.nnz = n;
    uint64_t cap = c->w_cap;
    while ((uint64_t)(2 * (n + extra)) > cap) cap <<= 1;
    if (cap != c->w_cap) return alloc_table(c, cap);
    return RECON_OK;
}

static void free_ctx(recon_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    void *ps[] = {c->xbits, c->xbitsT, c->phi, c->t,      c->h,      c->H,     c->T,     c->xg,
                  c->e,     c->mu,     c->s2,  c->Q, c->W.keys, c->W.vals, c->cnt};
    for (void *p : ps)
        if (p) cudaFree(p);
    if (c->cnt_host) cudaFreeHost(c->cnt_host);
    for (auto &t : c->timed) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
    if (tl_ctx == c) tl_ctx = nullptr;
    for (DBuf &b : c->bufs)
        if (b.p) cudaFree(b.p);
    free_search_bufs(c->sb);
    free_proposal(c->prop);
    if (c->nnd_exec) cudaGraphExecDestroy(c->nnd_exec);
    if (c->nnd_loop_exec) cudaGraphExecDestroy(c->nnd_loop_exec);
    for (cudaEvent_t e : {c->nnd_ea, c->nnd_eb})
        if (e) cudaEventDestroy(e);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    delete c;
}

static recon_status alloc_dev(recon_ctx *c, void **p, size_t bytes) {
    if (recon_malloc(p, std::max<size_t>(bytes, 4)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_err(c, RECON_ENOMEM, "device allocation of %zu bytes failed", bytes);
    }
    return RECON_OK;
}
#define ALLOC(ptr, bytes)                                                       \
    do {                                                                        \
        recon_status s_ = alloc_dev(c, (void **)&(ptr), (bytes));               \
        if (s_ != RECON_OK) return s_;                                          \
    } while (0)

// builds the device state of a fresh context from sample-major X
static recon_status build_state(recon_ctx *c, const void *X, int x_is_device) {
    const int64_t N = c->N, M = c->M;
    const size_t esz = c->model == RECON_ISING ? 1 : 4;
    const size_t xbytes = (size_t)N * M * esz;
    // the samples are kept only in the device layout (checkpoints unpack them)
    void *Xd = nullptr;
    if (x_is_device) {
        Xd = const_cast<void *>(X);
    } else {
        ENSURE(BUF_TMP0, xbytes);
        Xd = c->bufs[BUF_TMP0].p;
        CK(cudaMemcpyAsync(Xd, X, xbytes, cudaMemcpyHostToDevice, c->stream));
    }
    ALLOC(c->cnt, sizeof(unsigned long long) * CNT_N);
    CK(cudaMemsetAsync(c->cnt, 0, sizeof(unsigned long long) * CNT_N, c->stream));
    if (cudaMallocHost(&c->cnt_host, sizeof(unsigned long long) * CNT_N) != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, RECON_ENOMEM, "pinned host allocation failed");
    }
    const size_t rows = (size_t)N * c->Mp * sizeof(float);
    if (c->model == RECON_ISING) {
        ALLOC(c->xbits, (size_t)N * c->Mw * sizeof(uint32_t));
        ALLOC(c->xbitsT, (size_t)N * 32 * sizeof(uint32_t));
        ALLOC(c->phi, rows);
        ALLOC(c->t, rows);
        ALLOC(c->h, N * sizeof(float));
        ALLOC(c->H, N * sizeof(float));
        ALLOC(c->T, N * sizeof(float));
        CK(launch_ising_pack((const int8_t *)Xd, M, N, (int)c->Mw, c->xbits, c->cnt, c->stream));
        CK(launch_ising_transpose_bits(c->iv(), c->xbitsT, c->stream));
        CK(ising_score_seg_setup());
        CK(launch_ising_init_fields(c->iv(), c->opt.h_clamp, c->stream));
    } else {
        ALLOC(c->xg, rows);
        ALLOC(c->e, rows);
        ALLOC(c->mu, rows);
        ALLOC(c->s2, N * sizeof(float));
        ALLOC(c->Q, N * sizeof(float));
        CK(launch_gauss_pack((const float *)Xd, M, N, (int)c->Mp, c->xg, c->cnt, c->stream));
        CK(launch_gauss_init(c->gv(), c->stream));
    }
    uint64_t cap = 1;
    while (cap < (uint64_t)std::max<int64_t>(4096, 4 * N)) cap <<= 1;
    recon_status st = alloc_table(c, cap);
    if (st != RECON_OK) return st;
    unsigned long long flags = 0;
    st = read_err_flags(c, &flags);
    if (st != RECON_OK) return st;
    if (flags & ERR_BAD_SPIN) return set_err(c, RECON_EINVAL, "X holds a spin that is neither -1 nor +1");
    if (flags & ERR_BAD_VALUE) return set_err(c, RECON_EINVAL, "X holds a non-finite sample");
    return RECON_OK;
}

extern "C" recon_status recon_init(recon_ctx **out, const void *X, int64_t M, int64_t N, int32_t x_type,
                                   int32_t x_is_device, int32_t model, const recon_options *opt, void *stream) {
    if (!out) return set_err(nullptr, RECON_EINVAL, "out is NULL");
    *out = nullptr;
    if (!X) return set_err(nullptr, RECON_EINVAL, "X is NULL");
    if (N < 2) return set_err(nullptr, RECON_EINVAL, "N = %lld < 2", (long long)N);
    if (M < 1) return set_err(nullptr, RECON_EINVAL, "M = %lld < 1", (long long)M);
    if (N > 0x3fffffff) return set_err(nullptr, RECON_EINVAL, "N = %lld too large", (long long)N);
    if (model != RECON_ISING && model != RECON_GAUSSIAN) return set_err(nullptr, RECON_EINVAL, "unknown model %d", model);
    if (model == RECON_ISING && x_type != RECON_X_INT8)
        return set_err(nullptr, RECON_EINVAL, "the Ising model takes int8 spins");
    if (model == RECON_GAUSSIAN && x_type != RECON_X_FP32)
        return set_err(nullptr, RECON_EINVAL, "the Gaussian model takes float samples");
    recon_options o;
    recon_default_options(&o);
    if (opt) o = *opt;
    if (!(o.lambda >= 0.0) || !std::isfinite(o.lambda)) return set_err(nullptr, RECON_EINVAL, "lambda must be finite and >= 0");
    if (!(o.h_clamp > 0.f)) return set_err(nullptr, RECON_EINVAL, "h_clamp must be > 0");
    if (o.w_clamp < 0.f) return set_err(nullptr, RECON_EINVAL, "w_clamp must be >= 0");
    if (model == RECON_ISING && o.w_clamp > 8.f)
        return set_err(nullptr, RECON_EINVAL, "w_clamp above 8 is not supported for the Ising model");
    if (o.knn_mode < 0 || o.knn_mode > 3) return set_err(nullptr, RECON_EINVAL, "unknown knn_mode");
    if (o.distance != RECON_DIST_GAIN && o.distance != RECON_DIST_GRADIENT)
        return set_err(nullptr, RECON_EINVAL, "unknown distance");
    if (o.distance == RECON_DIST_GRADIENT && o.knn_mode == RECON_KNN_SCREEN)
        return set_err(nullptr, RECON_EUNSUPPORTED, "the gradient distance ranks pairs the screen does not keep");
    if (o.shard_count < 0 || (o.shard_count > 1 && (o.shard_index < 0 || o.shard_index >= o.shard_count)))
        return set_err(nullptr, RECON_EINVAL, "shard_index %d outside [0, shard_count = %d)", o.shard_index,
                       o.shard_count);
    if (o.shard_count > 1 && o.knn_mode != RECON_KNN_SCREEN)
        return set_err(nullptr, RECON_EUNSUPPORTED, "a sharded search needs RECON_KNN_SCREEN");
    if (o.screen_fp8 && model != RECON_ISING)
        return set_err(nullptr, RECON_EUNSUPPORTED, "fp8 screen operands are for the Ising model only");
    if (!(o.learned_frac >= 0.f && o.learned_frac <= 1.f))
        return set_err(nullptr, RECON_EINVAL, "learned_frac outside [0, 1]");
    if (o.seed_mode != RECON_SEED_RANDOM && o.seed_mode != RECON_SEED_LEARNED)
        return set_err(nullptr, RECON_EUNSUPPORTED, "seed_mode: RANDOM or LEARNED (the screen is knn_mode SCREEN)");
    if (o.seed_mode == RECON_SEED_LEARNED && model != RECON_ISING)
        return set_err(nullptr, RECON_EUNSUPPORTED, "the learned proposal is built for the Ising model");
    const int64_t Mp = (M + 31) / 32 * 32;
    if (model == RECON_ISING && Mp / 32 > ising_max_words())
        return set_err(nullptr, RECON_EUNSUPPORTED, "the Ising path supports M <= %d", 32 * ising_max_words());
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(nullptr, RECON_ECUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
    }
    recon_ctx *c = new recon_ctx();
    c->bufs.resize(BUF_NSLOTS);
    if (const char *lim = getenv("RECON_FAULT_ALLOC_LIMIT")) c->alloc_limit = strtoull(lim, nullptr, 10);
    if (const char *st = getenv("RECON_FAULT_SCREEN_STALL")) c->fault_screen_stall = atoi(st) != 0;
    if (const char *st = getenv("RECON_FAULT_SCORE_STALL")) c->fault_score_stall = atoi(st) != 0;
    // (tests: FindBest's small-level selection and final list by the general sorts)
    if (const char *st = getenv("RECON_FINDBEST_SORTS")) c->findbest_sorts = atoi(st) != 0;
    c->model = model;
    c->device = dev;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
    c->N = N;
    c->M = M;
    c->Mp = Mp;
    c->Mw = Mp / 32;
    c->opt = o;
    c->opt.w_clamp = effective_wclamp(model, o.w_clamp);
    c->stream = (cudaStream_t)stream;
    c->stats.samples = M;
    tl_ctx = c;
    recon_status st = build_state(c, X, x_is_device);
    if (st != RECON_OK) {
        g_err = c->err;
        free_ctx(c);
        return st;
    }
    *out = c;
    return RECON_OK;
}

extern "C" recon_status recon_objective(recon_ctx *c, double *out) {
    LIVE(c);
    if (!out) return set_err(c, RECON_EINVAL, "out is NULL");
    const int nb = 1024;
    ENSURE(BUF_TMP1, sizeof(double) * (nb + 256 + 2));
    double *part = buf<double>(c, BUF_TMP1);
    if (c->model == RECON_ISING)
        CK(launch_ising_objective(c->iv(), part, nb, c->stream));
    else
        CK(launch_gauss_objective(c->gv(), part, nb, c->stream));
    CK(launch_penalty(c->W, part + nb, c->stream));
    CK(launch_sum_doubles(part, nb, part + nb + 256, c->stream));
    CK(launch_sum_doubles(part + nb, 256, part + nb + 257, c->stream));
    double r[2];
    CK(cudaMemcpyAsync(r, part + nb + 256, sizeof r, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *out = r[0] - c->opt.lambda * r[1];
    return RECON_OK;
}

// device copy of a caller's pair list, checked
static recon_status stage_pairs(recon_ctx *c, const int32_t *pairs, int64_t P, int is_device, int slot,
                                const int32_t **dev) {
    if (is_device) {
        *dev = pairs;
    } else {
        ENSURE(slot, sizeof(int32_t) * 2 * P);
        CK(cudaMemcpyAsync(c->bufs[slot].p, pairs, sizeof(int32_t) * 2 * P, cudaMemcpyHostToDevice, c->stream));
        *dev = buf<int32_t>(c, slot);
    }
    CK(launch_check_pairs(*dev, P, (int)c->N, c->cnt, c->stream));
    unsigned long long flags = 0;
    recon_status st = read_err_flags(c, &flags);
    if (st != RECON_OK) return st;
    if (flags & ERR_BAD_VALUE) return set_err(c, RECON_EINVAL, "a pair has an id outside [0, N) or i == j");
    return RECON_OK;
}

extern "C" recon_status recon_score(recon_ctx *c, const int32_t *pairs, int64_t P, float *d_out, float *w_out,
                                    int32_t io_is_device) {
    LIVE(c);
    if (P < 0) return set_err(c, RECON_EINVAL, "P < 0");
    if (P == 0) return RECON_OK;
    if (!pairs || !d_out) return set_err(c, RECON_EINVAL, "pairs or d_out is NULL");
    const int32_t *dp = nullptr;
    recon_status st = stage_pairs(c, pairs, P, io_is_device, BUF_PAIRS, &dp);
    if (st != RECON_OK) return st;
    float *dd = d_out, *ww = w_out;
    if (!io_is_device) {
        ENSURE(BUF_GAIN, sizeof(float) * P);
        dd = buf<float>(c, BUF_GAIN);
        if (w_out) {
            ENSURE(BUF_WST, sizeof(float) * P);
            ww = buf<float>(c, BUF_WST);
        }
    }
    st = score_pairs_device(c, dp, P, nullptr, dd, ww);
    if (st != RECON_OK) return st;
    if (!io_is_device) {
        CK(cudaMemcpyAsync(d_out, dd, sizeof(float) * P, cudaMemcpyDeviceToHost, c->stream));
        if (w_out) CK(cudaMemcpyAsync(w_out, ww, sizeof(float) * P, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return RECON_OK;
}

static recon_status deliver_pairs(recon_ctx *c, const int32_t *pd, const float *dd, int64_t n, int32_t *pairs,
                                  float *d, int32_t out_is_device) {
    if (n == 0) return RECON_OK;
    cudaMemcpyKind kind = out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(pairs, pd, sizeof(int32_t) * 2 * n, kind, c->stream));
    if (d) CK(cudaMemcpyAsync(d, dd, sizeof(float) * n, kind, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return RECON_OK;
}

static int64_t round_half_up(double x) { return (int64_t)std::floor(x + 0.5); }

extern "C" recon_status recon_best_pairs(recon_ctx *c, int32_t k, double kappa, int32_t *pairs, float *d, int64_t cap,
                                         int64_t *m_out, int32_t out_is_device) {
    LIVE(c);
    if (!m_out) return set_err(c, RECON_EINVAL, "m_out is NULL");
    if (k < 1) return set_err(c, RECON_EINVAL, "k = %d < 1", k);
    if (!(kappa > 0.0) || !std::isfinite(kappa)) return set_err(c, RECON_EINVAL, "kappa must be > 0");
    const int64_t npairs = c->N * (c->N - 1) / 2;
    const int64_t m = std::min<int64_t>(round_half_up(kappa * (double)c->N), npairs);
    if (m < 1) return set_err(c, RECON_EINVAL, "kappa*N rounds to 0");
    if (cap < m || !pairs) {
        *m_out = m;
        return set_err(c, RECON_EINVAL, "cap %lld < m = %lld", (long long)cap, (long long)m);
    }
    int32_t *pd = nullptr;
    float *dd = nullptr;
    int64_t n = 0;
    recon_status st = findbest_run(c, k, m, &pd, &dd, &n);
    if (st != RECON_OK) return st;
    st = deliver_pairs(c, pd, dd, n, pairs, d, out_is_device);
    if (st != RECON_OK) return st;
    *m_out = n;
    return RECON_OK;
}

extern "C" recon_status recon_exhaustive_best(recon_ctx *c, int64_t m, int32_t *pairs, float *d, int64_t cap,
                                              int64_t *m_out, int32_t out_is_device) {
    LIVE(c);
    if (!m_out) return set_err(c, RECON_EINVAL, "m_out is NULL");
    if (m < 1) return set_err(c, RECON_EINVAL, "m < 1");
    m = std::min<int64_t>(m, c->N * (c->N - 1) / 2);
    if (cap < m || !pairs) {
        *m_out = m;
        return set_err(c, RECON_EINVAL, "cap %lld < m = %lld", (long long)cap, (long long)m);
    }
    int32_t *pd = nullptr;
    float *dd = nullptr;
    int64_t n = 0;
    recon_status st = exhaustive_run(c, m, &pd, &dd, &n);
    if (st != RECON_OK) return st;
    st = deliver_pairs(c, pd, dd, n, pairs, d, out_is_device);
    if (st != RECON_OK) return st;
    *m_out = n;
    return RECON_OK;
}

extern "C" recon_status recon_select_best(recon_ctx *c, const int32_t *pairs, const float *d, int64_t P, int64_t m,
                                          int32_t *out_pairs, float *out_d, int64_t cap, int64_t *count_out,
                                          int32_t io_is_device) {
    LIVE(c);
    if (!count_out) return set_err(c, RECON_EINVAL, "count_out is NULL");
    *count_out = 0;
    if (P < 0 || m < 0) return set_err(c, RECON_EINVAL, "P or m < 0");
    if (P > 0 && (!pairs || !d)) return set_err(c, RECON_EINVAL, "pairs or d is NULL");
    if (P == 0 || m == 0) return RECON_OK;
    const int32_t *pin = pairs;
    const float *din = d;
    if (!io_is_device) {
        ENSURE(BUF_TMP0, sizeof(int32_t) * 2 * P);
        ENSURE(BUF_TMP1, sizeof(float) * P);
        CK(cudaMemcpyAsync(c->bufs[BUF_TMP0].p, pairs, sizeof(int32_t) * 2 * P, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->bufs[BUF_TMP1].p, d, sizeof(float) * P, cudaMemcpyHostToDevice, c->stream));
        pin = buf<int32_t>(c, BUF_TMP0);
        din = buf<float>(c, BUF_TMP1);
    }
    int32_t *pd = nullptr;
    float *dd = nullptr;
    int64_t n = 0;
    recon_status st = select_run(c, pin, din, P, m, &pd, &dd, &n);
    if (st != RECON_OK) {
        if (st == RECON_EINVAL) return set_err(c, RECON_EINVAL, "a pair has an id outside [0, N) or i == j");
        return st;
    }
    if (cap < n || !out_pairs) {
        *count_out = n;
        return set_err(c, RECON_EINVAL, "cap %lld < %lld selected pairs", (long long)cap, (long long)n);
    }
    st = deliver_pairs(c, pd, dd, n, out_pairs, out_d, io_is_device);
    if (st != RECON_OK) return st;
    *count_out = n;
    return RECON_OK;
}

extern "C" recon_status recon_row_best(recon_ctx *c, const int32_t *rows, int64_t nrows, float d_cut, int32_t *pairs,
                                       float *d, int64_t cap, int64_t *count_out) {
    LIVE(c);
    if (!count_out) return set_err(c, RECON_EINVAL, "count_out is NULL");
    *count_out = 0;
    if (nrows < 0 || (nrows > 0 && !rows)) return set_err(c, RECON_EINVAL, "rows");
    if (cap < 0 || (cap > 0 && !pairs)) return set_err(c, RECON_EINVAL, "pairs / cap");
    if (std::isnan(d_cut)) return set_err(c, RECON_EINVAL, "d_cut is NaN");
    for (int64_t r = 0; r < nrows; ++r)
        if (rows[r] < 0 || rows[r] >= c->N) return set_err(c, RECON_EINVAL, "row %lld = %d outside [0, N)", (long long)r, rows[r]);
    if (nrows == 0 || c->N < 2) return RECON_OK;
    ENSURE(BUF_TMP2, sizeof(int32_t) * nrows);
    CK(cudaMemcpyAsync(c->bufs[BUF_TMP2].p, rows, sizeof(int32_t) * nrows, cudaMemcpyHostToDevice, c->stream));
    int32_t *pd = nullptr;
    float *dd = nullptr;
    int64_t n = 0;
    recon_status st = row_best_run(c, buf<int32_t>(c, BUF_TMP2), nrows, d_cut, &pd, &dd, &n);
    if (st != RECON_OK) return st;
    st = deliver_pairs(c, pd, dd, std::min(n, cap), pairs, d, 0);
    if (st != RECON_OK) return st;
    *count_out = n;
    return RECON_OK;
}

// the update loop over a device pair list (already checked)
static recon_status cd_sweep_dev(recon_ctx *c, const int32_t *dp, int64_t P, double *delta_out) {
    if (P == 0) {
        if (delta_out) *delta_out = 0.0;
        return RECON_OK;
    }
    recon_status st = table_reserve(c, P);
    if (st != RECON_OK) return st;
    ENSURE(BUF_BATCH, sizeof(int) * P);
    ENSURE(BUF_ORDER, sizeof(int) * P);
    ENSURE(BUF_OFF, sizeof(int) * (P + 2));
    ENSURE(BUF_DELTA, sizeof(double) * (P + 1));
    ENSURE(BUF_TMP2, sizeof(int) * 2);
    ENSURE(BUF_SORT0, sizeof(unsigned long long) * 2 * P);
    ENSURE(BUF_SORT1, sizeof(unsigned long long) * 2 * P);
    ENSURE(BUF_SORT2, sizeof(uint32_t) * 4 * P);
    ENSURE(BUF_SORT3, sizeof(int64_t) * layer_tmp_elems(P));
    ENSURE(BUF_SORT4, sizeof(int32_t) * 5 * P);
    int *nb_dev = buf<int>(c, BUF_TMP2);
    int32_t *links = buf<int32_t>(c, BUF_SORT4);
    uint32_t *vals = buf<uint32_t>(c, BUF_SORT2);
    CK(launch_layer_frontier(dp, P, (int)c->N, buf<unsigned long long>(c, BUF_SORT0),
                             buf<unsigned long long>(c, BUF_SORT1), vals, vals + 2 * P, buf<int64_t>(c, BUF_SORT3),
                             links, links + 2 * P, links + 3 * P, links + 4 * P, buf<int>(c, BUF_BATCH),
                             buf<int>(c, BUF_ORDER), buf<int>(c, BUF_OFF), nb_dev, c->stream));
    // the batch count and (usually all of) the batch offsets in one round trip
    int nb = 0;
    const int64_t guess = std::min<int64_t>(P + 1, 257);
    std::vector<int> off((size_t)guess);
    CK(cudaMemcpyAsync(&nb, nb_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(off.data(), buf<int>(c, BUF_OFF), sizeof(int) * guess, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (nb + 1 > guess) {
        off.resize(nb + 1);
        CK(cudaMemcpyAsync(off.data(), buf<int>(c, BUF_OFF), sizeof(int) * (nb + 1), cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    double *delta = buf<double>(c, BUF_DELTA);
    const int *offd = buf<int>(c, BUF_OFF), *order = buf<int>(c, BUF_ORDER);
    // a batch with at most `thin` pairs joins a run of thin batches that one block
    // applies in turn (block barriers between them); a wider batch gets a grid
    const int thin = c->model == RECON_ISING ? 8 : 64;
    for (int b = 0; b < nb;) {
        if (off[b + 1] - off[b] > thin) {
            if (c->model == RECON_ISING)
                CK(launch_ising_update(c->iv(), c->W, c->sp(), dp, order, off[b], off[b + 1], delta, c->cnt,
                                       c->stream));
            else
                CK(launch_gauss_update(c->gv(), c->W, c->sp(), dp, order, off[b], off[b + 1], delta, c->cnt,
                                       c->stream));
            ++b;
            continue;
        }
        int e = b;
        while (e < nb && off[e + 1] - off[e] <= thin) ++e;
        if (c->model == RECON_ISING)
            CK(launch_ising_update_rounds(c->iv(), c->W, c->sp(), dp, order, offd, b, e, delta, c->cnt, c->stream));
        else
            CK(launch_gauss_update_rounds(c->gv(), c->W, c->sp(), dp, order, offd, b, e, delta, c->cnt, c->stream));
        b = e;
    }
    c->stats.pair_evals += P;
    CK(launch_sum_doubles(delta, P, delta + P, c->stream));
    double r = 0.0;
    CK(cudaMemcpyAsync(&r, delta + P, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    unsigned long long flags = 0;
    st = read_err_flags(c, &flags);
    if (st != RECON_OK) return st;
    if (flags & ERR_TABLE_FULL) return set_err(c, RECON_ENOMEM, "coupling table full");
    if (delta_out) *delta_out = r;
    return RECON_OK;
}

extern "C" recon_status recon_cd_sweep(recon_ctx *c, const int32_t *pairs, int64_t P, int32_t pairs_is_device,
                                       double *delta_out) {
    LIVE(c);
    if (P < 0) return set_err(c, RECON_EINVAL, "P < 0");
    if (P > 0x7ffffff0) return set_err(c, RECON_EINVAL, "P too large");
    if (P > 0 && !pairs) return set_err(c, RECON_EINVAL, "pairs is NULL");
    const int32_t *dp = nullptr;
    if (P > 0) {
        recon_status st = stage_pairs(c, pairs, P, pairs_is_device, BUF_PAIRS, &dp);
        if (st != RECON_OK) return st;
    }
    return cd_sweep_dev(c, dp, P, delta_out);
}

extern "C" recon_status recon_field_sweep(recon_ctx *c, double *delta_out) {
    LIVE(c);
    ENSURE(BUF_DELTA, sizeof(double) * (c->N + 1));
    double *delta = buf<double>(c, BUF_DELTA);
    if (c->model == RECON_ISING)
        CK(launch_ising_field_sweep(c->iv(), c->sp(), delta, c->stream));
    else
        CK(launch_gauss_diag_sweep(c->gv(), delta, c->stream));
    CK(launch_sum_doubles(delta, c->N, delta + c->N, c->stream));
    double r = 0.0;
    CK(cudaMemcpyAsync(&r, delta + c->N, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (delta_out) *delta_out = r;
    return RECON_OK;
}

extern "C" recon_status recon_set_list_lengths(recon_ctx *c, const int32_t *k, int64_t n) {
    LIVE(c);
    if (n == 0) {
        c->klen_host.clear();
        return RECON_OK;
    }
    if (n != c->N || !k) return set_err(c, RECON_EINVAL, "give N = %lld lengths (or n = 0 to clear)", (long long)c->N);
    for (int64_t x = 0; x < n; ++x)
        if (k[x] < 1 || k[x] > 64) return set_err(c, RECON_EINVAL, "list length %d of node %lld outside [1, 64]", k[x], (long long)x);
    c->klen_host.assign(k, k + n);
    return RECON_OK;
}

extern "C" recon_status recon_knn_graph(recon_ctx *c, int32_t *ids, float *d, int64_t cap, int32_t *k_out,
                                        int64_t *n_out) {
    LIVE(c);
    if (cap < 0) return set_err(c, RECON_EINVAL, "cap < 0");
    return knn_graph_copy(c, ids, d, cap, k_out, n_out);
}

extern "C" recon_status recon_gcd_step(recon_ctx *c, int32_t k, double kappa, double *delta_out,
                                       double *objective_out, int64_t *m_out) {
    LIVE(c);
    if (c->opt.shard_count > 1)
        return set_err(c, RECON_EUNSUPPORTED, "a sharded context returns its shard's best pairs; merge them "
                                              "(recon_select_best) before the updates");
    if (k < 1) return set_err(c, RECON_EINVAL, "k = %d < 1", k);
    if (!(kappa > 0.0) || !std::isfinite(kappa)) return set_err(c, RECON_EINVAL, "kappa must be > 0");
    const int64_t m = std::min<int64_t>(round_half_up(kappa * (double)c->N), c->N * (c->N - 1) / 2);
    int32_t *pd = nullptr;
    float *dd = nullptr;
    int64_t n = 0;
    recon_status st = findbest_run(c, k, std::max<int64_t>(m, 1), &pd, &dd, &n);
    if (st != RECON_OK) return st;
    // the selected pairs are overwritten by later searches: keep a copy
    ENSURE(BUF_TMP3, sizeof(int32_t) * 2 * std::max<int64_t>(n, 1));
    CK(cudaMemcpyAsync(c->bufs[BUF_TMP3].p, pd, sizeof(int32_t) * 2 * n, cudaMemcpyDeviceToDevice, c->stream));
    double d1 = 0.0, d2 = 0.0;
    st = cd_sweep_dev(c, buf<int32_t>(c, BUF_TMP3), n, &d1);
    if (st != RECON_OK) return st;
    st = recon_field_sweep(c, &d2);
    if (st != RECON_OK) return st;
    if (delta_out) *delta_out = d1 + d2;
    if (m_out) *m_out = n;
    if (objective_out) return recon_objective(c, objective_out);
    return RECON_OK;
}

extern "C" recon_status recon_get_model(recon_ctx *c, int32_t *ij, float *w, int64_t cap, int64_t *nnz, float *fields) {
    LIVE(c);
    if (!nnz) return set_err(c, RECON_EINVAL, "nnz is NULL");
    int64_t n = 0;
    recon_status st = table_count(c, &n);
    if (st != RECON_OK) return st;
    *nnz = n;
    c->stats.nnz = n;
    if (cap < n || (n > 0 && (!ij || !w))) {
        if (fields) {
            CK(cudaMemcpyAsync(fields, c->model == RECON_ISING ? c->h : c->s2, sizeof(float) * c->N,
                               cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
        }
        if (cap < n) return set_err(c, RECON_EINVAL, "cap %lld < nnz %lld", (long long)cap, (long long)n);
        return set_err(c, RECON_EINVAL, "ij or w is NULL");
    }
    if (n > 0) {
        ENSURE(BUF_TMP1, sizeof(int32_t) * 2 * n);
        ENSURE(BUF_TMP2, sizeof(float) * n);
        CK(cudaMemsetAsync(c->cnt + CNT_SCRATCH1, 0, sizeof(unsigned long long), c->stream));
        CK(launch_table_dump(c->W, buf<int32_t>(c, BUF_TMP1), buf<float>(c, BUF_TMP2), c->cnt + CNT_SCRATCH1,
                             c->stream));
        std::vector<int32_t> hij(2 * n);
        std::vector<float> hw(n);
        CK(cudaMemcpyAsync(hij.data(), c->bufs[BUF_TMP1].p, sizeof(int32_t) * 2 * n, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(hw.data(), c->bufs[BUF_TMP2].p, sizeof(float) * n, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        std::vector<int64_t> ord(n);
        for (int64_t q = 0; q < n; ++q) ord[q] = q;
        std::sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) {
            return hij[2 * a] != hij[2 * b] ? hij[2 * a] < hij[2 * b] : hij[2 * a + 1] < hij[2 * b + 1];
        });
        for (int64_t q = 0; q < n; ++q) {
            ij[2 * q] = hij[2 * ord[q]];
            ij[2 * q + 1] = hij[2 * ord[q] + 1];
            w[q] = hw[ord[q]];
        }
    }
    if (fields) {
        CK(cudaMemcpyAsync(fields, c->model == RECON_ISING ? c->h : c->s2, sizeof(float) * c->N, cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return RECON_OK;
}

extern "C" recon_status recon_set_model(recon_ctx *c, const int32_t *ij, const float *w, int64_t nnz,
                                        const float *fields) {
    LIVE(c);
    if (nnz < 0 || (nnz > 0 && (!ij || !w))) return set_err(c, RECON_EINVAL, "bad coupling list");
    std::vector<int64_t> deg(c->N + 1, 0);
    std::vector<uint64_t> keys(nnz);
    for (int64_t q = 0; q < nnz; ++q) {
        int a = ij[2 * q], b = ij[2 * q + 1];
        if (a < 0 || b < 0 || a >= c->N || b >= c->N || a == b)
            return set_err(c, RECON_EINVAL, "coupling %lld has a bad pair (%d, %d)", (long long)q, a, b);
        if (!std::isfinite(w[q])) return set_err(c, RECON_EINVAL, "coupling %lld is not finite", (long long)q);
        keys[q] = pair_key(a, b);
        deg[a]++;
        deg[b]++;
    }
    {
        std::vector<uint64_t> s = keys;
        std::sort(s.begin(), s.end());
        if (std::adjacent_find(s.begin(), s.end()) != s.end()) return set_err(c, RECON_EINVAL, "a pair repeats");
    }
    if (fields)
        for (int64_t i = 0; i < c->N; ++i)
            if (!std::isfinite(fields[i]) || (c->model == RECON_GAUSSIAN && !(fields[i] > 0.f)))
                return set_err(c, RECON_EINVAL, "bad per-node parameter %lld", (long long)i);
    // CSR of the symmetric couplings, neighbours ascending
    std::vector<int64_t> off(c->N + 1, 0);
    for (int64_t i = 0; i < c->N; ++i) off[i + 1] = off[i] + deg[i];
    std::vector<std::pair<int32_t, float>> tmp(off[c->N]);
    std::vector<int64_t> cur(off.begin(), off.end() - 1);
    for (int64_t q = 0; q < nnz; ++q) {
        int a = ij[2 * q], b = ij[2 * q + 1];
        tmp[cur[a]++] = {b, w[q]};
        tmp[cur[b]++] = {a, w[q]};
    }
    std::vector<int32_t> nbr(off[c->N]);
    std::vector<float> wv(off[c->N]);
    for (int64_t i = 0; i < c->N; ++i) {
        std::sort(tmp.begin() + off[i], tmp.begin() + off[i + 1]);
        for (int64_t e = off[i]; e < off[i + 1]; ++e) {
            nbr[e] = tmp[e].first;
            wv[e] = tmp[e].second;
        }
    }
    // fresh table
    uint64_t cap = 1;
    while (cap < (uint64_t)std::max<int64_t>(4096, std::max<int64_t>(4 * c->N, 4 * nnz))) cap <<= 1;
    if (c->W.keys) {
        CK(cudaStreamSynchronize(c->stream));
        cudaFree(c->W.keys);
        cudaFree(c->W.vals);
        c->W = WTable{};
    }
    recon_status st = alloc_table(c, cap);
    if (st != RECON_OK) return st;
    const int64_t E = off[c->N];
    ENSURE(BUF_TMP0, sizeof(int64_t) * (c->N + 1) + sizeof(int32_t) * (E + 1) + sizeof(float) * (E + 1) + 64);
    ENSURE(BUF_TMP1, sizeof(int32_t) * 2 * (nnz + 1) + sizeof(float) * (nnz + 1) + 64);
    char *b0 = (char *)c->bufs[BUF_TMP0].p;
    int64_t *d_off = (int64_t *)b0;
    int32_t *d_nbr = (int32_t *)(b0 + sizeof(int64_t) * (c->N + 1));
    float *d_w = (float *)(b0 + sizeof(int64_t) * (c->N + 1) + sizeof(int32_t) * (E + 1));
    char *b1 = (char *)c->bufs[BUF_TMP1].p;
    int32_t *d_ij = (int32_t *)b1;
    float *d_wl = (float *)(b1 + sizeof(int32_t) * 2 * (nnz + 1));
    CK(cudaMemcpyAsync(d_off, off.data(), sizeof(int64_t) * (c->N + 1), cudaMemcpyHostToDevice, c->stream));
    if (E) {
        CK(cudaMemcpyAsync(d_nbr, nbr.data(), sizeof(int32_t) * E, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(d_w, wv.data(), sizeof(float) * E, cudaMemcpyHostToDevice, c->stream));
    }
    if (nnz) {
        CK(cudaMemcpyAsync(d_ij, ij, sizeof(int32_t) * 2 * nnz, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(d_wl, w, sizeof(float) * nnz, cudaMemcpyHostToDevice, c->stream));
        CK(launch_table_insert(c->W, d_ij, d_wl, nnz, c->cnt, c->stream));
    }
    if (c->model == RECON_ISING) {
        if (fields) CK(cudaMemcpyAsync(c->h, fields, sizeof(float) * c->N, cudaMemcpyHostToDevice, c->stream));
        CK(launch_ising_phi_from_csr(c->iv(), d_off, d_nbr, d_w, c->stream));
    } else {
        if (fields) CK(cudaMemcpyAsync(c->s2, fields, sizeof(float) * c->N, cudaMemcpyHostToDevice, c->stream));
        CK(launch_gauss_mu_from_csr(c->gv(), d_off, d_nbr, d_w, c->stream));
    }
    unsigned long long flags = 0;
    st = read_err_flags(c, &flags);
    if (st != RECON_OK) return st;
    if (flags) return set_err(c, RECON_ENOMEM, "coupling table full");
    c->stats.nnz = nnz;
    return RECON_OK;
}

extern "C" recon_status recon_get_stats(recon_ctx *c, recon_stats *out) {
    LIVE(c);
    if (!out) return set_err(c, RECON_EINVAL, "out is NULL");
    CK(cudaMemcpyAsync(c->cnt_host + CNT_NEWTON, c->cnt + CNT_NEWTON, sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->stats.newton_passes = (int64_t)c->cnt_host[CNT_NEWTON] + c->newton_extra;
    c->stats.device_bytes = (int64_t)c->alloc_total;
    for (auto &t : c->timed) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, t.a, t.b));
        if (t.pairs >= 0) {
            c->stats.score_ms += ms;
            c->stats.score_launches += 1;
            c->stats.score_pairs += t.pairs;
        } else {  // a screen launch; -pairs carries nothing, its work is in screen_flop
            c->stats.screen_ms += ms;
            c->stats.screen_launches += 1;
        }
        c->event_pool.push_back(t.a);
        c->event_pool.push_back(t.b);
    }
    c->timed.clear();
    *out = c->stats;
    return RECON_OK;
}

// ---------------------------------------------------------------------------
// checkpoints
// ---------------------------------------------------------------------------
static const char kMagic[8] = {'R', 'E', 'C', 'O', 'N', 'C', 'K', '3'};

// the tracked per-sample state, saved as is so that a resumed run continues
// bit for bit: Ising phi, t and H; Gaussian mu and e
static std::vector<std::pair<float *, size_t>> state_arrays(recon_ctx *c) {
    const size_t rows = (size_t)c->N * c->Mp;
    if (c->model == RECON_ISING) return {{c->phi, rows}, {c->t, rows}, {c->H, (size_t)c->N}, {c->T, (size_t)c->N}};
    return {{c->mu, rows}, {c->e, rows}, {c->Q, (size_t)c->N}};
}

extern "C" recon_status recon_save(recon_ctx *c, const char *path) {
    LIVE(c);
    if (!path) return set_err(c, RECON_EINVAL, "path is NULL");
    int64_t nnz = 0;
    recon_status st = table_count(c, &nnz);
    if (st != RECON_OK) return st;
    std::vector<int32_t> ij(2 * std::max<int64_t>(nnz, 1));
    std::vector<float> w(std::max<int64_t>(nnz, 1)), fields(c->N);
    st = recon_get_model(c, ij.data(), w.data(), nnz, &nnz, fields.data());
    if (st != RECON_OK) return st;
    recon_stats s{};
    st = recon_get_stats(c, &s);
    if (st != RECON_OK) return st;
    // the samples, sample-major as recon_init took them, rebuilt from the device layout
    const size_t xbytes = (size_t)c->N * c->M * (c->model == RECON_ISING ? 1 : 4);
    std::vector<uint8_t> xs(xbytes);
    ENSURE(BUF_TMP0, xbytes);
    if (c->model == RECON_ISING)
        CK(launch_ising_unpack(c->iv(), buf<int8_t>(c, BUF_TMP0), c->stream));
    else
        CK(launch_gauss_unpack(c->gv(), buf<float>(c, BUF_TMP0), c->stream));
    CK(cudaMemcpyAsync(xs.data(), c->bufs[BUF_TMP0].p, xbytes, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    FILE *f = fopen(path, "wb");
    if (!f) return set_err(c, RECON_EINVAL, "cannot open %s for writing", path);
    int64_t hdr[4] = {c->model, c->N, c->M, nnz};
    bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(hdr, sizeof hdr, 1, f) == 1 &&
              fwrite(&c->opt, sizeof c->opt, 1, f) == 1 && fwrite(&s, sizeof s, 1, f) == 1 &&
              fwrite(&c->stats_calls, sizeof c->stats_calls, 1, f) == 1 &&
              fwrite(xs.data(), 1, xs.size(), f) == xs.size() &&
              fwrite(fields.data(), sizeof(float), c->N, f) == (size_t)c->N &&
              (nnz == 0 || (fwrite(ij.data(), sizeof(int32_t), 2 * nnz, f) == (size_t)(2 * nnz) &&
                            fwrite(w.data(), sizeof(float), nnz, f) == (size_t)nnz));
    for (auto &a : state_arrays(c)) {
        if (!ok) break;
        std::vector<float> hbuf(a.second);
        if (cudaMemcpy(hbuf.data(), a.first, sizeof(float) * a.second, cudaMemcpyDeviceToHost) != cudaSuccess) {
            fclose(f);
            return cuda_fail(c, cudaGetLastError(), "checkpoint read-back");
        }
        ok = fwrite(hbuf.data(), sizeof(float), a.second, f) == a.second;
    }
    ok = (fclose(f) == 0) && ok;
    if (!ok) return set_err(c, RECON_EINVAL, "write to %s failed", path);
    return RECON_OK;
}

extern "C" recon_status recon_load(recon_ctx **out, const char *path, void *stream) {
    if (!out || !path) return set_err(nullptr, RECON_EINVAL, "out or path is NULL");
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) return set_err(nullptr, RECON_EINVAL, "cannot open %s", path);
    char magic[8];
    int64_t hdr[4];
    recon_options o;
    recon_stats s;
    uint64_t calls = 0;
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kMagic, 8) == 0 && fread(hdr, sizeof hdr, 1, f) == 1 &&
              fread(&o, sizeof o, 1, f) == 1 && fread(&s, sizeof s, 1, f) == 1 &&
              fread(&calls, sizeof calls, 1, f) == 1;
    if (!ok || hdr[1] < 2 || hdr[2] < 1 || hdr[3] < 0 || (hdr[0] != RECON_ISING && hdr[0] != RECON_GAUSSIAN)) {
        fclose(f);
        return set_err(nullptr, RECON_EINVAL, "%s is not a checkpoint of this version", path);
    }
    const int model = (int)hdr[0];
    const int64_t N = hdr[1], M = hdr[2], nnz = hdr[3];
    std::vector<uint8_t> X((size_t)N * M * (model == RECON_ISING ? 1 : 4));
    std::vector<float> fields(N);
    std::vector<int32_t> ij(2 * std::max<int64_t>(nnz, 1));
    std::vector<float> w(std::max<int64_t>(nnz, 1));
    ok = fread(X.data(), 1, X.size(), f) == X.size() && fread(fields.data(), sizeof(float), N, f) == (size_t)N &&
         (nnz == 0 || (fread(ij.data(), sizeof(int32_t), 2 * nnz, f) == (size_t)(2 * nnz) &&
                       fread(w.data(), sizeof(float), nnz, f) == (size_t)nnz));
    if (!ok) {
        fclose(f);
        return set_err(nullptr, RECON_EINVAL, "%s is truncated", path);
    }
    // w_clamp was stored resolved; it is valid input as is
    recon_ctx *c = nullptr;
    recon_status st = recon_init(&c, X.data(), M, N, model == RECON_ISING ? RECON_X_INT8 : RECON_X_FP32, 0, model, &o,
                                 stream);
    if (st != RECON_OK) {
        fclose(f);
        return st;
    }
    st = recon_set_model(c, ij.data(), w.data(), nnz, fields.data());
    if (st != RECON_OK) {
        fclose(f);
        g_err = c->err;
        recon_destroy(c);
        return st;
    }
    // the tracked per-sample sums and per-node totals as saved, so that the run
    // continues bit for bit (rebuilt ones could differ in their last bits)
    for (auto &a : state_arrays(c)) {
        std::vector<float> hbuf(a.second);
        if (fread(hbuf.data(), sizeof(float), a.second, f) != a.second) {
            fclose(f);
            recon_destroy(c);
            return set_err(nullptr, RECON_EINVAL, "%s is truncated", path);
        }
        if (cudaMemcpy(a.first, hbuf.data(), sizeof(float) * a.second, cudaMemcpyHostToDevice) != cudaSuccess) {
            fclose(f);
            g_err = "checkpoint upload failed";
            recon_destroy(c);
            return RECON_ECUDA;
        }
    }
    fclose(f);
    CK(cudaMemcpyAsync(c->cnt + CNT_NEWTON, &s.newton_passes, sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->stats = s;
    c->stats_calls = calls;
    *out = c;
    return RECON_OK;
}

extern "C" const char *recon_last_error(const recon_ctx *c) { return c ? c->err.c_str() : g_err.c_str(); }

extern "C" void recon_destroy(recon_ctx *c) { free_ctx(c); }
