// prop_api.cu -- C ABI of the learned proposal (recon_proposal_*), and the
// learned seeding of NNDescent's initial lists.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "proposal.cuh"
#include "search.cuh"

#define CK(call)                                                \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);  \
    } while (0)

namespace {

__global__ void k_rand_pairs(int64_t n, int N, uint64_t seed, int32_t *out) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const uint64_t r = mix64(seed ^ mix64((uint64_t)q));
    int a = (int)(r % (uint64_t)N);
    int b = (int)((r >> 32) % (uint64_t)(N - 1));
    if (b >= a) ++b;
    out[2 * q] = a < b ? a : b;
    out[2 * q + 1] = a < b ? b : a;
}

// tau = sign(w*) sqrt(2 gain): tau^2 / 2 is the exact gain of the pair
__global__ void k_tau(int64_t n, const float *d, const float *w, float *tau) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float g = fmaxf(-d[q], 0.f);
    tau[q] = copysignf(sqrtf(2.f * g), w[q]) * (w[q] != 0.f ? 1.f : 0.f);
}

// |<e_i, e_j>| of sampled pairs
__global__ void k_absdot(int64_t n, const int32_t *pairs, const float *emb, float *out) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float *a = emb + (int64_t)pairs[2 * q] * PROP_EMBED, *b = emb + (int64_t)pairs[2 * q + 1] * PROP_EMBED;
    float s = 0.f;
    for (int c = 0; c < PROP_EMBED; ++c) s = fmaf(a[c], b[c], s);
    out[q] = fabsf(s);
}

// each seed pair offered to both its nodes, keyed by -|<e_i, e_j>|
__global__ void k_seed_offers(int64_t n, const int32_t *pairs, const float *emb, int32_t *ot, int32_t *ov, float *od) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int i = pairs[2 * q], j = pairs[2 * q + 1];
    const float *a = emb + (int64_t)i * PROP_EMBED, *b = emb + (int64_t)j * PROP_EMBED;
    float s = 0.f;
    for (int c = 0; c < PROP_EMBED; ++c) s = fmaf(a[c], b[c], s);
    ot[2 * q] = i;
    ov[2 * q] = j;
    od[2 * q] = -fabsf(s);
    ot[2 * q + 1] = j;
    ov[2 * q + 1] = i;
    od[2 * q + 1] = -fabsf(s);
}

__global__ void k_count(int64_t n, const int32_t *t, int32_t *cnt) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) atomicAdd(&cnt[t[q]], 1);
}
__global__ void k_widen(const int32_t *a, int64_t *b, int64_t n) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) b[e] = a[e];
}
__global__ void k_scatter(int64_t n, const int32_t *t, const int32_t *v, const float *d, const int64_t *off,
                          int32_t *cursor, int32_t *sv, float *sd) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int x = t[q];
    const int pos = atomicAdd(&cursor[x], 1);
    sv[off[x] + pos] = v[q];
    sd[off[x] + pos] = d[q];
}

// the best seeds of each node (smallest key, ties by id), at most smax[x] =
// round(frac klen[x]) of them, then distinct random ids != x up to klen[x];
// -1 in the rest of the capacity K
__global__ void k_seed_lists(int n, int K, const int32_t *klen, float frac, const int64_t *off, const int32_t *sv,
                             const float *sd, uint64_t seed, int32_t *ids, int *nseeded) {
    const int lane = threadIdx.x & 31;
    const int x = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (x >= n) return;
    int32_t *L = ids + (int64_t)x * K;
    const int k = klen[x];
    const int smax = min(k, max(1, __float2int_rn(frac * (float)k)));
    const int64_t b = off[x], cntx = off[x + 1] - off[x];
    float last_d = -INFINITY;
    int last_v = -1;
    int q = 0;
    for (; q < smax && q < cntx; ++q) {
        float best = INFINITY;
        int bv = 0x7fffffff;
        for (int64_t r = lane; r < cntx; r += 32) {
            const float dv = sd[b + r];
            const int vv = sv[b + r];
            const bool after = dv > last_d || (dv == last_d && vv > last_v);
            if (after && (dv < best || (dv == best && vv < bv))) {
                best = dv;
                bv = vv;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int ov = __shfl_xor_sync(0xffffffffu, bv, o);
            if (ob < best || (ob == best && ov < bv)) {
                best = ob;
                bv = ov;
            }
        }
        if (bv == 0x7fffffff) break;
        if (lane == 0) L[q] = bv;
        last_d = best;
        last_v = bv;
    }
    __syncwarp();
    for (int r = k + lane; r < K; r += 32) L[r] = -1;
    if (lane == 0) {
        if (q > 0) atomicAdd(nseeded, 1);
        uint64_t ctr = 0;
        // k <= n - 1, so the fallback scan always completes the list
        while (q < k) {
            const int y = (int)(mix64(seed ^ mix64(((uint64_t)x << 32) ^ ctr++)) % (uint64_t)n);
            bool dup = y == x;
            for (int p = 0; p < q && !dup; ++p) dup = L[p] == y;
            if (!dup) L[q++] = y;
            if (ctr > 64ull * k)
                for (int yy = 0; q < k && yy < n; ++yy) {
                    bool d2 = yy == x;
                    for (int p = 0; p < q && !d2; ++p) d2 = L[p] == yy;
                    if (!d2) L[q++] = yy;
                }
        }
    }
}

inline unsigned nbk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

cudaError_t grow(DBuf &b, size_t bytes, cudaStream_t st) {
    if (b.bytes >= bytes) return cudaSuccess;
    if (b.p) {
        cudaStreamSynchronize(st);
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    cudaError_t e = recon_malloc(&b.p, bytes + bytes / 4);
    if (e == cudaSuccess) b.bytes = bytes + bytes / 4;
    return e;
}

}  // namespace

static recon_status ensure_prop(recon_ctx *c, uint64_t seed) {
    if (c->model != RECON_ISING) return set_err(c, RECON_EUNSUPPORTED, "the learned proposal sketches spins (Ising)");
    if (!c->prop) {
        c->prop = new Proposal();
        c->prop->omega_seed = mix64(seed ^ 0x0de9a5eedull);
    }
    CK(proposal_setup(c, *c->prop, seed));
    return RECON_OK;
}

extern "C" int64_t recon_proposal_param_count(void) { return proposal_param_count(); }

extern "C" void recon_default_train_opts(recon_train_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->steps = 300;
    o->lr = 3e-3f;
    o->seed = 7;
    o->n_best = 0;
    o->n_random = 0;
}

extern "C" recon_status recon_proposal_weights(recon_ctx *c, float *get_out, const float *set_in, int64_t count) {
    if (!c) return set_err(nullptr, RECON_EINVAL, "null context");
    tl_ctx = c;
    if (c->broken) return set_err(c, RECON_ESTATE, "context unusable after an earlier error: %s", c->err.c_str());
    const int64_t np = proposal_param_count();
    if (count != np) return set_err(c, RECON_EINVAL, "count must be %lld", (long long)np);
    recon_status st = ensure_prop(c, 7);
    if (st != RECON_OK) return st;
    Proposal &P = *c->prop;
    if (set_in) {
        for (int64_t q = 0; q < np; ++q)
            if (!std::isfinite(set_in[q])) return set_err(c, RECON_EINVAL, "weight %lld is not finite", (long long)q);
        CK(cudaMemcpyAsync(P.w.p, set_in, sizeof(float) * np, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemsetAsync(P.m1.p, 0, sizeof(float) * np, c->stream));
        CK(cudaMemsetAsync(P.m2.p, 0, sizeof(float) * np, c->stream));
        P.t = 0;
        P.trained = true;  // given weights are taken as a trained proposal
        CK(proposal_setup(c, P, 7));  // refreshes the bf16 copies
    }
    if (get_out) CK(cudaMemcpyAsync(get_out, P.w.p, sizeof(float) * np, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return RECON_OK;
}

extern "C" recon_status recon_proposal_embed(recon_ctx *c, float *sketch_out, float *embed_out) {
    if (!c) return set_err(nullptr, RECON_EINVAL, "null context");
    tl_ctx = c;
    if (c->broken) return set_err(c, RECON_ESTATE, "context unusable after an earlier error: %s", c->err.c_str());
    recon_status st = ensure_prop(c, 7);
    if (st != RECON_OK) return st;
    Proposal &P = *c->prop;
    CK(proposal_forward(c, P, false));
    if (sketch_out)
        CK(cudaMemcpyAsync(sketch_out, P.sketch.p, sizeof(float) * c->N * PROP_SKETCH, cudaMemcpyDeviceToHost,
                           c->stream));
    if (embed_out)
        CK(cudaMemcpyAsync(embed_out, P.emb.p, sizeof(float) * c->N * PROP_EMBED, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return RECON_OK;
}

static recon_status upload_training(recon_ctx *c, const int32_t *pairs, const float *targets, int64_t n) {
    Proposal &P = *c->prop;
    CK(grow(P.tpairs, sizeof(int32_t) * 2 * n, c->stream));
    CK(grow(P.ttau, sizeof(float) * n, c->stream));
    for (int64_t q = 0; q < n; ++q) {
        const int a = pairs[2 * q], b = pairs[2 * q + 1];
        if (a < 0 || b < 0 || a >= c->N || b >= c->N || a == b)
            return set_err(c, RECON_EINVAL, "training pair %lld is not valid", (long long)q);
    }
    CK(cudaMemcpyAsync(P.tpairs.p, pairs, sizeof(int32_t) * 2 * n, cudaMemcpyHostToDevice, c->stream));
    if (targets) {
        CK(cudaMemcpyAsync(P.ttau.p, targets, sizeof(float) * n, cudaMemcpyHostToDevice, c->stream));
    } else {
        DBuf d, w;
        CK(grow(d, sizeof(float) * n, c->stream));
        CK(grow(w, sizeof(float) * n, c->stream));
        recon_status st = score_pairs_device(c, (int32_t *)P.tpairs.p, n, nullptr, (float *)d.p, (float *)w.p);
        if (st == RECON_OK) {
            k_tau<<<nbk(n), 256, 0, c->stream>>>(n, (float *)d.p, (float *)w.p, (float *)P.ttau.p);
            note_launch();
        }
        cudaStreamSynchronize(c->stream);
        cudaFree(d.p);
        cudaFree(w.p);
        if (st != RECON_OK) return st;
    }
    return RECON_OK;
}

extern "C" recon_status recon_proposal_grad(recon_ctx *c, const int32_t *pairs, const float *targets, int64_t n,
                                            float *grad_out, double *loss_out) {
    if (!c) return set_err(nullptr, RECON_EINVAL, "null context");
    tl_ctx = c;
    if (c->broken) return set_err(c, RECON_ESTATE, "context unusable after an earlier error: %s", c->err.c_str());
    if (n < 1 || !pairs || !targets) return set_err(c, RECON_EINVAL, "pairs and targets are required");
    recon_status st = ensure_prop(c, 7);
    if (st != RECON_OK) return st;
    st = upload_training(c, pairs, targets, n);
    if (st != RECON_OK) return st;
    Proposal &P = *c->prop;
    CK(grow(P.loss, sizeof(double) * 2, c->stream));
    CK(proposal_grad(c, P, (int32_t *)P.tpairs.p, (float *)P.ttau.p, n, (double *)P.loss.p));
    if (grad_out)
        CK(cudaMemcpyAsync(grad_out, P.g.p, sizeof(float) * proposal_param_count(), cudaMemcpyDeviceToHost, c->stream));
    double l = 0.0;
    CK(cudaMemcpyAsync(&l, P.loss.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (loss_out) *loss_out = l;
    return RECON_OK;
}

extern "C" recon_status recon_proposal_train(recon_ctx *c, const recon_train_opts *opts, float *loss_out) {
    if (!c) return set_err(nullptr, RECON_EINVAL, "null context");
    tl_ctx = c;
    if (c->broken) return set_err(c, RECON_ESTATE, "context unusable after an earlier error: %s", c->err.c_str());
    recon_train_opts o;
    recon_default_train_opts(&o);
    if (opts) o = *opts;
    if (o.steps < 0 || !(o.lr > 0.f)) return set_err(c, RECON_EINVAL, "steps >= 0 and lr > 0 are required");
    // the targets are exact gains whatever distance the search ranks by
    struct ExactScores {
        recon_ctx *c;
        bool was;
        ~ExactScores() { c->force_exact = was; }
    } exact_guard{c, c->force_exact};
    c->force_exact = true;
    recon_status st = ensure_prop(c, o.seed);
    if (st != RECON_OK) return st;
    Proposal &P = *c->prop;
    int64_t n = 0;
    if (o.pairs && o.n_pairs > 0) {
        st = upload_training(c, o.pairs, o.targets, o.n_pairs);
        if (st != RECON_OK) return st;
        n = o.n_pairs;
    } else {
        // sampled: the exact best pairs (tensor-core screen) and uniform random pairs
        const int64_t nb_ = o.n_best > 0 ? o.n_best : c->N;
        const int64_t nr = o.n_random > 0 ? o.n_random : 8 * c->N;
        int32_t *bp = nullptr;
        float *bd = nullptr;
        int64_t got = 0;
        st = screen_run(c, nb_, &bp, &bd, &got);
        if (st != RECON_OK) return st;
        n = got + nr;
        std::vector<int32_t> hp(2 * n);
        CK(cudaMemcpyAsync(hp.data(), bp, sizeof(int32_t) * 2 * got, cudaMemcpyDeviceToHost, c->stream));
        DBuf rp;
        CK(grow(rp, sizeof(int32_t) * 2 * nr, c->stream));
        k_rand_pairs<<<nbk(nr), 256, 0, c->stream>>>(nr, (int)c->N, mix64(o.seed ^ 0x7a1ull), (int32_t *)rp.p);
        note_launch();
        CK(cudaMemcpyAsync(hp.data() + 2 * got, rp.p, sizeof(int32_t) * 2 * nr, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        cudaFree(rp.p);
        st = upload_training(c, hp.data(), nullptr, n);
        if (st != RECON_OK) return st;
    }
    CK(grow(P.loss, sizeof(double) * (o.steps + 1), c->stream));
    for (int s = 0; s < o.steps; ++s) {
        if (!o.fixed_sketch) CK(proposal_resketch(c, P, mix64(P.omega_seed ^ mix64(0x51ce7c4ull + (uint64_t)P.t))));
        CK(proposal_grad(c, P, (int32_t *)P.tpairs.p, (float *)P.ttau.p, n, (double *)P.loss.p + s));
        CK(proposal_adam(c, P, o.lr));
    }
    if (!o.fixed_sketch) CK(proposal_resketch(c, P, P.omega_seed));  // the context's own sketches again
    if (loss_out && o.steps > 0) {
        std::vector<double> l(o.steps);
        CK(cudaMemcpyAsync(l.data(), P.loss.p, sizeof(double) * o.steps, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        for (int s = 0; s < o.steps; ++s) loss_out[s] = (float)l[s];
    }
    CK(cudaStreamSynchronize(c->stream));
    P.trained = true;
    return RECON_OK;
}

// Initial lists of the first FindBest level from the learned embedding: the
// seed pairs are those with |<e_i, e_j>| above a threshold picked so that the
// tensor-core pass keeps about 2 f k_i seeds per node (estimated from 2^14
// random pairs); each node takes at most f k_i of its best seeds and random ids
// for the rest (f = learned_frac), so that the search keeps exploring.
recon_status learned_seed_lists(recon_ctx *c, int n, int K, const int32_t *klen, uint64_t seed, int32_t *ids,
                                int64_t *nseeded_out) {
    Proposal &P = *c->prop;
    const float f = c->opt.learned_frac > 0.f ? c->opt.learned_frac : 0.5f;
    CK(proposal_forward(c, P, false));
    CK(grow(P.seedA, sizeof(uint16_t) * (size_t)c->N * 64, c->stream));
    CK(proposal_seed_operands(c, P, P.seedA.p));
    // threshold from a sample
    const int64_t ns = 1 << 14;
    CK(grow(P.s_pairs, sizeof(int32_t) * 2 * ns, c->stream));
    CK(grow(P.s_vals, sizeof(float) * ns, c->stream));
    k_rand_pairs<<<nbk(ns), 256, 0, c->stream>>>(ns, n, mix64(seed ^ 0x5a3d1eull), (int32_t *)P.s_pairs.p);
    note_launch();
    k_absdot<<<nbk(ns), 256, 0, c->stream>>>(ns, (int32_t *)P.s_pairs.p, (float *)P.emb.p, (float *)P.s_vals.p);
    note_launch();
    std::vector<float> hv(ns);
    CK(cudaMemcpyAsync(hv.data(), P.s_vals.p, sizeof(float) * ns, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const double npairs = (double)n * (n - 1) / 2.0;
    const double frac = std::min(1.0, (double)f * n * K / npairs);  // about 2 f k seeds per node
    int64_t rank = std::min<int64_t>(ns - 1, (int64_t)(frac * ns));
    std::nth_element(hv.begin(), hv.begin() + (ns - 1 - rank), hv.end());
    const float thr = frac >= 1.0 ? -1.f : hv[ns - 1 - rank];
    // seed pairs through the tensor-core pass (K = 64: 32 embedding dims and zeros)
    int64_t cap = std::max<int64_t>((int64_t)(4.0 * f * n * K) + 1024, 1 << 16);
    unsigned long long cnt = 0;
    for (int attempt = 0; attempt < 3; ++attempt) {
        CK(grow(P.s_cands, sizeof(int32_t) * 2 * cap, c->stream));
        CK(cudaMemsetAsync(c->cnt + CNT_SCRATCH3, 0, sizeof(unsigned long long), c->stream));
        CK(launch_screen_ex(c, P.seedA.p, P.seedA.p, 64, thr, nullptr, 0.f, 0, false, (int32_t *)P.s_cands.p, cap,
                            c->cnt + CNT_SCRATCH3, nullptr, false, 0.f, 64, nullptr, false));
        CK(cudaMemcpyAsync(c->cnt_host + CNT_SCRATCH3, c->cnt + CNT_SCRATCH3, sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        cnt = c->cnt_host[CNT_SCRATCH3];
        if ((int64_t)cnt <= cap) break;
        cap = (int64_t)cnt + (int64_t)cnt / 4 + 1024;
    }
    const int64_t ne = 2 * (int64_t)std::min<unsigned long long>(cnt, (unsigned long long)cap);
    for (DBuf *b : {&P.s_ot, &P.s_ov, &P.s_sv}) CK(grow(*b, sizeof(int32_t) * (ne + 1), c->stream));
    for (DBuf *b : {&P.s_od, &P.s_sd}) CK(grow(*b, sizeof(float) * (ne + 1), c->stream));
    for (DBuf *b : {&P.s_cnt, &P.s_cur}) CK(grow(*b, sizeof(int32_t) * (n + 1), c->stream));
    for (DBuf *b : {&P.s_offw, &P.s_off}) CK(grow(*b, sizeof(int64_t) * (n + 1), c->stream));
    CK(grow(P.s_tmp, sizeof(int64_t) * scan_tmp_elems(n + 1), c->stream));
    int32_t *ot = (int32_t *)P.s_ot.p, *ov = (int32_t *)P.s_ov.p, *cntv = (int32_t *)P.s_cnt.p;
    float *od = (float *)P.s_od.p;
    int64_t *off = (int64_t *)P.s_off.p;
    if (ne) {
        k_seed_offers<<<nbk(ne / 2), 256, 0, c->stream>>>(ne / 2, (int32_t *)P.s_cands.p, (float *)P.emb.p, ot, ov, od);
        note_launch();
    }
    CK(cudaMemsetAsync(cntv, 0, sizeof(int32_t) * (n + 1), c->stream));
    CK(cudaMemsetAsync(P.s_cur.p, 0, sizeof(int32_t) * (n + 1), c->stream));
    if (ne) {
        k_count<<<nbk(ne), 256, 0, c->stream>>>(ne, ot, cntv);
        note_launch();
    }
    k_widen<<<nbk(n + 1), 256, 0, c->stream>>>(cntv, (int64_t *)P.s_offw.p, n + 1);
    note_launch();
    CK(launch_scan_i64((int64_t *)P.s_offw.p, off, n + 1, (int64_t *)P.s_tmp.p, c->stream));
    if (ne) {
        k_scatter<<<nbk(ne), 256, 0, c->stream>>>(ne, ot, ov, od, off, (int32_t *)P.s_cur.p, (int32_t *)P.s_sv.p,
                                                  (float *)P.s_sd.p);
        note_launch();
    }
    CK(cudaMemsetAsync(c->cnt + CNT_SCRATCH3, 0, sizeof(unsigned long long), c->stream));
    k_seed_lists<<<nbk((int64_t)n * 32), 256, 0, c->stream>>>(n, K, klen, f, off, (int32_t *)P.s_sv.p,
                                                               (float *)P.s_sd.p, seed, ids,
                                                               (int *)(c->cnt + CNT_SCRATCH3));
    note_launch();
    int nseeded = 0;
    CK(cudaMemcpyAsync(&nseeded, c->cnt + CNT_SCRATCH3, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (nseeded_out) *nseeded_out = nseeded;
    return RECON_OK;
}
