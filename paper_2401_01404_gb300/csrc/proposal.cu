// proposal.cu -- the learned proposal: a small MLP that maps each node's
// random-projection sketch of its samples to an embedding whose large
// |<e_i, e_j>| point at pairs with large gains; the best of those seed the
// initial NNDescent lists in place of random ones (Algorithm 4 draws them at
// random; random seeding remains the default).  It only proposes: every seeded
// pair is scored exactly before it can enter a list.
//
//   sketch  s_i = Omega^T x_i / sqrt(M), Omega in {-1,+1}^{M x 64} drawn from a
//           SplitMix64 stream (bit = top bit of mix64(seed + 2^32 c + m)); with
//           x and Omega as bits, s_ic = (M - 2 popcount(x_i xor omega_c)) / sqrt(M)
//   MLP     a_i = W1 s_i + b1 (128), h_i = relu(a_i), e_i = W2 h_i + b2 (32);
//           weights are kept in FP32 and used in BF16, accumulation in FP32
//   target  tau_ij = sign(w*_ij) sqrt(2 gain_ij), from the exact scorer (so that
//           tau^2/2 is the gain), and the loss is mean_(i,j) (<e_i, e_j> - tau_ij)^2
//   training: full-batch Adam over the given pairs, gradients by hand-written
//           backward kernels (a per-node pass for the hidden-layer gradient,
//           then the weight gradients as sums of outer products over nodes,
//           accumulated in registers per block).  Omega is drawn afresh at every
//           step unless asked otherwise: with a fixed Omega the network can learn
//           the nodes of its training data from their sketches (and carries
//           nothing to other data); with a new Omega per step only a function of
//           the sketches' similarity lowers the loss, and it holds for any Omega
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "proposal.cuh"

namespace {

constexpr int S = PROP_SKETCH, H = PROP_HIDDEN, E = PROP_EMBED;

inline unsigned nb(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

// Omega bits: word [c * Mw + w], bit l = sample 32 w + l; padding bits are 0
__global__ void k_omega(int M, int Mw, uint64_t seed, uint32_t *ob) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)S * Mw) return;
    const int c = (int)(e / Mw), w = (int)(e % Mw);
    uint32_t word = 0;
    for (int l = 0; l < 32; ++l) {
        const int m = 32 * w + l;
        if (m < M && (mix64(seed + ((uint64_t)c << 32) + (uint64_t)m) >> 63)) word |= 1u << l;
    }
    ob[e] = word;
}

// s_ic = (M - 2 popcount(x_i xor omega_c)) / sqrt(M); padding bits agree (both 0)
// and count as agreements, so they are removed from M's count exactly
__global__ void k_sketch(IsingView v, const uint32_t *ob, float *sk) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)v.N * S) return;
    const int64_t i = e / S;
    const int c = (int)(e % S);
    int dis = 0;
    for (int w = 0; w < v.Mw; ++w) dis += __popc(v.xbits[i * v.Mw + w] ^ ob[(int64_t)c * v.Mw + w]);
    sk[e] = (float)(v.M - 2 * dis) * rsqrtf((float)v.M);
}

// forward for every node: one warp per node, weights (bf16) in shared memory;
// lane l owns hidden units l, l+32, l+64, l+96 and embedding dimension l
__global__ void __launch_bounds__(256) k_fwd(int N, const float *sk, const __nv_bfloat16 *W1, const float *b1,
                                             const __nv_bfloat16 *W2, const float *b2, float *a_out, float *e_out) {
    __shared__ __nv_bfloat16 sW1[H * S];
    __shared__ __nv_bfloat16 sW2[E * H];
    __shared__ float sb1[H], sb2[E];
    for (int q = threadIdx.x; q < H * S; q += blockDim.x) sW1[q] = W1[q];
    for (int q = threadIdx.x; q < E * H; q += blockDim.x) sW2[q] = W2[q];
    for (int q = threadIdx.x; q < H; q += blockDim.x) sb1[q] = b1[q];
    for (int q = threadIdx.x; q < E; q += blockDim.x) sb2[q] = b2[q];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < N; i += nw) {
        const float s0 = sk[i * S + lane], s1 = sk[i * S + 32 + lane];
        float a[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = sb1[lane + 32 * r];
#pragma unroll 8
        for (int k = 0; k < S; ++k) {
            const float sv = __shfl_sync(0xffffffffu, k < 32 ? s0 : s1, k & 31);
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = fmaf(__bfloat162float(sW1[(lane + 32 * r) * S + k]), sv, a[r]);
        }
        float e = sb2[lane];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float hr = fmaxf(a[r], 0.f);
            for (int src = 0; src < 32; ++src) {
                const float hv = __shfl_sync(0xffffffffu, hr, src);
                e = fmaf(__bfloat162float(sW2[lane * H + src + 32 * r]), hv, e);
            }
            if (a_out) a_out[i * H + lane + 32 * r] = a[r];
        }
        e_out[i * E + lane] = e;
    }
}

// loss and embedding gradients of the pairs: one warp per pair, lane = dimension
__global__ void k_pair_grad(int64_t P, const int32_t *pairs, const float *tau, const float *emb, float scale,
                            float *de, double *loss) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double l = 0.0;
    for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < P; q += nw) {
        const int i = pairs[2 * q], j = pairs[2 * q + 1];
        const float ei = emb[(int64_t)i * E + lane], ej = emb[(int64_t)j * E + lane];
        const float p = warp_sum(ei * ej);
        const float r = p - tau[q];
        const float dp = 2.f * r * scale;
        atomicAdd(&de[(int64_t)i * E + lane], dp * ej);
        atomicAdd(&de[(int64_t)j * E + lane], dp * ei);
        if (lane == 0) l += (double)r * r * scale;
    }
    if (lane == 0 && l != 0.0) atomicAdd(loss, l);
}

// backward through the second layer, per node: dA_i = (W2^T de_i) * [a_i > 0]
// (one warp per node; lane l holds de_il and hidden units l + 32 r)
__global__ void __launch_bounds__(256) k_bwd_nodes(int N, const float *act, const float *de,
                                                   const __nv_bfloat16 *W2, float *dA) {
    __shared__ __nv_bfloat16 sW2[E * H];
    for (int q = threadIdx.x; q < E * H; q += blockDim.x) sW2[q] = W2[q];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < N; i += nw) {
        const float dei = de[i * E + lane];
        float dh[4] = {0.f, 0.f, 0.f, 0.f};
        for (int l = 0; l < 32; ++l) {
            const float del = __shfl_sync(0xffffffffu, dei, l);
#pragma unroll
            for (int r = 0; r < 4; ++r) dh[r] = fmaf(__bfloat162float(sW2[l * H + lane + 32 * r]), del, dh[r]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int h = lane + 32 * r;
            dA[i * H + h] = act[i * H + h] > 0.f ? dh[r] : 0.f;
        }
    }
}

// out[p][q] += sum_i X[i][p] f(Y[i][q]) for a small P x Q output (f = relu when
// relu_y): the weight gradients dW1 = dA^T S and dW2 = dE^T relu(A), and with
// Y = 1 (ones != 0) the bias gradients.  Each block sums a slice of rows in
// registers (thread t owns outputs t, t + 256, ...) and adds once per output.
template <int P, int Q>
__global__ void __launch_bounds__(256) k_outer(int N, const float *X, const float *Y, bool relu_y, bool ones,
                                               float *out, float *bias_out) {
    constexpr int R = 16;  // rows staged per round
    __shared__ float sx[R][P], sy[R][Q];
    constexpr int PER = (P * Q + 255) / 256;
    float acc[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) acc[u] = 0.f;
    float bacc = 0.f;
    const int64_t rows_per_block = ((int64_t)N + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block, r1 = min((int64_t)N, r0 + rows_per_block);
    for (int64_t base = r0; base < r1; base += R) {
        for (int q = threadIdx.x; q < R * P; q += blockDim.x) {
            const int64_t i = base + q / P;
            sx[q / P][q % P] = i < r1 ? X[i * P + q % P] : 0.f;
        }
        if (!ones)
            for (int q = threadIdx.x; q < R * Q; q += blockDim.x) {
                const int64_t i = base + q / Q;
                float y = i < r1 ? Y[i * Q + q % Q] : 0.f;
                sy[q / Q][q % Q] = relu_y ? fmaxf(y, 0.f) : y;
            }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int o = threadIdx.x + 256 * u;
            if (o < P * Q) {
                const int pp = o / Q, qq = o % Q;
                for (int rr = 0; rr < R; ++rr) acc[u] = fmaf(sx[rr][pp], ones ? 1.f : sy[rr][qq], acc[u]);
            }
        }
        if (bias_out && threadIdx.x < P)
            for (int rr = 0; rr < R; ++rr) bacc += sx[rr][threadIdx.x];
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int o = threadIdx.x + 256 * u;
        if (o < P * Q && acc[u] != 0.f) atomicAdd(&out[o], acc[u]);
    }
    if (bias_out && threadIdx.x < P && bacc != 0.f) atomicAdd(&bias_out[threadIdx.x], bacc);
}

// Adam (Kingma and Ba, 2015) on the FP32 parameters, refreshing their BF16 copies
__global__ void k_adam(int n, float *w, const float *g, float *m1, float *m2, float lr, float b1c, float b2c,
                       __nv_bfloat16 *wb, int nb1, __nv_bfloat16 *wb2, int off2, int nw2) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
    m1[q] = beta1 * m1[q] + (1.f - beta1) * g[q];
    m2[q] = beta2 * m2[q] + (1.f - beta2) * g[q] * g[q];
    w[q] -= lr * (m1[q] / b1c) / (sqrtf(m2[q] / b2c) + eps);
    if (q < nb1) wb[q] = __float2bfloat16_rn(w[q]);
    if (q >= off2 && q < off2 + nw2) wb2[q - off2] = __float2bfloat16_rn(w[q]);
}

__global__ void k_to_bf16(int n, const float *w, __nv_bfloat16 *wb) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) wb[q] = __float2bfloat16_rn(w[q]);
}

// seed operands: rows [e_i | 0] and [e_i | 0] as bf16 over K = 64
__global__ void k_seed_prep(int N, const float *emb, __nv_bfloat16 *A) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)N * 64) return;
    const int64_t i = q / 64;
    const int c = (int)(q % 64);
    A[q] = __float2bfloat16_rn(c < E ? emb[i * E + c] : 0.f);
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

// parameter block layout (floats): W1 [H x S] | b1 [H] | W2 [E x H] | b2 [E]
int64_t proposal_param_count() { return (int64_t)H * S + H + (int64_t)E * H + E; }

static cudaError_t ensure(DBuf &b, size_t bytes, cudaStream_t st) {
    if (b.bytes >= bytes) return cudaSuccess;
    if (b.p) {
        cudaStreamSynchronize(st);
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    cudaError_t e = recon_malloc(&b.p, bytes);
    if (e == cudaSuccess) b.bytes = bytes;
    return e;
}

cudaError_t proposal_setup(recon_ctx *c, Proposal &P, uint64_t seed) {
    cudaStream_t st = c->stream;
    const int64_t np = proposal_param_count();
    cudaError_t e;
    if ((e = ensure(P.w, sizeof(float) * np, st)) || (e = ensure(P.m1, sizeof(float) * np, st)) ||
        (e = ensure(P.m2, sizeof(float) * np, st)) || (e = ensure(P.g, sizeof(float) * np, st)) ||
        (e = ensure(P.w1b, sizeof(__nv_bfloat16) * H * S, st)) || (e = ensure(P.w2b, sizeof(__nv_bfloat16) * E * H, st)) ||
        (e = ensure(P.omega, sizeof(uint32_t) * S * c->Mw, st)) || (e = ensure(P.sketch, sizeof(float) * c->N * S, st)) ||
        (e = ensure(P.emb, sizeof(float) * c->N * E, st)) || (e = ensure(P.act, sizeof(float) * c->N * H, st)) ||
        (e = ensure(P.de, sizeof(float) * c->N * E, st)))
        return e;
    if (!P.ready) {
        // He-style initialisation from the seed (host, deterministic)
        std::vector<float> w(np);
        uint64_t ctr = 0;
        auto unif = [&]() { return (double)(mix64(seed ^ mix64(0xabcdefull + ctr++)) >> 11) * (1.0 / 9007199254740992.0); };
        auto gauss = [&]() {
            double u1 = unif(), u2 = unif();
            return std::sqrt(-2.0 * std::log(u1 + 1e-300)) * std::cos(6.283185307179586 * u2);
        };
        int64_t q = 0;
        for (int64_t t = 0; t < (int64_t)H * S; ++t) w[q++] = (float)(gauss() * std::sqrt(2.0 / S));
        for (int64_t t = 0; t < H; ++t) w[q++] = 0.f;
        for (int64_t t = 0; t < (int64_t)E * H; ++t) w[q++] = (float)(gauss() * std::sqrt(1.0 / H));
        for (int64_t t = 0; t < E; ++t) w[q++] = 0.f;
        if ((e = cudaMemcpyAsync(P.w.p, w.data(), sizeof(float) * np, cudaMemcpyHostToDevice, st))) return e;
        if ((e = cudaMemsetAsync(P.m1.p, 0, sizeof(float) * np, st)) || (e = cudaMemsetAsync(P.m2.p, 0, sizeof(float) * np, st)))
            return e;
        P.t = 0;
        if ((e = cudaStreamSynchronize(st))) return e;
        P.ready = true;
    }
    // refresh bf16 copies, Omega and the sketch
    k_to_bf16<<<nb(H * S), 256, 0, st>>>(H * S, (float *)P.w.p, (__nv_bfloat16 *)P.w1b.p);
    note_launch();
    k_to_bf16<<<nb(E * H), 256, 0, st>>>(E * H, (float *)P.w.p + H * S + H, (__nv_bfloat16 *)P.w2b.p);
    note_launch();
    k_omega<<<nb((int64_t)S * c->Mw), 256, 0, st>>>((int)c->M, (int)c->Mw, P.omega_seed, (uint32_t *)P.omega.p);
    note_launch();
    k_sketch<<<nb(c->N * S), 256, 0, st>>>(c->iv(), (uint32_t *)P.omega.p, (float *)P.sketch.p);
    note_launch();
    return cudaGetLastError();
}

// Omega drawn from `seed` and the sketches recomputed with it (training redraws
// Omega at every step; the context's own Omega comes from P.omega_seed)
cudaError_t proposal_resketch(recon_ctx *c, Proposal &P, uint64_t seed) {
    cudaStream_t st = c->stream;
    k_omega<<<nb((int64_t)S * c->Mw), 256, 0, st>>>((int)c->M, (int)c->Mw, seed, (uint32_t *)P.omega.p);
    note_launch();
    k_sketch<<<nb(c->N * S), 256, 0, st>>>(c->iv(), (uint32_t *)P.omega.p, (float *)P.sketch.p);
    note_launch();
    return cudaGetLastError();
}

cudaError_t proposal_forward(recon_ctx *c, Proposal &P, bool keep_act) {
    const float *w = (float *)P.w.p;
    const int64_t warps = c->N;
    const unsigned grid = (unsigned)std::min<int64_t>((warps * 32 + 255) / 256, 4096);
    k_fwd<<<grid, 256, 0, c->stream>>>((int)c->N, (float *)P.sketch.p, (__nv_bfloat16 *)P.w1b.p, w + H * S,
                                       (__nv_bfloat16 *)P.w2b.p, w + H * S + H + E * H,
                                       keep_act ? (float *)P.act.p : nullptr, (float *)P.emb.p);
    note_launch();
    return cudaGetLastError();
}

// loss and parameter gradient (into P.g) of the given device pairs / targets
cudaError_t proposal_grad(recon_ctx *c, Proposal &P, const int32_t *pairs, const float *tau, int64_t n,
                          double *loss_dev) {
    cudaStream_t st = c->stream;
    const int64_t np = proposal_param_count();
    cudaError_t e = proposal_forward(c, P, true);
    if (e) return e;
    if ((e = cudaMemsetAsync(P.de.p, 0, sizeof(float) * c->N * E, st)) ||
        (e = cudaMemsetAsync(P.g.p, 0, sizeof(float) * np, st)) || (e = cudaMemsetAsync(loss_dev, 0, sizeof(double), st)))
        return e;
    const unsigned gp = (unsigned)std::min<int64_t>((n * 32 + 255) / 256, 8192);
    k_pair_grad<<<gp, 256, 0, st>>>(n, pairs, tau, (float *)P.emb.p, 1.f / (float)std::max<int64_t>(n, 1),
                                     (float *)P.de.p, loss_dev);
    note_launch();
    float *g = (float *)P.g.p;
    if ((e = ensure(P.dA, sizeof(float) * c->N * H, st))) return e;
    const unsigned gn = (unsigned)std::min<int64_t>((c->N * 32 + 255) / 256, 4096);
    k_bwd_nodes<<<gn, 256, 0, st>>>((int)c->N, (float *)P.act.p, (float *)P.de.p, (__nv_bfloat16 *)P.w2b.p,
                                    (float *)P.dA.p);
    note_launch();
    const unsigned go = (unsigned)std::max<int64_t>(1, std::min<int64_t>(4 * c->num_sms, (c->N + 63) / 64));
    // dW1 = dA^T S and db1 = sum dA
    k_outer<H, S><<<go, 256, 0, st>>>((int)c->N, (float *)P.dA.p, (float *)P.sketch.p, false, false, g, g + H * S);
    note_launch();
    // dW2 = dE^T relu(A) and db2 = sum dE
    k_outer<E, H><<<go, 256, 0, st>>>((int)c->N, (float *)P.de.p, (float *)P.act.p, true, false, g + H * S + H,
                                      g + H * S + H + E * H);
    note_launch();
    return cudaGetLastError();
}

cudaError_t proposal_adam(recon_ctx *c, Proposal &P, float lr) {
    const int64_t np = proposal_param_count();
    P.t += 1;
    const float b1c = 1.f - std::pow(0.9f, (float)P.t), b2c = 1.f - std::pow(0.999f, (float)P.t);
    k_adam<<<nb(np), 256, 0, c->stream>>>((int)np, (float *)P.w.p, (float *)P.g.p, (float *)P.m1.p, (float *)P.m2.p,
                                          lr, b1c, b2c, (__nv_bfloat16 *)P.w1b.p, H * S, (__nv_bfloat16 *)P.w2b.p,
                                          H * S + H, E * H);
    note_launch();
    return cudaGetLastError();
}

cudaError_t proposal_seed_operands(recon_ctx *c, Proposal &P, void *A) {
    k_seed_prep<<<nb(c->N * 64), 256, 0, c->stream>>>((int)c->N, (float *)P.emb.p, (__nv_bfloat16 *)A);
    note_launch();
    return cudaGetLastError();
}

void free_proposal(Proposal *P) {
    if (!P) return;
    for (DBuf *b : {&P->w, &P->m1, &P->m2, &P->g, &P->w1b, &P->w2b, &P->omega, &P->sketch, &P->emb, &P->act, &P->de,
                    &P->dA, &P->tpairs, &P->ttau, &P->loss, &P->seedA, &P->s_pairs, &P->s_vals, &P->s_cands,
                    &P->s_ot, &P->s_ov, &P->s_od, &P->s_cnt, &P->s_offw, &P->s_off, &P->s_cur, &P->s_sv, &P->s_sd,
                    &P->s_tmp})
        if (b->p) cudaFree(b->p);
    delete P;
}
