// ising.cu -- Ising pseudo-likelihood kernels (App. A of arXiv:2401.01404).
//
// The pair problem.  Moving W_ij by delta shifts phi_i by delta*x_j and phi_j
// by delta*x_i in every sample.  With x = +-1 and tau = tanh(delta),
//     log cosh(phi + delta x) = log cosh(phi) + log cosh(delta) + log(1 + x tanh(phi) tau),
// so the change of the log pseudo-likelihood is a sum over samples of terms in
// u = x_j t_i and v = x_i t_j (t = tanh phi):
//     F(delta)  = sum_m [2 delta x_i x_j - 2 log cosh delta - log(1+tau u) - log(1+tau v)]
//     F'(delta) = 2 sum x_i x_j - sum [(u+tau)/(1+tau u) + (v+tau)/(1+tau v)]
//    -F''(delta)= (1 - tau^2) sum [(1-u^2)/(1+tau u)^2 + (1-v^2)/(1+tau v)^2]   (> 0)
// The gain of the best update under the Laplace prior (App. A) is
//     max_w F(w - W_ij) - lambda |w| + lambda |W_ij|,
// a concave 1-D problem: w = 0 when |F'(-W_ij)| <= lambda, otherwise the root
// of F'(w - W_ij) = lambda sign(w), found by Newton's method safeguarded by a
// bracket.  F is evaluated as delta*F'(0) plus per-sample remainders that are
// O(delta^2), never as a difference of two large sums.
//
// Thread mapping: lane l of a warp holds samples 32c + l.  The pair scorer
// (k_score) gives each pair a warp with both rows in registers (up to 1024
// samples; longer rows are re-read from L1/L2 on every pass).  The segmented
// scorer (k_score_seg) gives each node's candidate list a block: row i in shared
// memory, candidate rows brought into per-warp shared-memory stages by bulk
// asynchronous copies.  A wide matching batch of updates (k_update_blk) gives
// each pair a block whose warps split the samples (BlockRows); runs of thin
// batches (k_update_rounds) give each pair a warp.
#include "common.cuh"

namespace {

constexpr int MAX_NEWTON = 40;

// -------- row sources ------------------------------------------------------

// Sums over a pair's samples: a row source whose words one warp holds reduces
// with warp shuffles (BlockRows, whose words the warps of a block share,
// reduces across the block).
#define WARP_SUMS                                                                    \
    __device__ __forceinline__ float sum(float a) const { return warp_sum(a); }      \
    __device__ __forceinline__ void sum2(float &a, float &b) const {                 \
        a = warp_sum(a);                                                             \
        b = warp_sum(b);                                                             \
    }                                                                                \
    __device__ __forceinline__ void sum3(float &a, float &b, float &c) const {       \
        a = warp_sum(a);                                                             \
        b = warp_sum(b);                                                             \
        c = warp_sum(c);                                                             \
    }

template <int NW>
struct RegRows {  // both rows in registers (NW words of 32 samples)
    static constexpr int kNW = NW;
    WARP_SUMS
    float ti[NW], tj[NW];
    uint32_t pi, pj;  // bit c: x = -1 at sample 32c + lane
    int Mw;
    // coherent = true reads t with plain loads: rows that an earlier batch of
    // the same launch may have written (the read-only path could be stale)
    template <bool coherent = false>
    __device__ __forceinline__ void load(const IsingView &v, int i, int j, int lane) {
        Mw = v.Mw;
        const float *Ti = v.t + (int64_t)i * v.Mp, *Tj = v.t + (int64_t)j * v.Mp;
        const uint32_t *Bi = v.xbits + (int64_t)i * v.Mw, *Bj = v.xbits + (int64_t)j * v.Mw;
        pi = pj = 0u;
#pragma unroll
        for (int c = 0; c < NW; ++c) {
            if (c < Mw) {
                ti[c] = coherent ? Ti[32 * c + lane] : __ldg(Ti + 32 * c + lane);
                tj[c] = coherent ? Tj[32 * c + lane] : __ldg(Tj + 32 * c + lane);
                pi |= ((__ldg(Bi + c) >> lane) & 1u) << c;
                pj |= ((__ldg(Bj + c) >> lane) & 1u) << c;
            } else {
                ti[c] = tj[c] = 1.f;
            }
        }
    }
    __device__ __forceinline__ void get(int c, float &a, float &b, uint32_t &sa, uint32_t &sb) const {
        a = ti[c];
        b = tj[c];
        sa = (pi << (31 - c)) & 0x80000000u;
        sb = (pj << (31 - c)) & 0x80000000u;
    }
};

// Both rows over the warps of a block: warp w holds words w NWW .. w NWW + NWW - 1
// of each row in registers (lane l: sample 32 c + l); sums reduce across the
// block through shared memory, in two alternating scratch rows so that one
// barrier per reduction suffices.  Every warp takes part in every reduction.
template <int NWW>
struct BlockRows {
    static constexpr int kNW = NWW;
    float ti[NWW], tj[NWW];
    uint32_t pi, pj;  // bit c: x = -1 at sample 32 (w0 + c) + lane
    int Mw;           // this warp's words, 0 .. NWW
    int w0;           // its first word
    float *red;       // 2 x 3 x nw floats of shared scratch
    int nw, warp, lane;
    mutable int phase;
    __device__ __forceinline__ void setup(float *scratch) {
        red = scratch;
        nw = blockDim.x >> 5;
        warp = threadIdx.x >> 5;
        lane = threadIdx.x & 31;
        phase = 0;
    }
    template <bool coherent = false>
    __device__ __forceinline__ void load(const IsingView &v, int i, int j, int) {
        w0 = warp * NWW;
        Mw = max(0, min(NWW, v.Mw - w0));
        const float *Ti = v.t + (int64_t)i * v.Mp, *Tj = v.t + (int64_t)j * v.Mp;
        const uint32_t *Bi = v.xbits + (int64_t)i * v.Mw, *Bj = v.xbits + (int64_t)j * v.Mw;
        pi = pj = 0u;
#pragma unroll
        for (int c = 0; c < NWW; ++c) {
            if (c < Mw) {
                const int g = w0 + c;
                ti[c] = coherent ? Ti[32 * g + lane] : __ldg(Ti + 32 * g + lane);
                tj[c] = coherent ? Tj[32 * g + lane] : __ldg(Tj + 32 * g + lane);
                pi |= ((__ldg(Bi + g) >> lane) & 1u) << c;
                pj |= ((__ldg(Bj + g) >> lane) & 1u) << c;
            } else {
                ti[c] = tj[c] = 1.f;
            }
        }
    }
    __device__ __forceinline__ void get(int c, float &a, float &b, uint32_t &sa, uint32_t &sb) const {
        a = ti[c];
        b = tj[c];
        sa = (pi << (31 - c)) & 0x80000000u;
        sb = (pj << (31 - c)) & 0x80000000u;
    }
    __device__ __forceinline__ void sum3(float &a, float &b, float &c) const {
        a = warp_sum(a);
        b = warp_sum(b);
        c = warp_sum(c);
        float *r = red + (phase & 1) * 3 * nw;
        ++phase;
        if (lane == 0) {
            r[warp] = a;
            r[nw + warp] = b;
            r[2 * nw + warp] = c;
        }
        __syncthreads();
        a = b = c = 0.f;
        for (int w = 0; w < nw; ++w) {
            a += r[w];
            b += r[nw + w];
            c += r[2 * nw + w];
        }
    }
    __device__ __forceinline__ void sum2(float &a, float &b) const {
        float z = 0.f;
        sum3(a, b, z);
    }
    __device__ __forceinline__ float sum(float a) const {
        float y = 0.f, z = 0.f;
        sum3(a, y, z);
        return a;
    }
};

struct GlobRows {  // rows re-read every pass
    static constexpr int kNW = 0;
    WARP_SUMS
    const float *Ti, *Tj;
    const uint32_t *Bi, *Bj;
    int Mw, lane;
    bool coh;  // plain loads of t (rows written earlier in the same launch)
    template <bool coherent = false>
    __device__ __forceinline__ void load(const IsingView &v, int i, int j, int l) {
        Mw = v.Mw;
        lane = l;
        coh = coherent;
        Ti = v.t + (int64_t)i * v.Mp;
        Tj = v.t + (int64_t)j * v.Mp;
        Bi = v.xbits + (int64_t)i * v.Mw;
        Bj = v.xbits + (int64_t)j * v.Mw;
    }
    __device__ __forceinline__ void get(int c, float &a, float &b, uint32_t &sa, uint32_t &sb) const {
        a = coh ? Ti[32 * c + lane] : __ldg(Ti + 32 * c + lane);
        b = coh ? Tj[32 * c + lane] : __ldg(Tj + 32 * c + lane);
        sa = (__ldg(Bi + c) << (31 - lane)) & 0x80000000u;
        sb = (__ldg(Bj + c) << (31 - lane)) & 0x80000000u;
    }
};

template <class RS, class F>
__device__ __forceinline__ void for_words(const RS &R, F &&body) {
    if constexpr (RS::kNW > 0) {
#pragma unroll
        for (int c = 0; c < RS::kNW; ++c)
            if (c < R.Mw) body(c);
    } else {
        for (int c = 0; c < R.Mw; ++c) body(c);
    }
}

__device__ __forceinline__ float flip(float t, uint32_t s) { return __uint_as_float(__float_as_uint(t) ^ s); }

// log cosh(d) without cancellation at either end
__device__ __forceinline__ float logcosh_f(float d) {
    float a = fabsf(d);
    if (a < 0.5f) {
        float tt = tanhf(a);
        return -0.5f * log1pf(-tt * tt);
    }
    return a - 0.693147180559945309f + log1pf(expf(-2.f * a));
}

// pass at delta = 0: sum u, sum v, and the count of disagreeing spins
template <class RS>
__device__ __forceinline__ void pass0(const RS &R, float &su, float &sv, int &dis) {
    float a = 0.f, b = 0.f;
    int d = 0;
    for_words(R, [&](int c) {
        float ti, tj;
        uint32_t si, sj;
        R.get(c, ti, tj, si, sj);
        a += flip(ti, sj);
        b += flip(tj, si);
        d += (int)((si ^ sj) >> 31);
    });
    float df = (float)d;  // exact: at most 1024 samples
    R.sum3(a, b, df);
    su = a;
    sv = b;
    dis = (int)df;
}

// d1 = sum [(u+tau)/(1+tau u) + (v+tau)/(1+tau v)], d2 = sum [(1-u^2)/(1+tau u)^2 + ...]
template <class RS>
__device__ __forceinline__ void pass_newton(const RS &R, float tau, float &d1, float &d2) {
    float a1 = 0.f, a2 = 0.f;
    for_words(R, [&](int c) {
        float ti, tj;
        uint32_t si, sj;
        R.get(c, ti, tj, si, sj);
        float u = flip(ti, sj), v = flip(tj, si);
        float ru = rcp_approx(fmaf(tau, u, 1.f));
        float rv = rcp_approx(fmaf(tau, v, 1.f));
        a1 = fmaf(u + tau, ru, a1);
        a1 = fmaf(v + tau, rv, a1);
        a2 = fmaf(fmaf(-u, u, 1.f), ru * ru, a2);
        a2 = fmaf(fmaf(-v, v, 1.f), rv * rv, a2);
    });
    R.sum2(a1, a2);
    d1 = a1;
    d2 = a2;
}

// q = sum [(delta u - log(1+tau u)) + (delta v - log(1+tau v))]
template <class RS>
__device__ __forceinline__ float pass_gain(const RS &R, float delta, float tau) {
    float q = 0.f;
    for_words(R, [&](int c) {
        float ti, tj;
        uint32_t si, sj;
        R.get(c, ti, tj, si, sj);
        float u = flip(ti, sj), v = flip(tj, si);
        q += fmaf(delta, u, -log1pf(tau * u));
        q += fmaf(delta, v, -log1pf(tau * v));
    });
    return R.sum(q);
}

// The 1-D problem of one pair once its pass at delta = 0 is known (sums of u
// and v over the samples and the count of disagreeing spins).  All lanes of the
// warp take part and end with identical results.
template <class RS>
__device__ __forceinline__ void solve_from_pass0(const RS &R, int Mp, float su, float sv, int dis, float Hsum,
                                                 float W0, float lambda, float wclamp, float &gain, float &wstar,
                                                 int &passes) {
    const float twoA = 2.f * (float)(Mp - 2 * dis);
    const float D0 = twoA - su - sv;  // F'(0)
    passes = 0;
    float Dz, Dz2;  // F' and -F'' at w = 0
    if (W0 == 0.f) {
        Dz = D0;
        Dz2 = Hsum;
    } else {
        float tz = tanhf(-W0), d1, d2;
        pass_newton(R, tz, d1, d2);
        ++passes;
        Dz = twoA - d1;
        Dz2 = (1.f - tz * tz) * d2;
    }
    float w = 0.f;
    if (fabsf(Dz) > lambda) {
        const float s = Dz > 0.f ? 1.f : -1.f;
        // G(u) = s F'(s u - W0) - lambda is decreasing in the magnitude u >= 0
        float lo = 0.f, hi = wclamp, u = 0.f;
        float G = s * Dz - lambda, Gp = fmaxf(Dz2, 1e-30f);
        bool hi_seen = false;
        for (int it = 0; it < MAX_NEWTON; ++it) {
            float un = u + G / Gp;
            if (!(un > lo && un < hi)) un = hi_seen ? 0.5f * (lo + hi) : hi;
            float step = fabsf(un - u);
            u = un;
            float delta = s * u - W0, tau = tanhf(delta), d1, d2;
            pass_newton(R, tau, d1, d2);
            ++passes;
            G = s * (twoA - d1) - lambda;
            Gp = fmaxf((1.f - tau * tau) * d2, 1e-30f);
            if (G > 0.f) {
                lo = u;
                if (u >= wclamp) break;  // the optimum lies beyond the clamp
            } else {
                hi = u;
                hi_seen = true;
            }
            float tol = 2e-5f * fmaxf(u, 0.05f);
            if (step <= tol || (hi_seen && hi - lo <= tol)) break;
        }
        w = s * u;
    }
    const float dl = w - W0;
    float g = 0.f;
    if (dl != 0.f) {
        float tau = tanhf(dl);
        float q = pass_gain(R, dl, tau);
        ++passes;
        float F = dl * D0 + q - 2.f * (float)Mp * logcosh_f(dl);
        g = F - lambda * fabsf(w) + lambda * fabsf(W0);
    }
    gain = fmaxf(g, 0.f);
    wstar = w;
}

template <class RS>
__device__ __forceinline__ void solve_pair(const RS &R, int Mp, float Hsum, float W0, float lambda,
                                           float wclamp, float &gain, float &wstar, int &passes) {
    float su, sv;
    int dis;
    pass0(R, su, sv, dis);
    solve_from_pass0(R, Mp, su, sv, dis, Hsum, W0, lambda, wclamp, gain, wstar, passes);
}

// Both rows in shared memory (row j in a staging buffer), the spins as the
// lane's transposed bit columns: the Newton passes of a staged candidate touch
// no global memory.  The scorer builds it with the lower-numbered node of the
// pair as row i, so that the solve sees every pair in one orientation and both
// nodes' blocks give it the same score bit for bit (the passes add the two
// nodes' terms in a fixed order).
struct StageRows {
    static constexpr int kNW = 0;
    // (pass 0 of a staged candidate is pass0_consume: only the Newton and gain
    // passes sum through the row source)
    __device__ __forceinline__ float sum(float a) const { return warp_sum(a); }
    __device__ __forceinline__ void sum2(float &a, float &b) const {
        a = warp_sum(a);
        b = warp_sum(b);
    }
    const float *st;  // t_i
    const float *tj;  // t_j
    uint32_t ci, cj;  // bit c: the spin of sample 32 c + lane (1: -1)
    int Mw, lane;
    __device__ __forceinline__ void get(int c, float &a, float &b, uint32_t &sa, uint32_t &sb_) const {
        a = st[32 * c + lane];
        b = tj[32 * c + lane];
        sa = (ci << (31 - c)) & 0x80000000u;
        sb_ = (cj << (31 - c)) & 0x80000000u;
    }
};

// Pass 0 of the segmented scorer with row i staged in shared memory and both
// rows' spins as transposed bit columns (bit c of lane l's word: sample 32 c + l):
//   su = sum_m x_j t_i = T_i - 2 sum_{x_j = -1} t_i,
//   sv = sum_m x_i t_j = T_j - 2 sum_{x_i = -1} t_j,
//   dis = the samples where x_i != x_j;
// T_i, T_j are the stored row sums, so per sample there are two adds, each
// predicated on a spin bit, and a shared-memory load for the one over t_i.
template <int NW>
__device__ __forceinline__ void pass0_consume(const float *st, int lane, float Ti, float Tj, uint32_t ci,
                                              const float (&t)[NW], uint32_t cj, float &su, float &sv, int &dis) {
    float sj0 = 0.f, sj1 = 0.f, si0 = 0.f, si1 = 0.f;
#pragma unroll
    for (int c = 0; c < NW; c += 2) {
        if (ci & (1u << c)) sj0 += t[c];
        if (cj & (1u << c)) si0 += st[32 * c + lane];
        if (c + 1 < NW) {
            if (ci & (2u << c)) sj1 += t[c + 1];
            if (cj & (2u << c)) si1 += st[32 * (c + 1) + lane];
        }
    }
    su = Ti - 2.f * warp_sum(si0 + si1);
    sv = Tj - 2.f * warp_sum(sj0 + sj1);
    dis = warp_sum_i(__popc(ci ^ cj));
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// the per-node bit columns of IsingView::xT: one warp per node, lane l holding
// word l; lane k keeps the ballot of bit k, whose bit c is bit k of word c
__global__ void k_transpose_bits(IsingView v, uint32_t *xT) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= v.N) return;
    const uint32_t w = lane < v.Mw ? v.xbits[i * v.Mw + lane] : 0u;
    uint32_t mine = 0;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const uint32_t b = __ballot_sync(0xffffffffu, (w >> k) & 1u);
        if (lane == k) mine = b;
    }
    xT[i * 32 + lane] = mine;
}

__global__ void k_pack(const int8_t *X, int64_t M, int64_t N, int Mw, uint32_t *xbits,
                       unsigned long long *cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t ngroups = (N + 31) / 32;
    if (w >= ngroups * Mw) return;
    const int64_t g = w / Mw;
    const int c = (int)(w % Mw);
    const int64_t i = g * 32 + lane;
    if (i >= N) return;
    uint32_t word = 0;
    bool bad = false;
    for (int s = 0; s < 32; ++s) {
        int64_t m = (int64_t)c * 32 + s;
        if (m < M) {
            int8_t x = X[m * N + i];
            if (x == -1)
                word |= 1u << s;
            else if (x != 1)
                bad = true;
        }
    }
    xbits[i * Mw + c] = word;
    if (bad) atomicOr(&cnt[CNT_ERR], (unsigned long long)ERR_BAD_SPIN);
}

// W = 0 field optimum: sum_m (x - tanh h) = 0  =>  h = atanh(mean x), clamped
__global__ void k_init_fields(IsingView v, float h_clamp) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= v.N) return;
    int neg = 0;
    for (int c = lane; c < v.Mw; c += 32) neg += __popc(v.xbits[i * v.Mw + c]);
    neg = warp_sum_i(neg);
    double xbar = (double)(v.M - 2 * neg) / (double)v.M;
    double hh;
    if (xbar >= 1.0)
        hh = h_clamp;
    else if (xbar <= -1.0)
        hh = -h_clamp;
    else {
        hh = 0.5 * log((1.0 + xbar) / (1.0 - xbar));
        hh = fmin(fmax(hh, -(double)h_clamp), (double)h_clamp);
    }
    float h = (float)hh, th = tanhf(h);
    float hs = 0.f;
    for (int m = lane; m < v.Mp; m += 32) {
        bool real = m < v.M;
        v.phi[i * v.Mp + m] = real ? h : 0.f;
        v.t[i * v.Mp + m] = real ? th : 1.f;
        if (real) hs += 1.f - th * th;
    }
    hs = warp_sum(hs);
    if (lane == 0) {
        v.h[i] = h;
        v.H[i] = hs;
        v.T[i] = (float)v.M * th + (float)(v.Mp - v.M);
    }
}

// phi_i = h_i + sum_j W_ij x_j from a CSR of the couplings (deterministic order)
__global__ void k_phi_from_csr(IsingView v, const int64_t *off, const int32_t *nbr, const float *w) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= v.N) return;
    float hs = 0.f, ts = 0.f;
    const float hi = v.h[i];
    for (int m = lane; m < v.Mp; m += 32) {
        if (m >= v.M) {
            v.phi[i * v.Mp + m] = 0.f;
            v.t[i * v.Mp + m] = 1.f;
            continue;
        }
        float s = hi;
        for (int64_t e = off[i]; e < off[i + 1]; ++e) {
            int j = nbr[e];
            uint32_t bit = (v.xbits[(int64_t)j * v.Mw + (m >> 5)] >> (m & 31)) & 1u;
            s += bit ? -w[e] : w[e];
        }
        float tt = tanhf(s);
        v.phi[i * v.Mp + m] = s;
        v.t[i * v.Mp + m] = tt;
        hs += 1.f - tt * tt;
        ts += tt;
    }
    hs = warp_sum(hs);
    ts = warp_sum(ts);
    if (lane == 0) {
        v.H[i] = hs;
        v.T[i] = ts + (float)(v.Mp - v.M);
    }
}

// sum over nodes and samples of x phi - log(2 cosh phi): float terms, double sums
__global__ void k_objective(IsingView v, double *partials) {
    __shared__ double red[32];
    const int64_t total = (int64_t)v.N * v.M;
    double acc = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e / v.M;
        int m = (int)(e - i * v.M);
        float p = v.phi[i * v.Mp + m];
        uint32_t bit = (v.xbits[i * v.Mw + (m >> 5)] >> (m & 31)) & 1u;
        // x phi - log 2cosh phi = (x phi - |phi|) - log(1 + e^{-2|phi|}); the
        // first term is exactly 0 or -2|phi|
        float a = fabsf(p);
        float xp = bit ? -p : p;
        acc += (double)(xp - a) - (double)log1pf(expf(-2.f * a));
    }
    acc = warp_sum_d(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double r = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        r = warp_sum_d(r);
        if (threadIdx.x == 0) partials[blockIdx.x] = r;
    }
}

// Candidates grouped by their first node (one block per segment): segment s
// covers node x = seg_node[s] (local id) and candidates at output positions
// seg_start[s] .. + seg_count[s]; the second node of candidate q is
// cand[2*pos + 1] when cand is given, else seg_vbase[s] + q.  Row x is staged
// in shared memory once.  Each warp takes
// its candidates in chunks of 32: the lanes first resolve the chunk's ids,
// stored couplings and fields in parallel (one round of dependent loads per
// chunk, not per pair), then lane 0 keeps SEG_RING candidate rows (t and the
// bit column) in flight with bulk asynchronous copies into a ring of
// shared-memory stages, one mbarrier per stage.  Every wait is bounded
// (about 1 s); a warp that gives up sets ERR_TIMEOUT, lets its copies land
// (again bounded) and stops.  The error word is the launch's abort flag: a
// waiting warp that sees ERR_TIMEOUT there stops waiting, and a block that sees
// it at its start does no work, so one stall ends the launch in about a second
// however many blocks it has.
constexpr int SEG_RING = 2;

// err: the launch's error word, polled on the slow path (NULL: wait out the bound)
__device__ __forceinline__ bool seg_wait(uint64_t *b, uint32_t par, const unsigned long long *err) {
    if (mbar_try(b, par)) return true;
    uint64_t t0 = 0;
    for (uint32_t n = 1;; ++n) {
        if (mbar_try(b, par)) return true;
        if ((n & 255u) == 0) {
            if (err && (*(const volatile unsigned long long *)err & ERR_TIMEOUT)) return false;
            const uint64_t now = gtimer();
            if (t0 == 0)
                t0 = now;
            else if (now - t0 > 1000000000ull)
                return false;
        }
    }
}

// (at most 80 registers: with 256 threads, three blocks fit on an SM)
template <int NW>
__global__ void __maxnreg__(80) k_score_seg(IsingView v, WTable W, ScoreParams p, const int32_t *seg_node,
                                                      const int64_t *seg_start, const int32_t *seg_count,
                                                      const int32_t *seg_vbase, int64_t nseg, const int32_t *cand,
                                                      const int32_t *gid, float *d_out, unsigned long long *cnt) {
    extern __shared__ __align__(128) float sm[];
    const int64_t sidx = blockIdx.x;
    if (sidx >= nseg) return;
    const int count = seg_count[sidx];
    if (count <= 0) return;
    if (*(const volatile unsigned long long *)(cnt + CNT_ERR) & ERR_TIMEOUT) return;  // the launch gave up
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // layout: row x (Mp floats), its bits (32 words), per warp SEG_RING stages
    // of Mp + 32 words, the stages' mbarriers, then per warp the chunk's ids,
    // stored couplings, fields and row sums (32 each)
    const int stw = v.Mp + 32;
    float *st = sm;
    uint32_t *sb = (uint32_t *)(sm + v.Mp);
    float *ring = sm + v.Mp + 32;
    float *myring = ring + (size_t)warp * SEG_RING * stw;
    uint64_t *bars0 = (uint64_t *)(ring + (size_t)nw * SEG_RING * stw);
    uint64_t *bars = bars0 + warp * SEG_RING;
    int *cgj = (int *)(bars0 + nw * SEG_RING) + warp * 128;
    float *cW0 = (float *)(cgj + 32), *cHj = (float *)(cgj + 64), *cTj = (float *)(cgj + 96);
    if (lane == 0) {
        for (int r = 0; r < SEG_RING; ++r) mbar_init(bars + r, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const int x = seg_node[sidx];
    const int gx = gid ? gid[x] : x;
    const float *tx = v.t + (int64_t)gx * v.Mp;
    const uint32_t *Bx = v.xbits + (int64_t)gx * v.Mw;
    for (int m = threadIdx.x; m < v.Mp; m += blockDim.x) st[m] = tx[m];
    for (int c = threadIdx.x; c < v.Mw; c += blockDim.x) sb[c] = Bx[c];
    __syncthreads();
    const float Hx = v.H[gx];
    const int64_t start = seg_start[sidx];
    const int vbase = seg_vbase ? seg_vbase[sidx] : 0;
    unsigned long long npass = 0;
    const float Tx = v.T[gx];  // sum_m t_x over the Mp samples, padding included
    const uint32_t ci = __ldg(v.xT + (int64_t)gx * 32 + lane);
    const uint32_t stage_bytes = (uint32_t)(v.Mp * 4 + 128);
    const int mine = count > warp ? (count - warp + nw - 1) / nw : 0;  // candidates of this warp
    // lane 0: the warp's k-th candidate (chunk slot k - base) into stage k % SEG_RING
    auto issue = [&](int k, int base) {
        if (p.stall) return;  // fault injection: the stage's wait runs out
        const int s = k % SEG_RING;
        const int g = cgj[k - base];
        mbar_expect_tx(bars + s, stage_bytes);
        bulk_g2s(myring + s * stw, v.t + (int64_t)g * v.Mp, (uint32_t)(v.Mp * 4), bars + s);
        bulk_g2s(myring + s * stw + v.Mp, v.xT + (int64_t)g * 32, 128u, bars + s);
    };
    int k = 0;  // candidates of this warp consumed so far (also its stage sequence number)
    bool ok = true;
    for (int base = 0; base < mine && ok; base += 32) {
        const int nch = min(32, mine - base);
        {  // the chunk's ids, stored couplings and fields, one candidate per lane
            const int q = warp + (base + lane) * nw;
            if (lane < nch) {
                const int vl = cand ? __ldg(cand + 2 * (start + q) + 1) : vbase + q;
                const int g = gid ? gid[vl] : vl;
                cgj[lane] = g;
                cW0[lane] = wt_lookup(W, pair_key(gx, g));
                cHj[lane] = v.H[g];
                cTj[lane] = v.T[g];
            }
        }
        __syncwarp();
        if (lane == 0)
            for (int r = 0; r < SEG_RING && r < nch; ++r) issue(base + r, base);
        __syncwarp();
        for (int u = 0; u < nch; ++u, ++k) {
            const int q = warp + k * nw;
            const int64_t pos = start + q;
            const int s = k % SEG_RING;
            if (!__all_sync(0xffffffffu, seg_wait(bars + s, (uint32_t)((k / SEG_RING) & 1), cnt + CNT_ERR))) {
                ok = false;
                break;
            }
            const float W0 = cW0[u], Hj = cHj[u], Tj = cTj[u];
            const float *row = myring + s * stw;
            float tj[NW];
#pragma unroll
            for (int c = 0; c < NW; ++c) tj[c] = c < v.Mw ? row[32 * c + lane] : 0.f;
            const uint32_t cj = ((const uint32_t *)row)[v.Mp + lane];
            float su, sv;
            int dis;
            pass0_consume<NW>(st, lane, Tx, Tj, ci, tj, cj, su, sv, dis);
            // one orientation per pair: the lower-numbered node first
            const bool sw = cgj[u] < gx;
            if (sw) {
                const float tmp = su;
                su = sv;
                sv = tmp;
            }
            const StageRows R = sw ? StageRows{row, st, cj, ci, v.Mw, lane} : StageRows{st, row, ci, cj, v.Mw, lane};
            float g, w;
            int passes = 0;
            if (p.grad_only)
                g = grad_dist(2.f * (float)(v.Mp - 2 * dis) - su - sv, W0, p.lambda);
            else
                solve_from_pass0(R, v.Mp, su, sv, dis, Hx + Hj, W0, p.lambda, p.w_clamp, g, w, passes);
            if (lane == 0) {
                d_out[pos] = -g;
                npass += (unsigned long long)passes;
            }
            __syncwarp();  // every lane has read stage s: refill it within the chunk
            if (lane == 0 && u + SEG_RING < nch) issue(k + SEG_RING, base);
            __syncwarp();
        }
    }
    if (!ok && lane == 0) {
        atomicOr(&cnt[CNT_ERR], (unsigned long long)ERR_TIMEOUT);
        // the copies still in flight (issued within the chunk) land before the block can leave
        const int base = k / 32 * 32;
        const int nch = min(32, mine - base);
        for (int kk = k; !p.stall && kk < base + nch && kk < k + SEG_RING; ++kk)
            seg_wait(bars + kk % SEG_RING, (uint32_t)((kk / SEG_RING) & 1), nullptr);
    }
    if (lane == 0 && npass) atomicAdd(&cnt[CNT_NEWTON], npass);
}

template <class RS>
__global__ void __launch_bounds__(256) k_score(IsingView v, WTable W, ScoreParams p, const int32_t *pairs,
                                               int64_t P, const int32_t *gid, float *d_out, float *w_out,
                                               unsigned long long *cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long npass = 0;
    for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < P; q += nwarps) {
        int i = pairs[2 * q], j = pairs[2 * q + 1];
        if (gid) {
            i = gid[i];
            j = gid[j];
        }
        RS R;
        R.load(v, i, j, lane);
        float W0 = wt_lookup(W, pair_key(i, j));
        float g, w = W0;
        int passes = 0;
        float su, sv;
        int dis;
        pass0(R, su, sv, dis);
        if (p.grad_only)
            g = grad_dist(2.f * (float)(v.Mp - 2 * dis) - su - sv, W0, p.lambda);
        else
            solve_from_pass0(R, v.Mp, su, sv, dis, v.H[i] + v.H[j], W0, p.lambda, p.w_clamp, g, w, passes);
        if (lane == 0) {
            d_out[q] = -g;
            if (w_out) w_out[q] = w;
            npass += (unsigned long long)passes;
        }
    }
    if (lane == 0 && npass) atomicAdd(&cnt[CNT_NEWTON], npass);
}

// One pair of Algorithm 2's update loop: its 1-D maximiser, then rows i and j
// of phi and t, H_i, H_j and the stored coupling (one warp).
template <class RS>
__device__ __forceinline__ void update_one(IsingView v, WTable W, ScoreParams p, const int32_t *pairs, int pidx,
                                           double *delta, unsigned long long *cnt, int lane) {
    const int i = pairs[2 * pidx], j = pairs[2 * pidx + 1];
    RS R;
    R.template load<true>(v, i, j, lane);
    // the fields phi of both rows, in flight during the solve (one round trip for
    // the row update instead of one per chunk of words)
    constexpr int NWP = RS::kNW > 0 ? RS::kNW : 32;
    float *Pi = v.phi + (int64_t)i * v.Mp, *Pj = v.phi + (int64_t)j * v.Mp;
    float pa[NWP], pb[NWP];
#pragma unroll
    for (int c = 0; c < NWP; ++c) {
        const int m = 32 * c + lane;
        const bool ok = c < v.Mw && m < v.M;
        pa[c] = ok ? Pi[m] : 0.f;
        pb[c] = ok ? Pj[m] : 0.f;
    }
    const uint64_t key = pair_key(i, j);
    const float W0 = wt_lookup(W, key);
    float g, w;
    int passes;
    solve_pair(R, v.Mp, v.H[i] + v.H[j], W0, p.lambda, p.w_clamp, g, w, passes);
    const float dl = w - W0;
    if (dl != 0.f) {
        float *Ti = v.t + (int64_t)i * v.Mp, *Tj = v.t + (int64_t)j * v.Mp;
        float hi = 0.f, hj = 0.f, si_ = 0.f, sj_ = 0.f;
#pragma unroll
        for (int c = 0; c < NWP; ++c) {
            const int m = 32 * c + lane;
            if (c < v.Mw && m < v.M) {
                float a_, b_;
                uint32_t si, sj;
                R.get(c, a_, b_, si, sj);  // si, sj: the sign bits of x_i, x_j at m
                const float pi = pa[c] + (sj ? -dl : dl);
                const float pj = pb[c] + (si ? -dl : dl);
                const float a = tanhf(pi), b = tanhf(pj);
                Pi[m] = pi;
                Pj[m] = pj;
                Ti[m] = a;
                Tj[m] = b;
                hi += 1.f - a * a;
                hj += 1.f - b * b;
                si_ += a;
                sj_ += b;
            }
        }
        hi = warp_sum(hi);
        hj = warp_sum(hj);
        si_ = warp_sum(si_);
        sj_ = warp_sum(sj_);
        if (lane == 0) {
            v.H[i] = hi;
            v.H[j] = hj;
            v.T[i] = si_ + (float)(v.Mp - v.M);
            v.T[j] = sj_ + (float)(v.Mp - v.M);
            if (!wt_upsert(W, key, w)) atomicOr(&cnt[CNT_ERR], (unsigned long long)ERR_TABLE_FULL);
        }
    }
    if (lane == 0) {
        delta[pidx] = fabs((double)dl);
        atomicAdd(&cnt[CNT_NEWTON], (unsigned long long)passes);
    }
}

// One matching batch of the update loop (pairs order[begin..end) share no node,
// so their row updates are independent), one block per pair: the block's warps
// share the pair's samples (BlockRows), so each Newton pass and the row update
// take an eighth of a single warp's time.
template <int NWW>
__global__ void __launch_bounds__(256) k_update_blk(IsingView v, WTable W, ScoreParams p, const int32_t *pairs,
                                                    const int32_t *order, int64_t begin, double *delta,
                                                    unsigned long long *cnt) {
    __shared__ float red[2 * 3 * 8];
    const int pidx = order[begin + blockIdx.x];
    const int i = pairs[2 * pidx], j = pairs[2 * pidx + 1];
    BlockRows<NWW> R;
    R.setup(red);
    R.template load<true>(v, i, j, 0);
    const int lane = R.lane;
    float *Pi = v.phi + (int64_t)i * v.Mp, *Pj = v.phi + (int64_t)j * v.Mp;
    float pa[NWW], pb[NWW];
#pragma unroll
    for (int c = 0; c < NWW; ++c) {
        const int m = 32 * (R.w0 + c) + lane;
        const bool ok = c < R.Mw && m < v.M;
        pa[c] = ok ? Pi[m] : 0.f;
        pb[c] = ok ? Pj[m] : 0.f;
    }
    const uint64_t key = pair_key(i, j);
    const float W0 = wt_lookup(W, key);
    float g, w;
    int passes;
    solve_pair(R, v.Mp, v.H[i] + v.H[j], W0, p.lambda, p.w_clamp, g, w, passes);
    const float dl = w - W0;
    if (dl != 0.f) {
        float *Ti = v.t + (int64_t)i * v.Mp, *Tj = v.t + (int64_t)j * v.Mp;
        float hi = 0.f, hj = 0.f, si_ = 0.f, sj_ = 0.f;
#pragma unroll
        for (int c = 0; c < NWW; ++c) {
            const int m = 32 * (R.w0 + c) + lane;
            if (c < R.Mw && m < v.M) {
                float a_, b_;
                uint32_t si, sj;
                R.get(c, a_, b_, si, sj);
                const float pi = pa[c] + (sj ? -dl : dl);
                const float pj = pb[c] + (si ? -dl : dl);
                const float a = tanhf(pi), b = tanhf(pj);
                Pi[m] = pi;
                Pj[m] = pj;
                Ti[m] = a;
                Tj[m] = b;
                hi += 1.f - a * a;
                hj += 1.f - b * b;
                si_ += a;
                sj_ += b;
            }
        }
        R.sum2(hi, hj);
        R.sum2(si_, sj_);
        if (threadIdx.x == 0) {
            v.H[i] = hi;
            v.H[j] = hj;
            v.T[i] = si_ + (float)(v.Mp - v.M);
            v.T[j] = sj_ + (float)(v.Mp - v.M);
            if (!wt_upsert(W, key, w)) atomicOr(&cnt[CNT_ERR], (unsigned long long)ERR_TABLE_FULL);
        }
    }
    if (threadIdx.x == 0) {
        delta[pidx] = fabs((double)dl);
        atomicAdd(&cnt[CNT_NEWTON], (unsigned long long)passes);
    }
}

// Consecutive thin batches b0 .. b1-1 in one block: the batches run in turn,
// separated by block barriers (which also order the row writes of one batch
// before the reads of the next), each spread over the block's warps.
template <class RS>
__global__ void __launch_bounds__(256) k_update_rounds(IsingView v, WTable W, ScoreParams p, const int32_t *pairs,
                                                       const int32_t *order, const int32_t *off, int b0, int b1,
                                                       double *delta, unsigned long long *cnt) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int b = b0; b < b1; ++b) {
        for (int q = off[b] + warp; q < off[b + 1]; q += nw) update_one<RS>(v, W, p, pairs, order[q], delta, cnt, lane);
        __syncthreads();
    }
}

// Field sweep: h_i' = argmax sum_m [x phi - log 2cosh phi] with phi shifted by
// h_i' - h_i; sum_m (x - tanh(phi + D)) = 0 by safeguarded Newton using
// tanh(phi + D) = (t + T)/(1 + t T), T = tanh D.
template <int NW>
__global__ void __launch_bounds__(256) k_field(IsingView v, ScoreParams p, double *delta) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= v.N) return;
    const float *Ti = v.t + i * v.Mp;
    const uint32_t *Bi = v.xbits + i * v.Mw;
    float tr[NW], xr[NW];
#pragma unroll
    for (int c = 0; c < NW; ++c) {
        int m = 32 * c + lane;
        bool real = c < v.Mw && m < v.M;
        tr[c] = real ? Ti[m] : 0.f;
        xr[c] = real ? (((Bi[c] >> lane) & 1u) ? -1.f : 1.f) : 0.f;  // 0 masks padding
    }
    auto eval = [&](float T, float &S, float &Sp) {
        float a = 0.f, b = 0.f;
#pragma unroll
        for (int c = 0; c < NW; ++c) {
            if (c < v.Mw) {
                float r = rcp_approx(fmaf(tr[c], T, 1.f));
                float mask = xr[c] != 0.f ? 1.f : 0.f;
                a += mask * (xr[c] - (tr[c] + T) * r);
                b += mask * fmaf(-tr[c], tr[c], 1.f) * r * r;
            }
        }
        S = warp_sum(a);
        Sp = (1.f - T * T) * warp_sum(b);
    };
    const float h0 = v.h[i], hc = p.h_clamp;
    float S, Sp;
    eval(0.f, S, Sp);
    float lo = -hc, hi = hc, hcur = h0;  // bracket on the new value h'
    bool lo_seen = false, hi_seen = false;
    if (S > 0.f) { lo = h0; lo_seen = true; } else if (S < 0.f) { hi = h0; hi_seen = true; }
    if (S != 0.f) {
        for (int it = 0; it < MAX_NEWTON; ++it) {
            float hn = hcur + S / fmaxf(Sp, 1e-30f);
            if (!(hn > lo && hn < hi)) {
                if (lo_seen && hi_seen) hn = 0.5f * (lo + hi);
                else hn = lo_seen ? hi : lo;  // try the clamp on the open side
            }
            float step = fabsf(hn - hcur);
            hcur = hn;
            eval(tanhf(hcur - h0), S, Sp);
            if (S > 0.f) {
                lo = hcur;
                lo_seen = true;
                if (hcur >= hc) break;
            } else if (S < 0.f) {
                hi = hcur;
                hi_seen = true;
                if (hcur <= -hc) break;
            } else
                break;
            float tol = 2e-6f * fmaxf(fabsf(hcur), 1.f);
            if (step <= tol || (lo_seen && hi_seen && hi - lo <= tol)) break;
        }
    }
    const float dh = hcur - h0;
    if (dh != 0.f) {
        float *Pi = v.phi + i * v.Mp;
        float *Tw = v.t + i * v.Mp;
        float hs = 0.f, ts = 0.f;
        for (int m = lane; m < v.M; m += 32) {
            float ph = Pi[m] + dh, tt = tanhf(ph);
            Pi[m] = ph;
            Tw[m] = tt;
            hs += 1.f - tt * tt;
            ts += tt;
        }
        hs = warp_sum(hs);
        ts = warp_sum(ts);
        if (lane == 0) {
            v.h[i] = hcur;
            v.H[i] = hs;
            v.T[i] = ts + (float)(v.Mp - v.M);
        }
    }
    if (lane == 0) delta[i] = fabs((double)dh);
}

inline unsigned grid_for(int64_t warps, int threads = 256) {
    int64_t b = (warps * 32 + threads - 1) / threads;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

int ising_max_words() { return 32; }

cudaError_t launch_ising_pack(const int8_t *X_sm, int64_t M, int64_t N, int Mw, uint32_t *xbits,
                              unsigned long long *cnt, cudaStream_t s) {
    int64_t warps = ((N + 31) / 32) * Mw;
    k_pack<<<grid_for(warps), 256, 0, s>>>(X_sm, M, N, Mw, xbits, cnt); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_ising_transpose_bits(IsingView v, uint32_t *xT, cudaStream_t s) {
    k_transpose_bits<<<grid_for(v.N), 256, 0, s>>>(v, xT); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_ising_init_fields(IsingView v, float h_clamp, cudaStream_t s) {
    k_init_fields<<<grid_for(v.N), 256, 0, s>>>(v, h_clamp); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_ising_phi_from_csr(IsingView v, const int64_t *off, const int32_t *nbr, const float *w,
                                      cudaStream_t s) {
    k_phi_from_csr<<<grid_for(v.N), 256, 0, s>>>(v, off, nbr, w); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_ising_objective(IsingView v, double *partials, int nblocks, cudaStream_t s) {
    k_objective<<<nblocks, 256, 0, s>>>(v, partials); note_launch();
    return cudaGetLastError();
}

#define DISPATCH_ROWS(MW, CALL)        \
    do {                               \
        if ((MW) <= 4) {               \
            using RS = RegRows<4>;     \
            CALL;                      \
        } else if ((MW) <= 8) {        \
            using RS = RegRows<8>;     \
            CALL;                      \
        } else if ((MW) <= 16) {       \
            using RS = RegRows<16>;    \
            CALL;                      \
        } else if ((MW) <= 32) {       \
            using RS = RegRows<32>;    \
            CALL;                      \
        } else {                       \
            using RS = GlobRows;       \
            CALL;                      \
        }                              \
    } while (0)

cudaError_t launch_ising_score(IsingView v, WTable W, ScoreParams p, const int32_t *pairs, int64_t P,
                               const int32_t *gid, float *d_out, float *w_out, unsigned long long *cnt,
                               cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    int64_t want = P;
    int64_t cap = (int64_t)1 << 20;  // warps; grid-stride beyond
    unsigned grid = grid_for(want < cap ? want : cap);
    // most pairs stop after the first pass: stream both rows (low registers, high occupancy)
    k_score<GlobRows><<<grid, 256, 0, s>>>(v, W, p, pairs, P, gid, d_out, w_out, cnt);
    note_launch();
    return cudaGetLastError();
}

namespace {
constexpr size_t SEG_SMEM_MAX = 227 * 1024;
size_t seg_smem_bytes(int Mp, int nw) {
    return sizeof(float) * ((size_t)Mp + 32 + (size_t)nw * SEG_RING * (Mp + 32)) +
           (size_t)nw * SEG_RING * sizeof(uint64_t) + (size_t)nw * 128 * sizeof(int);
}
}  // namespace

// the segmented scorer's shared-memory opt-in, once per device (outside any
// stream capture)
cudaError_t ising_score_seg_setup() {
    cudaError_t e = cudaSuccess;
    for (cudaError_t r : {cudaFuncSetAttribute(k_score_seg<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SEG_SMEM_MAX),
                          cudaFuncSetAttribute(k_score_seg<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SEG_SMEM_MAX),
                          cudaFuncSetAttribute(k_score_seg<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SEG_SMEM_MAX),
                          cudaFuncSetAttribute(k_score_seg<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SEG_SMEM_MAX)})
        if (r != cudaSuccess) e = r;
    return e;
}

cudaError_t launch_ising_score_seg(IsingView v, WTable W, ScoreParams p, const int32_t *seg_node,
                                   const int64_t *seg_start, const int32_t *seg_count, const int32_t *seg_vbase,
                                   int64_t nseg, const int32_t *cand, const int32_t *gid, float *d_out,
                                   unsigned long long *cnt, int threads, cudaStream_t s) {
    if (nseg <= 0) return cudaSuccess;
    if (v.Mw > 32 || threads < 32 || threads > 512 || threads % 32) return cudaErrorInvalidValue;
    const size_t smem = seg_smem_bytes(v.Mp, threads / 32);
    if (smem > SEG_SMEM_MAX) return cudaErrorInvalidValue;
#define SEG_LAUNCH(NWV)                                                                                              \
    k_score_seg<NWV><<<(unsigned)nseg, threads, smem, s>>>(v, W, p, seg_node, seg_start, seg_count, seg_vbase, nseg, \
                                                           cand, gid, d_out, cnt)
    if (v.Mw <= 4)
        SEG_LAUNCH(4);
    else if (v.Mw <= 8)
        SEG_LAUNCH(8);
    else if (v.Mw <= 16)
        SEG_LAUNCH(16);
    else
        SEG_LAUNCH(32);
#undef SEG_LAUNCH
    note_launch();
    return cudaGetLastError();
}

// the spins back in the API's sample-major int8 layout (checkpoints)
__global__ void k_unpack_spins(IsingView v, int8_t *X_sm) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)v.N * v.M) return;
    const int64_t m = e / v.N, i = e - m * v.N;
    X_sm[e] = ((v.xbits[i * v.Mw + (m >> 5)] >> (m & 31)) & 1u) ? (int8_t)-1 : (int8_t)1;
}

cudaError_t launch_ising_unpack(IsingView v, int8_t *X_sm, cudaStream_t s) {
    const int64_t n = (int64_t)v.N * v.M;
    k_unpack_spins<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(v, X_sm);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_ising_update(IsingView v, WTable W, ScoreParams p, const int32_t *pairs, const int32_t *order,
                                int64_t begin, int64_t end, double *delta, unsigned long long *cnt,
                                cudaStream_t s) {
    if (end <= begin) return cudaSuccess;
    if (v.Mw > 32) return cudaErrorInvalidValue;
    // one block of 8 warps per pair, each warp ceil(Mw / 8) words
    const unsigned grid = (unsigned)(end - begin);
    if (v.Mw <= 8)
        k_update_blk<1><<<grid, 256, 0, s>>>(v, W, p, pairs, order, begin, delta, cnt);
    else if (v.Mw <= 16)
        k_update_blk<2><<<grid, 256, 0, s>>>(v, W, p, pairs, order, begin, delta, cnt);
    else
        k_update_blk<4><<<grid, 256, 0, s>>>(v, W, p, pairs, order, begin, delta, cnt);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_ising_update_rounds(IsingView v, WTable W, ScoreParams p, const int32_t *pairs,
                                       const int32_t *order, const int32_t *off, int b0, int b1, double *delta,
                                       unsigned long long *cnt, cudaStream_t s) {
    if (b1 <= b0) return cudaSuccess;
    DISPATCH_ROWS(v.Mw, (k_update_rounds<RS><<<1, 256, 0, s>>>(v, W, p, pairs, order, off, b0, b1, delta, cnt))); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_ising_field_sweep(IsingView v, ScoreParams p, double *delta, cudaStream_t s) {
    unsigned grid = grid_for(v.N);
    if (v.Mw > 32) return cudaErrorInvalidValue;
    if (v.Mw <= 4)
        k_field<4><<<grid, 256, 0, s>>>(v, p, delta);
    else if (v.Mw <= 8)
        k_field<8><<<grid, 256, 0, s>>>(v, p, delta);
    else if (v.Mw <= 16)
        k_field<16><<<grid, 256, 0, s>>>(v, p, delta);
    else
        k_field<32><<<grid, 256, 0, s>>>(v, p, delta);
    note_launch();
    return cudaGetLastError();
}
