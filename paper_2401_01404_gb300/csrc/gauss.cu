// gauss.cu -- multivariate-Gaussian pseudo-likelihood kernels (App. A of
// arXiv:2401.01404), the covariance-selection case.
//
// Node i's conditional is Normal(-s2_i mu_i, s2_i) with s2_i = theta_i^2 =
// 1/W_ii and mu_i = sum_{j != i} W_ij x_j.  With the residual
// e_i = x_i + s2_i mu_i, moving W_ij by delta changes the log pseudo-likelihood
// by exactly
//     a delta - b delta^2 / 2,   a = -sum_m (e_i x_j + e_j x_i),
//                                b = s2_i sum_m x_j^2 + s2_j sum_m x_i^2,
// so under the Laplace prior the best coupling is the soft threshold
// w* = sign(z) max(|z| - lambda/b, 0) with z = W_ij + a/b, and its gain is
// a (w* - W_ij) - b (w* - W_ij)^2/2 - lambda |w*| + lambda |W_ij|.  No
// iteration is needed: one pass of two dot products per pair.
// The diagonal (theta_i^2, no prior) maximises
//     sum_m [-(x_i + u mu_i)^2/(2u)] - (M/2) log u,
// whose stationarity condition C u^2 + M u - A = 0 (A = sum x_i^2,
// C = sum mu_i^2) gives u = 2A / (M + sqrt(M^2 + 4AC)).
#include "common.cuh"

namespace {

__global__ void k_gpack(const float *X, int64_t M, int64_t N, int Mp, float *xg, unsigned long long *cnt) {
    // one thread per (node, sample); reads are coalesced along nodes
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * (int64_t)Mp) return;
    int64_t m = e / N, i = e - m * N;
    float v = 0.f;
    if (m < M) {
        v = X[m * N + i];
        if (!isfinite(v)) {
            atomicOr(&cnt[CNT_ERR], (unsigned long long)ERR_BAD_VALUE);
            v = 0.f;
        }
    }
    xg[i * Mp + m] = v;
}

// W = 0: theta_i^2 = mean x_i^2, mu = 0, e = x
__global__ void k_ginit(GaussView v) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= v.N) return;
    double q = 0.0;
    for (int m = lane; m < v.Mp; m += 32) {
        float x = v.xg[i * v.Mp + m];
        q += (double)x * x;
        v.mu[i * v.Mp + m] = 0.f;
        v.e[i * v.Mp + m] = x;
    }
    q = warp_sum_d(q);
    if (lane == 0) {
        v.Q[i] = (float)q;
        v.s2[i] = (float)(q / v.M);
    }
}

__global__ void k_gmu_from_csr(GaussView v, const int64_t *off, const int32_t *nbr, const float *w) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= v.N) return;
    const float s2 = v.s2[i];
    for (int m = lane; m < v.Mp; m += 32) {
        float s = 0.f;
        for (int64_t q = off[i]; q < off[i + 1]; ++q) s += w[q] * v.xg[(int64_t)nbr[q] * v.Mp + m];
        v.mu[i * v.Mp + m] = s;
        v.e[i * v.Mp + m] = v.xg[i * v.Mp + m] + s2 * s;
    }
}

__global__ void k_gobjective(GaussView v, double *partials) {
    __shared__ double red[32];
    const int64_t total = (int64_t)v.N * v.M;
    const double half_log_2pi = 0.91893853320467274178;
    double acc = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e / v.M;
        int m = (int)(e - i * v.M);
        float r = v.e[i * v.Mp + m];
        float s2 = v.s2[i];
        acc += (double)(-r * r / (2.f * s2)) - 0.5 * log((double)s2) - half_log_2pi;
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

// a = -sum (e_i x_j + e_j x_i), over float4 chunks (Mp is a multiple of 32)
// coherent = true reads e with plain loads (rows that an earlier batch of the
// same launch may have written; the read-only path could be stale)
template <bool coherent = false>
__device__ __forceinline__ float gauss_a(const GaussView &v, int i, int j, int lane) {
    const float4 *xi = (const float4 *)(v.xg + (int64_t)i * v.Mp), *xj = (const float4 *)(v.xg + (int64_t)j * v.Mp);
    const float4 *ei = (const float4 *)(v.e + (int64_t)i * v.Mp), *ej = (const float4 *)(v.e + (int64_t)j * v.Mp);
    float acc = 0.f;
    for (int q = lane; q < v.Mp / 4; q += 32) {
        float4 a = coherent ? ei[q] : __ldg(ei + q), b = __ldg(xj + q), c = coherent ? ej[q] : __ldg(ej + q),
               d = __ldg(xi + q);
        acc = fmaf(a.x, b.x, acc);
        acc = fmaf(a.y, b.y, acc);
        acc = fmaf(a.z, b.z, acc);
        acc = fmaf(a.w, b.w, acc);
        acc = fmaf(c.x, d.x, acc);
        acc = fmaf(c.y, d.y, acc);
        acc = fmaf(c.z, d.z, acc);
        acc = fmaf(c.w, d.w, acc);
    }
    return -warp_sum(acc);
}

__device__ __forceinline__ void gauss_solve(float a, float b, float W0, float lambda, float wclamp, float &gain,
                                            float &w) {
    float z = W0 + a / b;
    float mag = fmaxf(fabsf(z) - lambda / b, 0.f);
    w = copysignf(fminf(mag, wclamp), z);
    if (mag == 0.f) w = 0.f;
    float dl = w - W0;
    float g = a * dl - 0.5f * b * dl * dl - lambda * fabsf(w) + lambda * fabsf(W0);
    gain = fmaxf(g, 0.f);
}

__global__ void __launch_bounds__(256) k_gscore(GaussView v, WTable W, ScoreParams p, const int32_t *pairs,
                                                int64_t P, const int32_t *gid, float *d_out, float *w_out) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < P; q += nwarps) {
        int i = pairs[2 * q], j = pairs[2 * q + 1];
        if (gid) {
            i = gid[i];
            j = gid[j];
        }
        float a = gauss_a(v, i, j, lane);
        float b = v.s2[i] * v.Q[j] + v.s2[j] * v.Q[i];
        float W0 = wt_lookup(W, pair_key(i, j));
        float g, w = W0;
        if (p.grad_only)
            g = grad_dist(a, W0, p.lambda);
        else
            gauss_solve(a, b, W0, p.lambda, p.w_clamp, g, w);
        if (lane == 0) {
            d_out[q] = -g;
            if (w_out) w_out[q] = w;
        }
    }
}

// Segmented form (see k_score_seg in ising.cu): one block per segment, row x
// (x_x and e_x) staged in shared memory, each warp streams the rows of its
// candidates with float4 loads.  The block width is a launch parameter (the
// autotuner picks it).
__global__ void k_gscore_seg(GaussView v, WTable W, ScoreParams p, const int32_t *seg_node, const int64_t *seg_start,
                             const int32_t *seg_count, const int32_t *seg_vbase, int64_t nseg, const int32_t *cand,
                             const int32_t *gid, float *d_out) {
    extern __shared__ float sm[];
    const int64_t sidx = blockIdx.x;
    if (sidx >= nseg) return;
    const int count = seg_count[sidx];
    if (count <= 0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float *sx = sm, *se = sm + v.Mp;
    const int x = seg_node[sidx];
    const int gx = gid ? gid[x] : x;
    for (int m = threadIdx.x; m < v.Mp; m += blockDim.x) {
        sx[m] = v.xg[(int64_t)gx * v.Mp + m];
        se[m] = v.e[(int64_t)gx * v.Mp + m];
    }
    __syncthreads();
    const float s2x = v.s2[gx], Qx = v.Q[gx];
    const int64_t start = seg_start[sidx];
    const int vbase = seg_vbase ? seg_vbase[sidx] : 0;
    const float4 *sx4 = (const float4 *)sx, *se4 = (const float4 *)se;
    for (int q = warp; q < count; q += nw) {
        const int64_t pos = start + q;
        const int vl = cand ? cand[2 * pos + 1] : vbase + q;
        const int gj = gid ? gid[vl] : vl;
        const float4 *xj = (const float4 *)(v.xg + (int64_t)gj * v.Mp), *ej = (const float4 *)(v.e + (int64_t)gj * v.Mp);
        float a0 = 0.f, a1 = 0.f;
        for (int c4 = lane; c4 < v.Mp / 4; c4 += 32) {
            const float4 b = __ldg(xj + c4), d = __ldg(ej + c4), ex = se4[c4], xx = sx4[c4];
            a0 = fmaf(ex.x, b.x, a0);
            a0 = fmaf(ex.y, b.y, a0);
            a0 = fmaf(ex.z, b.z, a0);
            a0 = fmaf(ex.w, b.w, a0);
            a1 = fmaf(d.x, xx.x, a1);
            a1 = fmaf(d.y, xx.y, a1);
            a1 = fmaf(d.z, xx.z, a1);
            a1 = fmaf(d.w, xx.w, a1);
        }
        const float a = -warp_sum(a0 + a1);
        const float b = s2x * v.Q[gj] + v.s2[gj] * Qx;
        const float W0 = wt_lookup(W, pair_key(gx, gj));
        float g, w;
        if (p.grad_only)
            g = grad_dist(a, W0, p.lambda);
        else
            gauss_solve(a, b, W0, p.lambda, p.w_clamp, g, w);
        if (lane == 0) d_out[pos] = -g;
    }
}

// One pair of Algorithm 2's update loop (closed-form maximiser), then rows i
// and j of mu and e and the stored coupling (one warp).
__device__ __forceinline__ void gupdate_one(GaussView v, WTable W, ScoreParams p, const int32_t *pairs, int pidx,
                                            double *delta, unsigned long long *cnt, int lane) {
    const int i = pairs[2 * pidx], j = pairs[2 * pidx + 1];
    const uint64_t key = pair_key(i, j);
    const float W0 = wt_lookup(W, key);
    float a = gauss_a<true>(v, i, j, lane);
    float b = v.s2[i] * v.Q[j] + v.s2[j] * v.Q[i];
    float g, w;
    gauss_solve(a, b, W0, p.lambda, p.w_clamp, g, w);
    const float dl = w - W0;
    if (dl != 0.f) {
        const float s2i = v.s2[i], s2j = v.s2[j];
        const float *Xi = v.xg + (int64_t)i * v.Mp, *Xj = v.xg + (int64_t)j * v.Mp;
        float *Ui = v.mu + (int64_t)i * v.Mp, *Uj = v.mu + (int64_t)j * v.Mp;
        float *Ei = v.e + (int64_t)i * v.Mp, *Ej = v.e + (int64_t)j * v.Mp;
        // samples in chunks of 8 per lane: every load of a chunk is in flight
        // before the first is used (one round trip to L2 per chunk)
        constexpr int UCH = 8;
        for (int m0 = 0; m0 < v.M; m0 += 32 * UCH) {
            float xa[UCH], xb[UCH], ua[UCH], ub[UCH];
#pragma unroll
            for (int q = 0; q < UCH; ++q) {
                const int m = m0 + 32 * q + lane;
                const bool ok = m < v.M;
                xa[q] = ok ? __ldg(Xi + m) : 0.f;
                xb[q] = ok ? __ldg(Xj + m) : 0.f;
                ua[q] = ok ? Ui[m] : 0.f;
                ub[q] = ok ? Uj[m] : 0.f;
            }
#pragma unroll
            for (int q = 0; q < UCH; ++q) {
                const int m = m0 + 32 * q + lane;
                if (m < v.M) {
                    const float mi = ua[q] + dl * xb[q], mj = ub[q] + dl * xa[q];
                    Ui[m] = mi;
                    Uj[m] = mj;
                    Ei[m] = fmaf(s2i, mi, xa[q]);
                    Ej[m] = fmaf(s2j, mj, xb[q]);
                }
            }
        }
        if (lane == 0 && !wt_upsert(W, key, w)) atomicOr(&cnt[CNT_ERR], (unsigned long long)ERR_TABLE_FULL);
    }
    if (lane == 0) delta[pidx] = fabs((double)dl);
}

__global__ void __launch_bounds__(256) k_gupdate(GaussView v, WTable W, ScoreParams p, const int32_t *pairs,
                                                 const int32_t *order, int64_t begin, int64_t end, double *delta,
                                                 unsigned long long *cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t q = begin + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (q >= end) return;
    gupdate_one(v, W, p, pairs, order[q], delta, cnt, lane);
}

// Consecutive thin batches b0 .. b1-1 in one block, separated by block barriers.
__global__ void __launch_bounds__(1024) k_gupdate_rounds(GaussView v, WTable W, ScoreParams p, const int32_t *pairs,
                                                         const int32_t *order, const int32_t *off, int b0, int b1,
                                                         double *delta, unsigned long long *cnt) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int b = b0; b < b1; ++b) {
        for (int q = off[b] + warp; q < off[b + 1]; q += nw) gupdate_one(v, W, p, pairs, order[q], delta, cnt, lane);
        __syncthreads();
    }
}

__global__ void k_gdiag(GaussView v, double *delta) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= v.N) return;
    double C = 0.0;
    for (int m = lane; m < v.M; m += 32) {
        double mu = v.mu[i * v.Mp + m];
        C += mu * mu;
    }
    C = warp_sum_d(C);
    const double A = v.Q[i], M = v.M;
    const double u = 2.0 * A / (M + sqrt(M * M + 4.0 * A * C));
    const float uf = (float)u;
    const float old = v.s2[i];
    if (uf != old) {
        for (int m = lane; m < v.M; m += 32)
            v.e[i * v.Mp + m] = fmaf(uf, v.mu[i * v.Mp + m], v.xg[i * v.Mp + m]);
    }
    if (lane == 0) {
        v.s2[i] = uf;
        delta[i] = fabs((double)uf - (double)old);
    }
}

inline unsigned grid_for(int64_t warps, int threads = 256) {
    int64_t b = (warps * 32 + threads - 1) / threads;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

// the samples back in the API's sample-major layout (checkpoints)
__global__ void k_gunpack(GaussView v, float *X_sm) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)v.N * v.M) return;
    const int64_t m = e / v.N, i = e - m * v.N;
    X_sm[e] = v.xg[i * v.Mp + m];
}

cudaError_t launch_gauss_unpack(GaussView v, float *X_sm, cudaStream_t s) {
    const int64_t n = (int64_t)v.N * v.M;
    k_gunpack<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(v, X_sm);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_gauss_pack(const float *X_sm, int64_t M, int64_t N, int Mp, float *xg, unsigned long long *cnt,
                              cudaStream_t s) {
    int64_t n = N * (int64_t)Mp;
    k_gpack<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(X_sm, M, N, Mp, xg, cnt); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_gauss_init(GaussView v, cudaStream_t s) {
    k_ginit<<<grid_for(v.N), 256, 0, s>>>(v); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_gauss_mu_from_csr(GaussView v, const int64_t *off, const int32_t *nbr, const float *w,
                                     cudaStream_t s) {
    k_gmu_from_csr<<<grid_for(v.N), 256, 0, s>>>(v, off, nbr, w); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_gauss_objective(GaussView v, double *partials, int nblocks, cudaStream_t s) {
    k_gobjective<<<nblocks, 256, 0, s>>>(v, partials); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_gauss_score(GaussView v, WTable W, ScoreParams p, const int32_t *pairs, int64_t P,
                               const int32_t *gid, float *d_out, float *w_out, unsigned long long *cnt,
                               cudaStream_t s) {
    (void)cnt;
    if (P <= 0) return cudaSuccess;
    int64_t cap = (int64_t)1 << 20;
    k_gscore<<<grid_for(P < cap ? P : cap), 256, 0, s>>>(v, W, p, pairs, P, gid, d_out, w_out); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_gauss_score_seg(GaussView v, WTable W, ScoreParams p, const int32_t *seg_node,
                                   const int64_t *seg_start, const int32_t *seg_count, const int32_t *seg_vbase,
                                   int64_t nseg, const int32_t *cand, const int32_t *gid, float *d_out, int threads,
                                   cudaStream_t s) {
    if (nseg <= 0) return cudaSuccess;
    const size_t smem = sizeof(float) * 2 * v.Mp;
    // the limit depends on M, so it is set for every launch that needs more than
    // the default (a host-side attribute call, also legal during graph capture)
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_gscore_seg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_gscore_seg<<<(unsigned)nseg, threads, smem, s>>>(v, W, p, seg_node, seg_start, seg_count, seg_vbase, nseg, cand,
                                                       gid, d_out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_gauss_update(GaussView v, WTable W, ScoreParams p, const int32_t *pairs, const int32_t *order,
                                int64_t begin, int64_t end, double *delta, unsigned long long *cnt,
                                cudaStream_t s) {
    if (end <= begin) return cudaSuccess;
    k_gupdate<<<grid_for(end - begin), 256, 0, s>>>(v, W, p, pairs, order, begin, end, delta, cnt); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_gauss_update_rounds(GaussView v, WTable W, ScoreParams p, const int32_t *pairs,
                                       const int32_t *order, const int32_t *off, int b0, int b1, double *delta,
                                       unsigned long long *cnt, cudaStream_t s) {
    if (b1 <= b0) return cudaSuccess;
    k_gupdate_rounds<<<1, 1024, 0, s>>>(v, W, p, pairs, order, off, b0, b1, delta, cnt); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_gauss_diag_sweep(GaussView v, double *delta, cudaStream_t s) {
    k_gdiag<<<grid_for(v.N), 256, 0, s>>>(v, delta); note_launch();
    return cudaGetLastError();
}
