// util.cu -- generic device utilities of librecon: reductions, scans, a stable
// LSD radix sort, the coupling table maintenance, and the matching-batch
// layering of the parallel coordinate updates (App. B).
#include "common.cuh"

namespace {

// -------- reductions --------------------------------------------------------

__global__ void k_penalty(WTable W, double *out) {
    __shared__ double red[32];
    double acc = 0.0;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s <= W.mask;
         s += (uint64_t)gridDim.x * blockDim.x)
        if (W.keys[s] != RECON_EMPTY_KEY) acc += fabs((double)W.vals[s]);
    acc = warp_sum_d(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double r = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        r = warp_sum_d(r);
        if (threadIdx.x == 0) out[blockIdx.x] = r;
    }
}

// fixed-order sum of n doubles (one block; deterministic)
__global__ void k_sum_doubles(const double *in, int64_t n, double *out) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) acc += in[e];
    acc = warp_sum_d(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double r = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        r = warp_sum_d(r);
        if (threadIdx.x == 0) *out = r;
    }
}

__global__ void k_fill_u64(unsigned long long *p, unsigned long long v, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        p[e] = v;
}
__global__ void k_fill_i32(int32_t *p, int32_t v, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        p[e] = v;
}

__global__ void k_table_count(WTable W, unsigned long long *out) {
    unsigned long long c = 0;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s <= W.mask;
         s += (uint64_t)gridDim.x * blockDim.x)
        c += W.keys[s] != RECON_EMPTY_KEY;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

__global__ void k_table_dump(WTable W, int32_t *ij, float *w, unsigned long long *cursor) {
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s <= W.mask;
         s += (uint64_t)gridDim.x * blockDim.x) {
        unsigned long long k = W.keys[s];
        if (k == RECON_EMPTY_KEY) continue;
        unsigned long long q = atomicAdd(cursor, 1ull);
        ij[2 * q] = (int32_t)(k >> 32);
        ij[2 * q + 1] = (int32_t)(k & 0xffffffffu);
        w[q] = W.vals[s];
    }
}

__global__ void k_table_insert(WTable T, const int32_t *ij, const float *w, int64_t n, unsigned long long *cnt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        if (!wt_upsert(T, pair_key(ij[2 * e], ij[2 * e + 1]), w[e]))
            atomicOr(&cnt[CNT_ERR], (unsigned long long)ERR_TABLE_FULL);
}

// every id in [0, n) and the two ends different
__global__ void k_check_pairs(const int32_t *pairs, int64_t P, int n, unsigned long long *cnt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (int64_t)gridDim.x * blockDim.x) {
        int a = pairs[2 * e], b = pairs[2 * e + 1];
        if (a < 0 || a >= n || b < 0 || b >= n || a == b)
            atomicOr(&cnt[CNT_ERR], (unsigned long long)ERR_BAD_VALUE);
    }
}

__global__ void k_table_rehash(WTable from, WTable to) {
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s <= from.mask;
         s += (uint64_t)gridDim.x * blockDim.x) {
        unsigned long long k = from.keys[s];
        if (k != RECON_EMPTY_KEY) wt_upsert(to, k, from.vals[s]);
    }
}

// -------- matching batches in O(P) -------------------------------------------
// Algorithm 2's update loop in matching batches: a pair goes into the batch after
// the latest batch holding an earlier pair that shares a node with it, so that
// applying the batches in turn (the pairs of a batch share no node) equals the
// sequential loop.  The batches are found through the per-node order of the pairs:
// entry e = 2p + side stands for pair p at node pairs[e]; after a stable sort of
// the entries by node, the entry that follows e at the same node is the next
// pair there.  A pair's batch is one more than the latest batch among the
// pairs before it at its two nodes, i.e. it joins the frontier after both its
// predecessors have been placed.
__global__ void k_node_entries(const int32_t *pairs, int64_t P, unsigned long long *keys, uint32_t *vals) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 2 * P) return;
    keys[e] = ((unsigned long long)(uint32_t)pairs[e] << 32) | (unsigned long long)(uint32_t)e;
    vals[e] = (uint32_t)e;
}

__global__ void k_node_links(const unsigned long long *keys, int64_t n2, int32_t *succ, int32_t *indeg) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n2) return;
    const unsigned long long cur = keys[k];
    int32_t nxt = -1;
    if (k + 1 < n2 && (keys[k + 1] >> 32) == (cur >> 32)) {
        nxt = (int32_t)((uint32_t)keys[k + 1] >> 1);
        atomicAdd(&indeg[nxt], 1);
    }
    succ[(uint32_t)cur] = nxt;
}

// One block.  Each pair enters exactly one frontier (links only go from a pair
// to a later one), so the loop ends after at most P batches.
__global__ void __launch_bounds__(1024) k_frontier(int64_t P, const int32_t *succ, int32_t *indeg, int *batch,
                                                   int32_t *fa, int32_t *fb, int *nb_out) {
    __shared__ int n_cur, n_next;
    if (threadIdx.x == 0) n_cur = 0;
    __syncthreads();
    for (int64_t p = threadIdx.x; p < P; p += blockDim.x)
        if (indeg[p] == 0) fa[atomicAdd(&n_cur, 1)] = (int32_t)p;
    __syncthreads();
    int r = 0;
    int32_t *cur = fa, *nxt = fb;
    while (n_cur > 0) {
        if (threadIdx.x == 0) n_next = 0;
        __syncthreads();
        const int nc = n_cur;
        for (int q = threadIdx.x; q < nc; q += blockDim.x) {
            const int p = cur[q];
            batch[p] = r;
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const int sc = succ[2 * p + side];
                if (sc >= 0 && atomicSub(&indeg[sc], 1) == 1) nxt[atomicAdd(&n_next, 1)] = sc;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) n_cur = n_next;
        int32_t *t = cur;
        cur = nxt;
        nxt = t;
        ++r;
        __syncthreads();
    }
    if (threadIdx.x == 0) *nb_out = r;
}

// pairs grouped by batch (order within a batch is free: its pairs are
// independent); boff[b] = the start of batch b, boff[nb] = P
__global__ void __launch_bounds__(1024) k_batch_order(int64_t P, const int *batch, const int *nb_in, int *order,
                                                      int *boff) {
    const int nb = *nb_in;
    for (int b = threadIdx.x; b <= nb; b += blockDim.x) boff[b] = 0;
    __syncthreads();
    for (int64_t p = threadIdx.x; p < P; p += blockDim.x) atomicAdd(&boff[batch[p] + 1], 1);
    __syncthreads();
    if (threadIdx.x == 0)
        for (int b = 0; b < nb; ++b) boff[b + 1] += boff[b];
    __syncthreads();
    for (int64_t p = threadIdx.x; p < P; p += blockDim.x) order[atomicAdd(&boff[batch[p]], 1)] = (int)p;
    __syncthreads();
    if (threadIdx.x == 0) {  // boff[b] now holds the end of batch b
        for (int b = nb; b > 0; --b) boff[b] = boff[b - 1];
        boff[0] = 0;
    }
}

// -------- scan ---------------------------------------------------------------
constexpr int SCAN_B = 1024;

constexpr int64_t SMALL_SCAN = 64 * 1024;

__global__ void __launch_bounds__(SCAN_B) k_scan_small(const int64_t *in, int64_t *out, int64_t n) {
    __shared__ int64_t s[SCAN_B];
    const int64_t per = (n + SCAN_B - 1) / SCAN_B;
    const int64_t b = threadIdx.x * per, e = min(n, b + per);
    int64_t sum = 0;
    for (int64_t q = b; q < e; ++q) sum += in[q];
    s[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < SCAN_B; o <<= 1) {
        int64_t add = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
        __syncthreads();
        s[threadIdx.x] += add;
        __syncthreads();
    }
    int64_t run = s[threadIdx.x] - sum;  // exclusive prefix of this thread's run
    for (int64_t q = b; q < e; ++q) {
        const int64_t v = in[q];
        out[q] = run;
        run += v;
    }
}

__global__ void k_scan_block(const int64_t *in, int64_t *out, int64_t n, int64_t *sums) {
    __shared__ int64_t s[SCAN_B];
    int64_t g = (int64_t)blockIdx.x * SCAN_B + threadIdx.x;
    int64_t v = g < n ? in[g] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < SCAN_B; o <<= 1) {
        int64_t add = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
        __syncthreads();
        s[threadIdx.x] += add;
        __syncthreads();
    }
    if (g < n) out[g] = s[threadIdx.x] - v;  // exclusive
    if (threadIdx.x == SCAN_B - 1 && sums) sums[blockIdx.x] = s[threadIdx.x];
}

__global__ void k_scan_add(int64_t *out, int64_t n, const int64_t *offs) {
    int64_t g = (int64_t)blockIdx.x * SCAN_B + threadIdx.x;
    if (g < n) out[g] += offs[blockIdx.x];
}

// -------- radix sort ------------------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const unsigned long long *keys, int64_t n, int shift,
                                                        int64_t ntiles, int64_t *hist) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int it = 0; it < RS_ITEMS; ++it) {
        int64_t e = base + it * RS_THREADS + threadIdx.x;
        if (e < n) atomicAdd(&h[(keys[e] >> shift) & 0xff], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const unsigned long long *keys, const uint32_t *vals,
                                                           unsigned long long *keys_out, uint32_t *vals_out,
                                                           int64_t n, int shift, int64_t ntiles,
                                                           const int64_t *offs) {
    __shared__ int64_t base_off[256];
    __shared__ int cnt[RS_THREADS / 32][256];
    __shared__ int run[256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    base_off[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    run[threadIdx.x] = 0;
    const int64_t tile = (int64_t)blockIdx.x * RS_TILE;
    for (int it = 0; it < RS_ITEMS; ++it) {
        for (int w = 0; w < RS_THREADS / 32; ++w) cnt[w][threadIdx.x] = 0;
        __syncthreads();
        int64_t e = tile + it * RS_THREADS + threadIdx.x;
        bool valid = e < n;
        unsigned long long k = valid ? keys[e] : 0ull;
        uint32_t val = valid ? vals[e] : 0u;
        int d = valid ? (int)((k >> shift) & 0xff) : 256 + lane;  // invalid lanes never match valid ones
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & ((1u << lane) - 1u));
        int leader = __ffs(peers) - 1;
        if (valid && lane == leader) cnt[warp][d] = __popc(peers);
        __syncthreads();
        {
            int acc = run[threadIdx.x];
            for (int w = 0; w < RS_THREADS / 32; ++w) {
                int c = cnt[w][threadIdx.x];
                cnt[w][threadIdx.x] = acc;
                acc += c;
            }
            run[threadIdx.x] = acc;
        }
        __syncthreads();
        if (valid) {
            int64_t pos = base_off[d] + cnt[warp][d] + rank;
            keys_out[pos] = k;
            vals_out[pos] = val;
        }
        __syncthreads();
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

cudaError_t launch_penalty(WTable W, double *out, cudaStream_t s) {
    // out must hold 256 partials; caller sums them
    k_penalty<<<256, 256, 0, s>>>(W, out); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_sum_doubles(const double *in, int64_t n, double *out, cudaStream_t s) {
    k_sum_doubles<<<1, 1024, 0, s>>>(in, n, out); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_fill_u64(unsigned long long *p, unsigned long long v, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int64_t b = (n + 255) / 256;
    k_fill_u64<<<(unsigned)(b > 4096 ? 4096 : b), 256, 0, s>>>(p, v, n); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_fill_i32(int32_t *p, int32_t v, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int64_t b = (n + 255) / 256;
    k_fill_i32<<<(unsigned)(b > 4096 ? 4096 : b), 256, 0, s>>>(p, v, n); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_table_count(WTable W, unsigned long long *out, cudaStream_t s) {
    k_table_count<<<512, 256, 0, s>>>(W, out); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_table_dump(WTable W, int32_t *ij, float *w, unsigned long long *cursor, cudaStream_t s) {
    k_table_dump<<<512, 256, 0, s>>>(W, ij, w, cursor); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_table_insert(WTable T, const int32_t *ij, const float *w, int64_t n, unsigned long long *cnt,
                                cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_table_insert<<<256, 256, 0, s>>>(T, ij, w, n, cnt); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_check_pairs(const int32_t *pairs, int64_t P, int n, unsigned long long *cnt, cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    int64_t b = (P + 255) / 256;
    k_check_pairs<<<(unsigned)(b > 4096 ? 4096 : b), 256, 0, s>>>(pairs, P, n, cnt); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_table_rehash(WTable from, WTable to, cudaStream_t s) {
    k_table_rehash<<<512, 256, 0, s>>>(from, to); note_launch();
    return cudaGetLastError();
}

int64_t scan_tmp_elems(int64_t n) {
    int64_t total = 0;
    while (n > SCAN_B) {
        n = (n + SCAN_B - 1) / SCAN_B;
        total += 2 * n;
    }
    return total + 2;
}

// exclusive scan, recursive over block sums; up to SMALL_SCAN elements in one
// block (each thread scans a contiguous run, the runs' sums are scanned in
// shared memory), which saves the recursion's launches on the many short scans
// of a search
cudaError_t launch_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (n > SCAN_B && n <= SMALL_SCAN) {
        k_scan_small<<<1, SCAN_B, 0, s>>>(in, out, n); note_launch();
        return cudaGetLastError();
    }
    int64_t nb = (n + SCAN_B - 1) / SCAN_B;
    if (nb == 1) {
        k_scan_block<<<1, SCAN_B, 0, s>>>(in, out, n, nullptr); note_launch();
        return cudaGetLastError();
    }
    int64_t *sums = tmp, *sums_scan = tmp + nb;
    k_scan_block<<<(unsigned)nb, SCAN_B, 0, s>>>(in, out, n, sums); note_launch();
    cudaError_t e = launch_scan_i64(sums, sums_scan, nb, tmp + 2 * nb, s);
    if (e != cudaSuccess) return e;
    k_scan_add<<<(unsigned)nb, SCAN_B, 0, s>>>(out, n, sums_scan); note_launch();
    return cudaGetLastError();
}

int64_t radix_tmp_elems(int64_t n) {
    int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    int64_t h = 256 * ntiles;
    return 2 * h + scan_tmp_elems(h);
}

cudaError_t radix_sort_u64(unsigned long long *keys, uint32_t *vals, unsigned long long *keys_alt,
                           uint32_t *vals_alt, int64_t n, int bit0, int bit1, int64_t *tmp,
                           bool *result_in_alt, cudaStream_t s) {
    *result_in_alt = false;
    if (n <= 1) return cudaSuccess;
    int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    int64_t h = 256 * ntiles;
    int64_t *hist = tmp, *offs = tmp + h, *stmp = tmp + 2 * h;
    unsigned long long *ki = keys, *ko = keys_alt;
    uint32_t *vi = vals, *vo = vals_alt;
    bool alt = false;
    for (int shift = bit0; shift < bit1; shift += 8) {
        k_rs_hist<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(ki, n, shift, ntiles, hist); note_launch();
        cudaError_t e = launch_scan_i64(hist, offs, h, stmp, s);
        if (e != cudaSuccess) return e;
        k_rs_scatter<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(ki, vi, ko, vo, n, shift, ntiles, offs); note_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        unsigned long long *tk = ki;
        ki = ko;
        ko = tk;
        uint32_t *tv = vi;
        vi = vo;
        vo = tv;
        alt = !alt;
    }
    *result_in_alt = alt;
    return cudaSuccess;
}

int64_t layer_tmp_elems(int64_t P) { return radix_tmp_elems(std::max<int64_t>(2 * P, 2)); }

cudaError_t launch_layer_frontier(const int32_t *pairs, int64_t P, int N, unsigned long long *keys,
                                  unsigned long long *keys_alt, uint32_t *vals, uint32_t *vals_alt, int64_t *tmp,
                                  int32_t *succ, int32_t *indeg, int32_t *fa, int32_t *fb, int *batch, int *order,
                                  int *boff, int *nb, cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    const int64_t n2 = 2 * P;
    const unsigned g2 = (unsigned)((n2 + 255) / 256);
    k_node_entries<<<g2, 256, 0, s>>>(pairs, P, keys, vals); note_launch();
    int bits = 8;
    while (bits < 32 && ((int64_t)1 << bits) < (int64_t)N) bits += 8;
    bool alt = false;
    cudaError_t e = radix_sort_u64(keys, vals, keys_alt, vals_alt, n2, 32, 32 + bits, tmp, &alt, s);
    if (e != cudaSuccess) return e;
    const unsigned long long *sorted = alt ? keys_alt : keys;
    e = cudaMemsetAsync(indeg, 0, sizeof(int32_t) * P, s);
    if (e != cudaSuccess) return e;
    k_node_links<<<g2, 256, 0, s>>>(sorted, n2, succ, indeg); note_launch();
    k_frontier<<<1, 1024, 0, s>>>(P, succ, indeg, batch, fa, fb, nb); note_launch();
    k_batch_order<<<1, 1024, 0, s>>>(P, batch, nb, order, boff); note_launch();
    return cudaGetLastError();
}
