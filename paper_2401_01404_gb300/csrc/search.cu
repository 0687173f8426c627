// search.cu -- FindBest (Algorithm 3) over FindKNN by NNDescent (Algorithm 4)
// or exhaustive scoring, on the GPU.
//
// NNDescent, GPU form.  Every node owns its k-list (kept sorted by d; App. B
// notes that the per-node list updates need no synchronisation).  One
// iteration:
//   1. U = the undirected version of G: each node's k out-neighbours plus at
//      most k of its in-neighbours, sampled afresh every iteration (the cap on
//      second neighbours of Sec. III);
//   2. candidates of x: second neighbours v in U(U(x)), v != x, deduplicated
//      in shared memory, minus x's own list.  A path x - j - v whose reverse
//      v - j - x exists too (x in U(j) and j in U(v)) is taken from its smaller
//      end only, so that the pair is scored once; a path without its reverse
//      (U is not symmetric when in-neighbours are sampled) is taken from x
//      whatever the order, as Algorithm 4 has each node search all its own
//      second neighbours.  A path is taken only if one of its two edges is new
//      since the last iteration: an undirected edge {x, y} is new when a list
//      entry between x and y is new, or when one of them took the other's entry
//      as an in-edge for the first time since the previous iteration (so no
//      path through a once-unsampled in-edge is skipped for good).  This plays
//      the role of the score cache of App. B: a pair reached along the same
//      path is scored once;
//   3. each canonical candidate pair is scored once (the exact gain) and
//      offered to both endpoints if it beats their worst entry;
//   4. each list becomes the best k of (old list u offers), old entries winning
//      ties (Algorithm 4 replaces only on strict improvement); Delta counts the
//      entries that are new.
// The loop stops when Delta/(k|S|) < eps or after the iteration cap.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <cmath>

#include "common.cuh"
#include "proposal.cuh"
#include "search.cuh"

namespace {

constexpr int NND_MAX_K = 64;  // list capacity handled by the merge (two entries per lane)

__device__ __forceinline__ bool key_less(float da, uint32_t ra, float db, uint32_t rb) {
    return da < db || (da == db && ra < rb);
}

// random lists: klen[x] distinct ids != x (every other node when klen >= n-1),
// -1 in the unused slots of the capacity K
__global__ void k_knn_init(int n, int K, const int32_t *klen, uint64_t seed, int32_t *ids) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    int32_t *L = ids + (int64_t)x * K;
    const int k = klen[x];
    for (int r = k; r < K; ++r) L[r] = -1;
    int q = 0;
    if (k >= n - 1) {
        for (int y = 0; y < n && q < k; ++y)
            if (y != x) L[q++] = y;
        return;
    }
    uint64_t ctr = 0;
    while (q < k && ctr < 64ull * (uint64_t)k) {
        uint64_t r = mix64(seed ^ mix64(((uint64_t)x << 32) ^ ctr++));
        int y = (int)(r % (uint64_t)n);
        if (y == x) continue;
        bool dup = false;
        for (int p = 0; p < q; ++p) dup |= L[p] == y;
        if (!dup) L[q++] = y;
    }
    for (int y = 0; q < k && y < n; ++y) {
        if (y == x) continue;
        bool dup = false;
        for (int p = 0; p < q; ++p) dup |= L[p] == y;
        if (!dup) L[q++] = y;
    }
}

__global__ void k_list_pairs(int n, int K, const int32_t *ids, const int32_t *klen, int32_t *pairs, int32_t *seg_node,
                             int64_t *seg_start, int32_t *seg_count) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * K) return;
    const int x = (int)(e / K);
    pairs[2 * e] = x;
    pairs[2 * e + 1] = ids[e] >= 0 ? ids[e] : x;
    if (e % K == 0) {
        seg_node[x] = x;
        seg_start[x] = e;
        seg_count[x] = klen[x];
    }
}

// sort each initial list by (d, pair hash); every entry is new; unused slots
// hold id -1 and d = +inf
__global__ void k_sort_lists(int n, int K, const int32_t *klen, const int32_t *gid, int32_t *ids, float *dd,
                             uint8_t *isnew) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    int32_t *L = ids + (int64_t)x * K;
    float *D = dd + (int64_t)x * K;
    const int k = klen[x];
    for (int r = k; r < K; ++r) D[r] = INFINITY;
    for (int a = 1; a < k; ++a) {
        int32_t id = L[a];
        float d = D[a];
        uint32_t r = (uint32_t)(mix64(pair_key(gid[x], gid[id])) >> 33);
        int b = a - 1;
        while (b >= 0) {
            uint32_t rb = (uint32_t)(mix64(pair_key(gid[x], gid[L[b]])) >> 33);
            if (!key_less(d, r, D[b], rb)) break;
            L[b + 1] = L[b];
            D[b + 1] = D[b];
            --b;
        }
        L[b + 1] = id;
        D[b + 1] = d;
    }
    for (int a = 0; a < K; ++a) isnew[(int64_t)x * K + a] = a < k;
}

__global__ void k_in_count(int64_t nk, const int32_t *ids, int32_t *indeg) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nk && ids[e] >= 0) atomicAdd(&indeg[ids[e]], 1);
}

__global__ void k_i32_to_i64(const int32_t *a, int64_t *b, int64_t n) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) b[e] = a[e];
}

__global__ void k_in_fill(int64_t nk, const int32_t *ids, const int64_t *inoff, int32_t *cursor, int32_t *in_e) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nk) return;
    int y = ids[e];
    if (y < 0) return;
    int pos = atomicAdd(&cursor[y], 1);
    in_e[inoff[y] + pos] = (int32_t)e;
}

// U(x) = out(x) u (at most in_cap in-neighbours, smallest random priority)
// an in-edge (slot e of a list) counts as new when its entry is new or when it
// was not in U in the previous iteration (in_last[e] holds the iteration that
// last took it, in_fresh[e] the iteration that took it without the one before)
__global__ void k_build_U(int n, int K, const int32_t *klen, int in_cap, int Ucap, const unsigned long long *seed0,
                          const int *iter,
                          const int32_t *ids,
                          const uint8_t *isnew, const int64_t *inoff, const int32_t *indeg, const int32_t *in_e,
                          int32_t *in_last, int32_t *in_fresh, int32_t *U, uint8_t *Uf, int32_t *Udeg) {
    extern __shared__ int32_t sm[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int x = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (x >= n) return;
    const uint64_t seed = mix64(*seed0 ^ (0x5bd1e995ull * (uint64_t)*iter));
    int32_t *sid = sm + wib * 2 * Ucap;
    int32_t *sfl = sid + Ucap;
    const int k = klen[x];
    for (int r = lane; r < k; r += 32) {
        sid[r] = ids[(int64_t)x * K + r];
        sfl[r] = isnew[(int64_t)x * K + r];
    }
    __syncwarp();
    int d = k;
    const int64_t b = inoff[x];
    const int deg = indeg[x];
    const int take = deg < in_cap ? deg : in_cap;
    uint64_t last = 0;
    for (int s = 0; s < take; ++s) {
        int e_sel;
        if (deg <= in_cap) {
            e_sel = in_e[b + s];
        } else {
            uint64_t best = ~0ull;
            int best_e = -1;
            for (int q = lane; q < deg; q += 32) {
                int e = in_e[b + q];
                uint64_t pr = mix64(seed ^ ((uint64_t)x << 32) ^ (uint64_t)(e / K));
                if ((s == 0 || pr > last) && (pr < best || (pr == best && e < best_e))) {
                    best = pr;
                    best_e = e;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                uint64_t ob = __shfl_xor_sync(0xffffffffu, best, o);
                int oe = __shfl_xor_sync(0xffffffffu, best_e, o);
                if (ob < best || (ob == best && oe < best_e)) {
                    best = ob;
                    best_e = oe;
                }
            }
            if (best_e < 0) break;
            last = best;
            e_sel = best_e;
        }
        const int y = e_sel / K;
        const int it = *iter, prev = in_last[e_sel];
        const int fl = isnew[e_sel] || prev != it - 1;
        if (lane == 0) {
            in_last[e_sel] = it;
            if (prev != it - 1) in_fresh[e_sel] = it;
        }
        int found = -1;
        for (int r = lane; r < k; r += 32)
            if (sid[r] == y) found = r;
        for (int o = 16; o > 0; o >>= 1) found = max(found, __shfl_xor_sync(0xffffffffu, found, o));
        if (lane == 0) {
            if (found >= 0) {
                if (fl) sfl[found] = 1;
            } else {
                sid[d] = y;
                sfl[d] = fl;
            }
        }
        if (found < 0) ++d;
        __syncwarp();
    }
    for (int r = lane; r < d; r += 32) {
        U[(int64_t)x * Ucap + r] = sid[r];
        Uf[(int64_t)x * Ucap + r] = (uint8_t)sfl[r];
    }
    if (lane == 0) Udeg[x] = d;
}

// per U entry (x, a) -> y: Usym = whether x is in U(y), and Uf becomes the
// undirected edge's flag: new if any list entry between x and y (x -> y at
// position a < k_x, y -> x wherever x sits in y's list) is new or was taken as
// an in-edge for the first time this iteration
__global__ void k_U_sym(int n, int K, const int32_t *klen, int Ucap, const int *iter, const int32_t *ids,
                        const uint8_t *isnew, const int32_t *in_fresh, const int32_t *U, uint8_t *Uf,
                        const int32_t *Udeg, uint8_t *Usym) {
    const int lane = threadIdx.x & 31;
    const int x = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (x >= n) return;
    const int it = *iter, degx = Udeg[x], kx = klen[x];
    for (int a = lane; a < degx; a += 32) {
        const int y = U[(int64_t)x * Ucap + a];
        bool sym = false;
        const int degy = Udeg[y];
        for (int b = 0; b < degy && !sym; ++b) sym = U[(int64_t)y * Ucap + b] == x;
        uint8_t f = Uf[(int64_t)x * Ucap + a];
        if (a < kx) f |= in_fresh[(int64_t)x * K + a] == it;
        const int ky = klen[y];
        for (int r = 0; r < ky; ++r) {
            const int64_t e = (int64_t)y * K + r;
            if (ids[e] == x) f |= isnew[e] | (uint8_t)(in_fresh[e] == it);
        }
        Uf[(int64_t)x * Ucap + a] = f;
        Usym[(int64_t)x * Ucap + a] = sym;
    }
}

__device__ __forceinline__ int sh_insert(int32_t *h, int hmask, int32_t v) {
    uint32_t s = ((uint32_t)v * 2654435761u) & (uint32_t)hmask;
    for (int probe = 0; probe <= hmask; ++probe) {
        int32_t prev = atomicCAS(&h[s], -1, v);
        if (prev == -1) return 1;
        if (prev == v) return 0;
        s = (s + 1) & (uint32_t)hmask;
    }
    return -1;
}

// candidates of x: v in U(U(x)), v != x, not in x's list, reached by a new edge
// (paths with a reverse path from the smaller end only)
__global__ void k_gen(int n, int K, const int32_t *klen, int Ucap, const int32_t *U, const uint8_t *Uf,
                      const uint8_t *Usym, const int32_t *Udeg, const int32_t *ids, int hsize, int lcap,
                      int32_t *cand, int64_t cap,
                      unsigned long long *counter, unsigned long long *cnt, int32_t *seg_node, int64_t *seg_start,
                      int32_t *seg_count) {
    extern __shared__ int32_t sm[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int x = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (x >= n) return;
    int32_t *h = sm + wib * (hsize + lcap + 1);
    int32_t *list = h + hsize;
    int32_t *wcount = list + lcap;
    for (int s = lane; s < hsize; s += 32) h[s] = -1;
    if (lane == 0) *wcount = 0;
    __syncwarp();
    for (int r = lane; r < klen[x]; r += 32) sh_insert(h, hsize - 1, ids[(int64_t)x * K + r]);
    __syncwarp();
    const int degx = Udeg[x];
    bool overflow = false, dropped = false;
    for (int a = 0; a < degx; ++a) {
        const int j = U[(int64_t)x * Ucap + a];
        const int fxj = Uf[(int64_t)x * Ucap + a];
        const int sxj = Usym[(int64_t)x * Ucap + a];
        const int degj = Udeg[j];
        for (int b = lane; b < degj; b += 32) {
            const int v = U[(int64_t)j * Ucap + b];
            const int fjv = Uf[(int64_t)j * Ucap + b];
            // from the smaller end when the reverse path v - j - x exists, else from x
            const bool mine = v > x || !(sxj && Usym[(int64_t)j * Ucap + b]);
            if (v != x && (fxj | fjv) && mine) {
                // past the per-node cap the remaining second neighbours are
                // skipped this iteration (the paper's cap on the second-neighbour
                // loop); they stay reachable in later iterations
                int r = sh_insert(h, hsize - 1, v);
                if (r == 1) {
                    int pos = atomicAdd(wcount, 1);
                    if (pos < lcap) list[pos] = v;
                    else dropped = true;
                } else if (r < 0)
                    dropped = true;
            }
        }
    }
    __syncwarp();
    int count = min(*wcount, lcap);
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(counter, (unsigned long long)count);
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((int64_t)base + count > cap) {
        overflow = true;
        count = (int64_t)base >= cap ? 0 : (int)(cap - (int64_t)base);
    }
    for (int q = lane; q < count; q += 32) {
        cand[2 * (base + q)] = x;
        cand[2 * (base + q) + 1] = list[q];
    }
    if (lane == 0) {
        seg_node[x] = x;
        seg_start[x] = (int64_t)base;
        seg_count[x] = count;
    }
    if (__any_sync(0xffffffffu, overflow) && lane == 0) atomicOr(&cnt[CNT_ERR], (unsigned long long)ERR_OVERFLOW);
    if (__any_sync(0xffffffffu, dropped) && lane == 0) atomicAdd(&cnt[CNT_SCRATCH3], 1ull);
}

// offer each scored candidate to both endpoints if it beats their worst entry
__global__ void k_offer(const unsigned long long *Pdev, int64_t Pcap, const int32_t *cand, const float *dc, int K,
                        const int32_t *klen, const float *knn_d, int32_t *ot, int32_t *ov, float *od,
                        unsigned long long *counter, int64_t cap, unsigned long long *dropped) {
    const int64_t P = min((int64_t)*Pdev, Pcap);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < P; q += (int64_t)gridDim.x * blockDim.x) {
    const int x = cand[2 * q], v = cand[2 * q + 1];
    const float d = dc[q];
    const bool to_x = d < knn_d[(int64_t)x * K + klen[x] - 1];
    const bool to_v = d < knn_d[(int64_t)v * K + klen[v] - 1];
    int nn = (int)to_x + (int)to_v;
    if (!nn) continue;
    unsigned long long pos = atomicAdd(counter, (unsigned long long)nn);
    if ((int64_t)(pos + nn) > cap) {  // offer buffer full: the offer is dropped this iteration
        atomicAdd(dropped, 1ull);
        // slots below cap that this offer reserved stay marked empty
        for (int64_t s = (int64_t)pos; s < (int64_t)pos + nn && s < cap; ++s) ot[s] = -1;
        continue;
    }
    if (to_x) {
        ot[pos] = x;
        ov[pos] = v;
        od[pos] = d;
        ++pos;
    }
    if (to_v) {
        ot[pos] = v;
        ov[pos] = x;
        od[pos] = d;
    }
    }
}

__global__ void k_count_targets(const unsigned long long *Pdev, int64_t Pcap, const int32_t *ot, int32_t *cntv) {
    const int64_t P = min((int64_t)*Pdev, Pcap);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < P; q += (int64_t)gridDim.x * blockDim.x)
        if (ot[q] >= 0) atomicAdd(&cntv[ot[q]], 1);
}

__global__ void k_scatter_offers(const unsigned long long *Pdev, int64_t Pcap, const int32_t *ot, const int32_t *ov,
                                 const float *od, const int64_t *off, int32_t *cursor, int32_t *sv, float *sd) {
    const int64_t P = min((int64_t)*Pdev, Pcap);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < P; q += (int64_t)gridDim.x * blockDim.x) {
        const int x = ot[q];
        if (x < 0) continue;
        const int pos = atomicAdd(&cursor[x], 1);
        sv[off[x] + pos] = ov[q];
        sd[off[x] + pos] = od[q];
    }
}

// iteration counter of a (possibly graph-replayed) NNDescent loop
__global__ void k_next_iter(int *it) { *it += 1; }

// The stopping test of Algorithm 4 on the device, at the end of an iteration of
// the graph's WHILE loop: go on while more than eps of the list entries changed
// (k_merge's count), fewer than max_iters iterations ran and no error was
// raised.  Also adds up what the host loop reads after each iteration:
// acc[0] candidates scored, acc[1] offers dropped for want of space.
__global__ void k_nnd_continue(cudaGraphConditionalHandle h, const unsigned long long *cnt, const int *iter,
                               int max_iters, double klen_sum, double eps, unsigned long long cand_cap,
                               unsigned long long *acc) {
    const unsigned long long ncand = cnt[CNT_SCRATCH0] < cand_cap ? cnt[CNT_SCRATCH0] : cand_cap;
    acc[0] += ncand;
    acc[1] += cnt[CNT_SCRATCH3];
    const bool converged = (double)cnt[CNT_SCRATCH2] / klen_sum < eps;
    const bool go = !converged && *iter < max_iters && cnt[CNT_ERR] == 0;
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

// best k of (old list u offers) per node; old entries win ties.  A warp holds
// the list, entry r in lane r (slot A) and entry r + 32 in lane r (slot B), so
// lists of up to 64 entries; node x keeps klen[x] of them.
__global__ void k_merge(int n, int K, const int32_t *klen, const int32_t *gid, int32_t *ids, float *dd, uint8_t *isnew,
                        const int64_t *off, const int32_t *sv, const float *sd, unsigned long long *delta) {
    const int lane = threadIdx.x & 31;
    const int x = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (x >= n) return;
    const int k = klen[x];
    int idA = -1, idB = -1;
    float dA = INFINITY, dB = INFINITY;
    uint32_t rA = 0xffffffffu, rB = 0xffffffffu;
    if (lane < k) {
        idA = ids[(int64_t)x * K + lane];
        dA = dd[(int64_t)x * K + lane];
        rA = 0;
    }
    if (lane + 32 < k) {
        idB = ids[(int64_t)x * K + lane + 32];
        dB = dd[(int64_t)x * K + lane + 32];
        rB = 0;
    }
    const int gx = gid[x];
    const int last = k - 1;
    for (int64_t q = off[x]; q < off[x + 1]; ++q) {
        const int v = sv[q];
        const float dv = sd[q];
        if (__any_sync(0xffffffffu, idA == v || idB == v)) continue;
        const uint32_t rv = 1u + (uint32_t)(mix64(pair_key(gx, gid[v])) >> 33);
        const float dw = last < 32 ? __shfl_sync(0xffffffffu, dA, last) : __shfl_sync(0xffffffffu, dB, last - 32);
        const uint32_t rw = last < 32 ? __shfl_sync(0xffffffffu, rA, last) : __shfl_sync(0xffffffffu, rB, last - 32);
        if (!key_less(dv, rv, dw, rw)) continue;
        const int pos = __popc(__ballot_sync(0xffffffffu, lane < k && key_less(dA, rA, dv, rv))) +
                        __popc(__ballot_sync(0xffffffffu, lane + 32 < k && key_less(dB, rB, dv, rv)));
        // shift entries at positions >= pos one place up; the carry into slot B
        // lane 0 is slot A lane 31
        const int idA_up = __shfl_up_sync(0xffffffffu, idA, 1), idB_up = __shfl_up_sync(0xffffffffu, idB, 1);
        const float dA_up = __shfl_up_sync(0xffffffffu, dA, 1), dB_up = __shfl_up_sync(0xffffffffu, dB, 1);
        const uint32_t rA_up = __shfl_up_sync(0xffffffffu, rA, 1), rB_up = __shfl_up_sync(0xffffffffu, rB, 1);
        const int idA31 = __shfl_sync(0xffffffffu, idA, 31);
        const float dA31 = __shfl_sync(0xffffffffu, dA, 31);
        const uint32_t rA31 = __shfl_sync(0xffffffffu, rA, 31);
        const int pB = lane + 32;
        if (pB < k && pB > pos) {
            idB = lane == 0 ? idA31 : idB_up;
            dB = lane == 0 ? dA31 : dB_up;
            rB = lane == 0 ? rA31 : rB_up;
        }
        if (pB == pos) {
            idB = v;
            dB = dv;
            rB = rv;
        }
        if (lane < k && lane > pos) {
            idA = idA_up;
            dA = dA_up;
            rA = rA_up;
        }
        if (lane == pos) {
            idA = v;
            dA = dv;
            rA = rv;
        }
    }
    if (lane < K) {
        ids[(int64_t)x * K + lane] = lane < k ? idA : -1;
        dd[(int64_t)x * K + lane] = lane < k ? dA : INFINITY;
        isnew[(int64_t)x * K + lane] = lane < k && rA != 0;
    }
    if (lane + 32 < K) {
        ids[(int64_t)x * K + lane + 32] = lane + 32 < k ? idB : -1;
        dd[(int64_t)x * K + lane + 32] = lane + 32 < k ? dB : INFINITY;
        isnew[(int64_t)x * K + lane + 32] = lane + 32 < k && rB != 0;
    }
    const int nnew = __popc(__ballot_sync(0xffffffffu, lane < k && rA != 0)) +
                     __popc(__ballot_sync(0xffffffffu, lane + 32 < k && rB != 0));
    if (lane == 0 && nnew) atomicAdd(delta, (unsigned long long)nnew);
}

// D+ selection keys: (d, hash of the unordered pair); equal pairs stay adjacent
__global__ void k_edge_keys(int n, int k, const int32_t *gid, const int32_t *ids, const float *dd,
                            unsigned long long *keys, uint32_t *vals) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * k) return;
    const int x = (int)(e / k), y = ids[e];
    if (y < 0) {  // unused slot: after every edge
        keys[e] = ~0ull;
        vals[e] = (uint32_t)e;
        return;
    }
    const uint32_t hsh = (uint32_t)(mix64(pair_key(gid[x], gid[y])) >> 32);
    keys[e] = ((unsigned long long)float_key(dd[e]) << 32) | hsh;
    vals[e] = (uint32_t)e;
}

// D = unique undirected pairs of D+ (set insertion), written as global pairs
__global__ void k_take_D(int64_t nDp, int k, const int32_t *gid, const int32_t *ids, const float *dd,
                         const uint32_t *sorted_e, unsigned long long *dset, uint64_t dmask, int32_t *Dp,
                         float *Dd, unsigned long long *counter, unsigned long long *cnt) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nDp) return;
    const uint32_t e = sorted_e[q];
    const int x = (int)(e / (uint32_t)k), y = ids[e];
    const int a = gid[x], b = gid[y];
    const int r = set_insert(dset, dmask, pair_key(a, b));
    if (r < 0) atomicOr(&cnt[CNT_ERR], (unsigned long long)ERR_TABLE_FULL);
    if (r != 1) return;
    unsigned long long pos = atomicAdd(counter, 1ull);
    Dp[2 * pos] = a < b ? a : b;
    Dp[2 * pos + 1] = a < b ? b : a;
    Dd[pos] = dd[e];
}

// D+ of a small level (n k <= SEL_SMALL keys) in one CTA of 1024 threads,
// instead of a full sort: the want-th smallest key T, digit by digit from the
// top (eight 8-bit histogram passes over keys that sit in L2 at this size),
// then every key below T and the lowest-index ones of the keys equal to T,
// which are the first `want` keys of a stable sort.  Writes their edge
// indices to out_e[0 .. want), in no particular order (D is a set).  Each
// thread keeps SEL_BATCH loads in flight; a key equals T only for the two
// directed copies of one pair (the key holds d and a hash of the pair), so the
// equal keys go to a small buffer and are ordered by index at the end (more
// than SEL_EQ of them, and the compaction runs again in index order).
constexpr int64_t SEL_SMALL = 1 << 16;
constexpr int SEL_BATCH = 8, SEL_EQ = 256;
__global__ void __launch_bounds__(1024) k_select_small(int64_t nk, int64_t want, const unsigned long long *keys,
                                                       uint32_t *out_e) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t wcount[32];
    __shared__ uint32_t eqbuf[SEL_EQ];
    __shared__ unsigned long long s_prefix, s_out;
    __shared__ long long s_rem, s_eq;
    __shared__ uint32_t s_neq;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    constexpr int NT = 1024;
    if (tid == 0) {
        s_prefix = 0;
        s_rem = want;
        s_out = 0;
        s_eq = 0;
        s_neq = 0;
    }
    unsigned long long mask = 0;
    __syncthreads();
    for (int pass = 7; pass >= 0; --pass) {
        if (tid < 256) hist[tid] = 0;
        __syncthreads();
        const unsigned long long prefix = s_prefix;
        const int sh = 8 * pass;
        for (int64_t e0 = 0; e0 < nk; e0 += (int64_t)NT * SEL_BATCH) {
            unsigned long long kk[SEL_BATCH];
#pragma unroll
            for (int u = 0; u < SEL_BATCH; ++u) {
                const int64_t e = e0 + (int64_t)u * NT + tid;
                kk[u] = e < nk ? keys[e] : ~0ull;
            }
#pragma unroll
            for (int u = 0; u < SEL_BATCH; ++u) {
                const int64_t e = e0 + (int64_t)u * NT + tid;
                const uint32_t dg = (e < nk && (kk[u] & mask) == prefix) ? (uint32_t)(kk[u] >> sh) & 255u : 256u;
                // the common case in the leading bytes: the whole warp holds one digit
                const uint32_t d0 = __shfl_sync(0xffffffffu, dg, 0);
                if (__all_sync(0xffffffffu, dg == d0)) {
                    if (lane == 0 && d0 < 256u) atomicAdd(&hist[d0], 32u);
                } else if (dg < 256u) {
                    atomicAdd(&hist[dg], 1u);
                }
            }
        }
        __syncthreads();
        if (w == 0) {  // the bucket that holds the rem-th key of the prefix: lane l scans buckets 8l .. 8l + 7
            uint32_t c8[8], sum = 0;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                c8[u] = hist[8 * lane + u];
                sum += c8[u];
            }
            uint32_t incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const long long rem = s_rem;
            long long acc = (long long)(incl - sum);
            if (acc < rem && rem <= (long long)incl) {
                int bk = 8 * lane + 7;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (acc + (long long)c8[u] >= rem) {
                        bk = 8 * lane + u;
                        break;
                    }
                    acc += c8[u];
                }
                s_rem = rem - acc;
                s_prefix = prefix | ((unsigned long long)bk << sh);
            }
        }
        mask |= 255ull << sh;
        __syncthreads();
    }
    const unsigned long long T = s_prefix;
    const long long take_eq = s_rem;  // keys equal to T to take, lowest indices first
    // one pass: keys below T straight to the output, keys equal to T to the buffer
    for (int64_t e0 = 0; e0 < nk; e0 += (int64_t)NT * SEL_BATCH) {
        unsigned long long kk[SEL_BATCH];
#pragma unroll
        for (int u = 0; u < SEL_BATCH; ++u) {
            const int64_t e = e0 + (int64_t)u * NT + tid;
            kk[u] = e < nk ? keys[e] : ~0ull;
        }
#pragma unroll
        for (int u = 0; u < SEL_BATCH; ++u) {
            const int64_t e = e0 + (int64_t)u * NT + tid;
            const bool lt = e < nk && kk[u] < T;
            const uint32_t bt = __ballot_sync(0xffffffffu, lt);
            unsigned long long base = 0;
            if (lane == 0 && bt) base = atomicAdd(&s_out, (unsigned long long)__popc(bt));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (lt) out_e[base + __popc(bt & ((1u << lane) - 1u))] = (uint32_t)e;
            if (e < nk && kk[u] == T) {
                const uint32_t q = atomicAdd(&s_neq, 1u);
                if (q < SEL_EQ) eqbuf[q] = (uint32_t)e;
            }
        }
    }
    __syncthreads();
    const uint32_t neq = s_neq;
    if (neq <= (uint32_t)SEL_EQ) {
        // the take_eq lowest indices of the buffer (at most SEL_EQ entries): rank by count
        for (uint32_t q = tid; q < neq; q += NT) {
            const uint32_t e = eqbuf[q];
            uint32_t r = 0;
            for (uint32_t o = 0; o < neq; ++o) r += eqbuf[o] < e;
            if ((long long)r < take_eq) out_e[(want - take_eq) + r] = e;
        }
        return;
    }
    // many equal keys (hash collisions at the cut): their lowest indices in index order
    for (int64_t e0 = 0; e0 < nk; e0 += NT) {
        const int64_t e = e0 + tid;
        const bool eq = e < nk && keys[e] == T;
        const uint32_t be = __ballot_sync(0xffffffffu, eq);
        if (lane == 0) wcount[w] = (uint32_t)__popc(be);
        __syncthreads();
        long long before = s_eq + __popc(be & ((1u << lane) - 1u));
        for (int u = 0; u < w; ++u) before += wcount[u];
        if (eq && before < take_eq) out_e[(want - take_eq) + before] = (uint32_t)e;
        __syncthreads();
        if (tid == 0) {
            long long tot = 0;
            for (int u = 0; u < 32; ++u) tot += wcount[u];
            s_eq += tot;
        }
        __syncthreads();
    }
}

// The final list of a small result set (P <= FIN_SMALL pairs) in one CTA: a
// bitonic sort in shared memory by (d, i, j, position) -- the order that the
// stable radix sorts give -- then the first of each run of equal pairs, the
// m best of them to outp/outd and their number to *count.
constexpr int64_t FIN_SMALL = 8192;
struct FinItem {
    uint32_t dk;  // float_key(d)
    int32_t i, j;
    uint32_t q;   // position in the input
};
__device__ __forceinline__ bool fin_less(const FinItem &a, const FinItem &b) {
    if (a.dk != b.dk) return a.dk < b.dk;
    if (a.i != b.i) return a.i < b.i;
    if (a.j != b.j) return a.j < b.j;
    return a.q < b.q;
}
__global__ void __launch_bounds__(1024) k_finish_small(int P, int np2, int64_t m, const int32_t *pairs, const float *dd,
                                                       int32_t *outp, float *outd, unsigned long long *count) {
    extern __shared__ __align__(16) FinItem it[];
    __shared__ uint32_t wcount[32];
    __shared__ long long s_base;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int q = tid; q < np2; q += blockDim.x) {
        FinItem x;
        if (q < P) {
            x.dk = float_key(dd[q]);
            x.i = pairs[2 * q];
            x.j = pairs[2 * q + 1];
            x.q = (uint32_t)q;
        } else {  // after every real entry
            x.dk = 0xffffffffu;
            x.i = 0x7fffffff;
            x.j = 0x7fffffff;
            x.q = 0xffffffffu;
        }
        it[q] = x;
    }
    if (tid == 0) s_base = 0;
    __syncthreads();
    for (int size = 2; size <= np2; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = tid; t < np2 / 2; t += blockDim.x) {
                const int lo = 2 * t - (t & (stride - 1)), hi = lo + stride;
                const bool up = (lo & size) == 0;
                const FinItem a = it[lo], b = it[hi];
                if (up ? fin_less(b, a) : fin_less(a, b)) {
                    it[lo] = b;
                    it[hi] = a;
                }
            }
            __syncthreads();
        }
    for (int q0 = 0; q0 < P; q0 += blockDim.x) {
        const int q = q0 + tid;
        const bool first = q < P && (q == 0 || it[q].i != it[q - 1].i || it[q].j != it[q - 1].j);
        const uint32_t bf = __ballot_sync(0xffffffffu, first);
        if (lane == 0) wcount[w] = (uint32_t)__popc(bf);
        __syncthreads();
        long long pos = s_base + __popc(bf & ((1u << lane) - 1u));
        for (int u = 0; u < w; ++u) pos += wcount[u];
        if (first && pos < m) {
            const FinItem x = it[q];
            outp[2 * pos] = x.i;
            outp[2 * pos + 1] = x.j;
            outd[pos] = dd[x.q];
        }
        __syncthreads();
        if (tid == 0) {
            long long tot = 0;
            for (int u = 0; u < 32; ++u) tot += wcount[u];
            s_base += tot;
        }
        __syncthreads();
    }
    if (tid == 0) *count = (unsigned long long)(s_base < m ? s_base : m);
}

// saturated nodes: every out-edge in D
__global__ void k_saturated(int n, int k, const int32_t *klen, const int32_t *gid, const int32_t *ids,
                            const unsigned long long *dset, uint64_t dmask, int64_t *flag) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    bool all = true;
    for (int r = 0; r < klen[x] && all; ++r)
        all = set_contains(dset, dmask, pair_key(gid[x], gid[ids[(int64_t)x * k + r]]));
    flag[x] = all ? 1 : 0;
}

__global__ void k_compact_nodes(int n, const int64_t *flag, const int64_t *pos, const int32_t *gid, int32_t *out) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < n && flag[x]) out[pos[x]] = gid[x];
}

// all pairs x < y of a node set of size n, lexicographic
__device__ __forceinline__ void tri_unrank(int64_t e, int64_t n, int &x, int &y) {
    // rows x hold n-1-x pairs; row start s(x) = x(2n - x - 1)/2
    double nn = (double)n;
    double disc = (2 * nn - 1) * (2 * nn - 1) - 8.0 * (double)e;
    int64_t xx = (int64_t)floor(((2 * nn - 1) - sqrt(fmax(disc, 0.0))) / 2);
    if (xx < 0) xx = 0;
    if (xx > n - 2) xx = n - 2;
    auto start = [&](int64_t r) { return r * (2 * n - r - 1) / 2; };
    while (xx > 0 && start(xx) > e) --xx;
    while (xx < n - 2 && start(xx + 1) <= e) ++xx;
    x = (int)xx;
    y = (int)(e - start(xx) + xx + 1);
}

__global__ void k_all_pairs(int64_t n, int64_t np, int32_t *pairs) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= np) return;
    int x, y;
    tri_unrank(e, n, x, y);
    pairs[2 * e] = x;
    pairs[2 * e + 1] = y;
}

// keys (d, lexicographic rank): ascending order is (d, i, j)
__global__ void k_rank_keys(int64_t np, const float *dd, unsigned long long *keys, uint32_t *vals) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= np) return;
    keys[e] = ((unsigned long long)float_key(dd[e]) << 32) | (uint32_t)e;
    vals[e] = (uint32_t)e;
}

__global__ void k_gather_pairs(int64_t m, const uint32_t *sel, const int32_t *pairs_local, const int32_t *gid,
                               const float *dd, int32_t *outp, float *outd) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= m) return;
    const uint32_t e = sel[q];
    int a = pairs_local[2 * (int64_t)e], b = pairs_local[2 * (int64_t)e + 1];
    if (gid) {
        a = gid[a];
        b = gid[b];
    }
    outp[2 * q] = a < b ? a : b;
    outp[2 * q + 1] = a < b ? b : a;
    outd[q] = dd[e];
}

// dense symmetric d matrix of a node set (diagonal +inf) from all-pairs scores
__global__ void k_dense_fill(int64_t n, int64_t np, const int32_t *pairs, const float *dd, float *Dm) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) Dm[e * n + e] = INFINITY;
    if (e >= np) return;
    const int x = pairs[2 * e], y = pairs[2 * e + 1];
    Dm[(int64_t)x * n + y] = dd[e];
    Dm[(int64_t)y * n + x] = dd[e];
}

// exact k smallest of each row by (d, column): radix select on the float key,
// then an ordered gather; one block per row
__global__ void __launch_bounds__(256) k_row_topk(int64_t n, int k, const float *Dm, int32_t *ids, float *dd) {
    __shared__ int hist[256];
    __shared__ uint32_t s_prefix;
    __shared__ int s_rem;
    __shared__ int scan[257];
    const int64_t x = blockIdx.x;
    const float *row = Dm + x * n;
    uint32_t prefix = 0;
    int rem = k;
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        hist[threadIdx.x] = 0;
        __syncthreads();
        const uint32_t hmask = pass == 0 ? 0u : (0xffffffffu << (32 - 8 * pass));
        for (int64_t y = threadIdx.x; y < n; y += blockDim.x) {
            uint32_t kk = float_key(row[y]);
            if ((kk & hmask) == (prefix & hmask)) atomicAdd(&hist[(kk >> shift) & 0xff], 1);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = 0, dsel = 255;
            for (int dg = 0; dg < 256; ++dg) {
                if (acc + hist[dg] >= rem) {
                    dsel = dg;
                    break;
                }
                acc += hist[dg];
            }
            s_prefix = prefix | ((uint32_t)dsel << shift);
            s_rem = rem - acc;
        }
        __syncthreads();
        prefix = s_prefix;
        rem = s_rem;
        __syncthreads();
    }
    // prefix = key of the k-th smallest; take all keys < prefix and the first
    // `rem` keys == prefix in column order
    const int64_t chunk = (n + blockDim.x - 1) / blockDim.x;
    const int64_t y0 = threadIdx.x * chunk, y1 = min(n, y0 + chunk);
    int nl = 0, ne = 0;
    for (int64_t y = y0; y < y1; ++y) {
        uint32_t kk = float_key(row[y]);
        nl += kk < prefix;
        ne += kk == prefix;
    }
    // exclusive scans of nl and ne (two passes through `scan`)
    scan[threadIdx.x + 1] = nl;
    if (threadIdx.x == 0) scan[0] = 0;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int t = 1; t <= (int)blockDim.x; ++t) scan[t] += scan[t - 1];
    __syncthreads();
    int base_l = scan[threadIdx.x];
    __syncthreads();
    scan[threadIdx.x + 1] = ne;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int t = 1; t <= (int)blockDim.x; ++t) scan[t] += scan[t - 1];
    __syncthreads();
    int base_e = scan[threadIdx.x];
    const int n_less = k - rem;
    int pl = base_l, pe = base_e;
    for (int64_t y = y0; y < y1; ++y) {
        float v = row[y];
        uint32_t kk = float_key(v);
        int slot = -1;
        if (kk < prefix)
            slot = pl++;
        else if (kk == prefix) {
            if (pe < rem) slot = n_less + pe;
            ++pe;
        }
        if (slot >= 0 && slot < k) {
            ids[x * k + slot] = (int32_t)y;
            dd[x * k + slot] = v;
        }
    }
}

__global__ void k_pair_keys(int64_t P, const int32_t *pairs, unsigned long long *keys, uint32_t *vals) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= P) return;
    keys[q] = ((unsigned long long)(uint32_t)pairs[2 * q] << 32) | (uint32_t)pairs[2 * q + 1];
    vals[q] = (uint32_t)q;
}

__global__ void k_d_keys(int64_t P, const uint32_t *perm, const float *dd, unsigned long long *keys,
                         uint32_t *vals) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= P) return;
    keys[q] = float_key(dd[perm[q]]);
    vals[q] = perm[q];
}

// first occurrence flags of equal pairs that are adjacent in `perm` order
__global__ void k_unique_flags(int64_t P, const uint32_t *perm, const int32_t *pairs, int64_t *flag) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= P) return;
    bool first = true;
    if (q > 0) {
        uint32_t a = perm[q], b = perm[q - 1];
        first = !(pairs[2 * (int64_t)a] == pairs[2 * (int64_t)b] && pairs[2 * (int64_t)a + 1] == pairs[2 * (int64_t)b + 1]);
    }
    flag[q] = first ? 1 : 0;
}

__global__ void k_unique_gather(int64_t P, int64_t m, const uint32_t *perm, const int64_t *flag,
                                const int64_t *pos, const int32_t *pairs, const float *dd, int32_t *outp,
                                float *outd) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= P || !flag[q] || pos[q] >= m) return;
    const uint32_t a = perm[q];
    outp[2 * pos[q]] = pairs[2 * (int64_t)a];
    outp[2 * pos[q] + 1] = pairs[2 * (int64_t)a + 1];
    outd[pos[q]] = dd[a];
}

// canonical copy (i < j) of a scored pair list; ids outside [0, n) or i == j
// raise ERR_BAD_VALUE
__global__ void k_canon_pairs(int64_t P, int n, const int32_t *in, const float *din, int32_t *out, float *dout,
                              unsigned long long *cnt) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= P) return;
    const int a = in[2 * q], b = in[2 * q + 1];
    if (a < 0 || a >= n || b < 0 || b >= n || a == b) atomicOr(&cnt[CNT_ERR], (unsigned long long)ERR_BAD_VALUE);
    out[2 * q] = a < b ? a : b;
    out[2 * q + 1] = a < b ? b : a;
    dout[q] = din[q];
}

__global__ void k_iota(int32_t *p, int64_t n) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) p[e] = (int32_t)e;
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

#define CKS(call)                                                \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);   \
    } while (0)

static bool grow(recon_ctx *c, DBuf &b, size_t bytes) {
    if (b.bytes >= bytes) return true;
    if (b.p) {
        cudaStreamSynchronize(c->stream);
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    size_t want = std::max<size_t>(bytes, 256);
    want = want + want / 4;
    if (recon_malloc(&b.p, want) != cudaSuccess) {
        cudaGetLastError();
        set_err(c, RECON_ENOMEM, "device allocation of %zu bytes failed", want);
        return false;
    }
    b.bytes = want;
    return true;
}
// grows b to at least `bytes`, keeping its first `keep` bytes
static bool grow_keep(recon_ctx *c, DBuf &b, size_t bytes, size_t keep) {
    if (b.bytes >= bytes) return true;
    size_t want = std::max<size_t>(bytes, 256);
    want = want + want / 2;
    void *p = nullptr;
    if (recon_malloc(&p, want) != cudaSuccess) {
        cudaGetLastError();
        set_err(c, RECON_ENOMEM, "device allocation of %zu bytes failed", want);
        return false;
    }
    if (b.p) {
        if (keep) cudaMemcpyAsync(p, b.p, std::min(keep, b.bytes), cudaMemcpyDeviceToDevice, c->stream);
        cudaStreamSynchronize(c->stream);
        cudaFree(b.p);
    }
    b.p = p;
    b.bytes = want;
    return true;
}
#define GROW_KEEP(buf, bytes, keep)                                   \
    do {                                                              \
        if (!grow_keep(c, (buf), (bytes), (keep))) return RECON_ENOMEM; \
    } while (0)

#define GROW(buf, bytes)                                   \
    do {                                                   \
        if (!grow(c, (buf), (bytes))) return RECON_ENOMEM; \
    } while (0)

void free_search_bufs(SearchBufs *sb) {
    if (!sb) return;
    for (DBuf *b : sb->all())
        if (b->p) cudaFree(b->p);
    delete sb;
}

static SearchBufs &SB(recon_ctx *c) {
    if (!c->sb) c->sb = new SearchBufs();
    return *c->sb;
}

static unsigned long long *counter(recon_ctx *c, int slot) { return c->cnt + slot; }

static recon_status read_counter(recon_ctx *c, int slot, unsigned long long *out) {
    CKS(cudaMemcpyAsync(c->cnt_host + slot, c->cnt + slot, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                        c->stream));
    CKS(cudaStreamSynchronize(c->stream));
    *out = c->cnt_host[slot];
    return RECON_OK;
}

static recon_status check_err_flags(recon_ctx *c, const char *where) {
    unsigned long long f = 0;
    recon_status st = read_counter(c, CNT_ERR, &f);
    if (st != RECON_OK) return st;
    if (f) {
        CKS(cudaMemsetAsync(c->cnt + CNT_ERR, 0, sizeof(unsigned long long), c->stream));
        if (f & ERR_OVERFLOW) return set_err(c, RECON_ENOMEM, "%s: a search buffer overflowed", where);
        if (f & ERR_TABLE_FULL) return set_err(c, RECON_ENOMEM, "%s: a hash table is full", where);
        if (f & ERR_TIMEOUT) {
            c->broken = true;
            return set_err(c, RECON_ETIMEOUT, "%s: a bounded wait on the device ran out", where);
        }
        return set_err(c, RECON_EINVAL, "%s: device-side check failed (flags %llx)", where, f);
    }
    return RECON_OK;
}

// score `P` pairs (local ids through gid, or global when gid == NULL) into d
recon_status score_pairs_device(recon_ctx *c, const int32_t *pairs, int64_t P, const int32_t *gid, float *d,
                                float *w) {
    if (P <= 0) return RECON_OK;
    cudaEvent_t ea = nullptr, eb = nullptr;
    if (c->opt.timing) {
        for (cudaEvent_t *ev : {&ea, &eb}) {
            if (!c->event_pool.empty()) {
                *ev = c->event_pool.back();
                c->event_pool.pop_back();
            } else
                CKS(cudaEventCreate(ev));
        }
        CKS(cudaEventRecord(ea, c->stream));
    }
    cudaError_t e;
    if (c->model == RECON_ISING)
        e = launch_ising_score(c->iv(), c->W, c->sp(), pairs, P, gid, d, w, c->cnt, c->stream);
    else
        e = launch_gauss_score(c->gv(), c->W, c->sp(), pairs, P, gid, d, w, c->cnt, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "score kernel");
    if (c->opt.timing) {
        CKS(cudaEventRecord(eb, c->stream));
        c->timed.push_back({ea, eb, P});
    }
    c->stats.pair_evals += P;
    return RECON_OK;
}

// score grouped candidates (see k_score_seg); the Gaussian model scores the
// pair list directly
static cudaError_t launch_seg(recon_ctx *c, const int32_t *seg_node, const int64_t *seg_start, const int32_t *seg_count,
                              const int32_t *seg_vbase, int64_t nseg, const int32_t *cand, const int32_t *gid, float *d,
                              int threads, cudaStream_t st = nullptr) {
    if (!st) st = c->stream;
    if (c->model == RECON_ISING)
        return launch_ising_score_seg(c->iv(), c->W, c->sp(), seg_node, seg_start, seg_count, seg_vbase, nseg, cand,
                                      gid, d, c->cnt, threads, st);
    return launch_gauss_score_seg(c->gv(), c->W, c->sp(), seg_node, seg_start, seg_count, seg_vbase, nseg, cand, gid,
                                  d, threads, st);
}

// The block width of the segmented scorer is picked once per context by
// timing each candidate width on the first launch that carries enough work
// (the kernel is idempotent, so the timing runs are ordinary launches).
static recon_status autotune_segments(recon_ctx *c, const int32_t *seg_node, const int64_t *seg_start,
                                      const int32_t *seg_count, const int32_t *seg_vbase, int64_t nseg,
                                      const int32_t *cand, const int32_t *gid, float *d) {
    const int widths[4] = {64, 128, 256, 512};
    cudaEvent_t a, b;
    CKS(cudaEventCreate(&a));
    CKS(cudaEventCreate(&b));
    // one untimed launch (the rows then sit in L2 for every width alike), then two
    // rounds over the widths, each width keeping its best time: one cold or noisy
    // timing would otherwise decide the width for the whole process
    CKS(launch_seg(c, seg_node, seg_start, seg_count, seg_vbase, nseg, cand, gid, d, 256));
    float best_ms[4] = {1e30f, 1e30f, 1e30f, 1e30f};
    for (int round = 0; round < 2; ++round)
        for (int q = 0; q < 4; ++q) {
            CKS(cudaEventRecord(a, c->stream));
            CKS(launch_seg(c, seg_node, seg_start, seg_count, seg_vbase, nseg, cand, gid, d, widths[q]));
            CKS(cudaEventRecord(b, c->stream));
            CKS(cudaEventSynchronize(b));
            float ms = 0.f;
            CKS(cudaEventElapsedTime(&ms, a, b));
            best_ms[q] = std::min(best_ms[q], ms);
        }
    int best_w = 256;
    float best = 1e30f;
    for (int q = 0; q < 4; ++q)
        if (best_ms[q] < best) {
            best = best_ms[q];
            best_w = widths[q];
        }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    c->tuned_threads = best_w;
    c->stats.tuned_threads = best_w;
    return RECON_OK;
}

recon_status score_segments_device(recon_ctx *c, const int32_t *seg_node, const int64_t *seg_start,
                                   const int32_t *seg_count, const int32_t *seg_vbase, int64_t nseg,
                                   const int32_t *cand, int64_t P, const int32_t *gid, float *d) {
    if (P <= 0) return RECON_OK;
    // tuned on a launch with at least 32 candidates per node on average: the initial
    // lists (k per node) favour narrow blocks that the NNDescent iterations (about
    // 100 per node) run slower with
    if (c->tuned_threads == 0 && nseg >= 256 && P >= 32 * nseg) {
        // the width is a property of the kernel, the device and the row length:
        // tuned once per process for each (device, model, Mp)
        static std::mutex mu;
        static std::map<std::tuple<int, int, int64_t>, int> tuned;
        const auto key = std::make_tuple(c->device, c->model, c->Mp);
        {
            std::lock_guard<std::mutex> lk(mu);
            auto it = tuned.find(key);
            if (it != tuned.end()) {
                c->tuned_threads = it->second;
                c->stats.tuned_threads = it->second;
            }
        }
        if (c->tuned_threads == 0) {
            recon_status st = autotune_segments(c, seg_node, seg_start, seg_count, seg_vbase, nseg, cand, gid, d);
            if (st != RECON_OK) return st;
            std::lock_guard<std::mutex> lk(mu);
            tuned[key] = c->tuned_threads;
        }
    }
    const int threads = c->tuned_threads ? c->tuned_threads : 256;
    cudaEvent_t ea = nullptr, eb = nullptr;
    if (c->opt.timing) {
        for (cudaEvent_t *ev : {&ea, &eb}) {
            if (!c->event_pool.empty()) {
                *ev = c->event_pool.back();
                c->event_pool.pop_back();
            } else
                CKS(cudaEventCreate(ev));
        }
        CKS(cudaEventRecord(ea, c->stream));
    }
    cudaError_t e = launch_seg(c, seg_node, seg_start, seg_count, seg_vbase, nseg, cand, gid, d, threads);
    if (e != cudaSuccess) return cuda_fail(c, e, "segmented score kernel");
    if (c->opt.timing) {
        CKS(cudaEventRecord(eb, c->stream));
        c->timed.push_back({ea, eb, P});
    }
    c->stats.pair_evals += P;
    return RECON_OK;
}

// all pairs x < y of n nodes as segments of at most 512 candidates each, in
// lexicographic output order
static recon_status all_pair_segments(recon_ctx *c, int64_t n, int64_t *nseg_out) {
    SearchBufs &S = SB(c);
    std::vector<int32_t> node, cntv, vb;
    std::vector<int64_t> start;
    int64_t pos = 0;
    for (int64_t x = 0; x + 1 < n; ++x) {
        for (int64_t y0 = x + 1; y0 < n; y0 += 512) {
            int64_t cc = std::min<int64_t>(512, n - y0);
            node.push_back((int32_t)x);
            start.push_back(pos);
            cntv.push_back((int32_t)cc);
            vb.push_back((int32_t)y0);
            pos += cc;
        }
    }
    const int64_t ns = (int64_t)node.size();
    GROW(S.seg_node, sizeof(int32_t) * std::max<int64_t>(ns, 1));
    GROW(S.seg_start, sizeof(int64_t) * std::max<int64_t>(ns, 1));
    GROW(S.seg_count, sizeof(int32_t) * std::max<int64_t>(ns, 1));
    GROW(S.seg_vbase, sizeof(int32_t) * std::max<int64_t>(ns, 1));
    if (ns) {
        CKS(cudaMemcpyAsync(S.seg_node.p, node.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, c->stream));
        CKS(cudaMemcpyAsync(S.seg_start.p, start.data(), sizeof(int64_t) * ns, cudaMemcpyHostToDevice, c->stream));
        CKS(cudaMemcpyAsync(S.seg_count.p, cntv.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, c->stream));
        CKS(cudaMemcpyAsync(S.seg_vbase.p, vb.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, c->stream));
        CKS(cudaStreamSynchronize(c->stream));  // the host vectors go out of scope
    }
    *nseg_out = ns;
    return RECON_OK;
}

// scores every pair x < y of the node set (local ids; gid maps them) into d,
// in lexicographic order; pairs (local) are written too
static recon_status score_all_pairs(recon_ctx *c, const int32_t *gid, int64_t n, int32_t *pairs, float *d) {
    SearchBufs &S = SB(c);
    const int64_t np = n * (n - 1) / 2;
    k_all_pairs<<<nblk(np), 256, 0, c->stream>>>(n, np, pairs);
    note_launch();
    CKS(cudaGetLastError());
    int64_t ns = 0;
    recon_status st = all_pair_segments(c, n, &ns);
    if (st != RECON_OK) return st;
    return score_segments_device(c, (int32_t *)S.seg_node.p, (int64_t *)S.seg_start.p, (int32_t *)S.seg_count.p,
                                 (int32_t *)S.seg_vbase.p, ns, nullptr, np, gid, d);
}

// sort (key, val) pairs; the sorted result is left in (keys, vals)
static recon_status sort_kv(recon_ctx *c, unsigned long long *keys, uint32_t *vals, int64_t n, int bit0,
                            int bit1) {
    SearchBufs &S = SB(c);
    GROW(S.sort_k2, sizeof(unsigned long long) * std::max<int64_t>(n, 1));
    GROW(S.sort_v2, sizeof(uint32_t) * std::max<int64_t>(n, 1));
    GROW(S.sort_tmp, sizeof(int64_t) * radix_tmp_elems(std::max<int64_t>(n, 1)));
    bool alt = false;
    CKS(radix_sort_u64(keys, vals, (unsigned long long *)S.sort_k2.p, (uint32_t *)S.sort_v2.p, n, bit0, bit1,
                       (int64_t *)S.sort_tmp.p, &alt, c->stream));
    if (alt) {
        CKS(cudaMemcpyAsync(keys, S.sort_k2.p, sizeof(unsigned long long) * n, cudaMemcpyDeviceToDevice, c->stream));
        CKS(cudaMemcpyAsync(vals, S.sort_v2.p, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, c->stream));
    }
    return RECON_OK;
}

// m best pairs among all pairs of the node set gid[0..n) (gid NULL: all nodes);
// appends them (global ids) to the result list
static recon_status exhaustive_best_set(recon_ctx *c, const int32_t *gid, int64_t n, int64_t m) {
    SearchBufs &S = SB(c);
    const int64_t np = n * (n - 1) / 2;
    if (np <= 0 || m <= 0) return RECON_OK;
    if (np >= ((int64_t)1 << 32)) return set_err(c, RECON_EUNSUPPORTED, "exhaustive search over %lld nodes", (long long)n);
    GROW(S.ex_pairs, sizeof(int32_t) * 2 * np);
    GROW(S.ex_d, sizeof(float) * np);
    GROW(S.ex_keys, sizeof(unsigned long long) * np);
    GROW(S.ex_vals, sizeof(uint32_t) * np);
    recon_status st = score_all_pairs(c, gid, n, (int32_t *)S.ex_pairs.p, (float *)S.ex_d.p);
    if (st != RECON_OK) return st;
    k_rank_keys<<<nblk(np), 256, 0, c->stream>>>(np, (float *)S.ex_d.p, (unsigned long long *)S.ex_keys.p,
                                                 (uint32_t *)S.ex_vals.p); note_launch();
    CKS(cudaGetLastError());
    st = sort_kv(c, (unsigned long long *)S.ex_keys.p, (uint32_t *)S.ex_vals.p, np, 0, 64);
    if (st != RECON_OK) return st;
    const int64_t take = std::min(m, np);
    GROW_KEEP(S.res_pairs, sizeof(int32_t) * 2 * (S.res_n + take), sizeof(int32_t) * 2 * S.res_n);
    GROW_KEEP(S.res_d, sizeof(float) * (S.res_n + take), sizeof(float) * S.res_n);
    k_gather_pairs<<<nblk(take), 256, 0, c->stream>>>(take, (uint32_t *)S.ex_vals.p, (int32_t *)S.ex_pairs.p, gid,
                                                      (float *)S.ex_d.p, (int32_t *)S.res_pairs.p + 2 * S.res_n,
                                                      (float *)S.res_d.p + S.res_n); note_launch();
    CKS(cudaGetLastError());
    S.res_n += take;
    return RECON_OK;
}

// exact KNN of a node set: all pairs scored once, then the k smallest per row
static recon_status knn_exhaustive(recon_ctx *c, const int32_t *gid, int n, int k) {
    SearchBufs &S = SB(c);
    const int64_t np = (int64_t)n * (n - 1) / 2;
    GROW(S.ex_pairs, sizeof(int32_t) * 2 * np);
    GROW(S.ex_d, sizeof(float) * np);
    GROW(S.dense, sizeof(float) * (size_t)n * n);
    recon_status st = score_all_pairs(c, gid, n, (int32_t *)S.ex_pairs.p, (float *)S.ex_d.p);
    if (st != RECON_OK) return st;
    k_dense_fill<<<nblk(std::max<int64_t>(np, n)), 256, 0, c->stream>>>(n, np, (int32_t *)S.ex_pairs.p,
                                                                           (float *)S.ex_d.p, (float *)S.dense.p); note_launch();
    CKS(cudaGetLastError());
    k_row_topk<<<n, 256, 0, c->stream>>>(n, k, (float *)S.dense.p, (int32_t *)S.knn_id.p, (float *)S.knn_d.p); note_launch();
    CKS(cudaGetLastError());
    return RECON_OK;
}

// NNDescent on the node set gid[0..n) with lists of k; returns iterations
// NNDescent over lists of capacity K with per-node lengths klen (device, n)
static recon_status knn_nndescent(recon_ctx *c, const int32_t *gid, int n, int k, const int32_t *klen,
                                  uint64_t seed, int *iters_out, bool learned) {
    SearchBufs &S = SB(c);
    const int64_t nk = (int64_t)n * k;
    const int in_cap = k, Ucap = k + in_cap;
    GROW(S.pairs_tmp, sizeof(int32_t) * 2 * nk);
    // 1. random initial lists, scored
    if (learned) {
        // first level: seeds from the learned embedding, random ids for the rest
        int64_t nseeded = 0;
        recon_status st0 = learned_seed_lists(c, n, k, klen, seed, (int32_t *)S.knn_id.p, &nseeded);
        if (st0 != RECON_OK) return st0;
        c->stats.seeded_nodes = nseeded;
    } else {
        k_knn_init<<<nblk(n), 256, 0, c->stream>>>(n, k, klen, seed, (int32_t *)S.knn_id.p); note_launch();
        CKS(cudaGetLastError());
    }
    GROW(S.seg_node, sizeof(int32_t) * n);
    GROW(S.seg_start, sizeof(int64_t) * n);
    GROW(S.seg_count, sizeof(int32_t) * n);
    k_list_pairs<<<nblk(nk), 256, 0, c->stream>>>(n, k, (int32_t *)S.knn_id.p, klen, (int32_t *)S.pairs_tmp.p,
                                                  (int32_t *)S.seg_node.p, (int64_t *)S.seg_start.p,
                                                  (int32_t *)S.seg_count.p); note_launch();
    CKS(cudaGetLastError());
    recon_status st = score_segments_device(c, (int32_t *)S.seg_node.p, (int64_t *)S.seg_start.p,
                                            (int32_t *)S.seg_count.p, nullptr, n, (int32_t *)S.pairs_tmp.p, nk, gid,
                                            (float *)S.knn_d.p);
    if (st != RECON_OK) return st;
    k_sort_lists<<<nblk(n, 128), 128, 0, c->stream>>>(n, k, klen, gid, (int32_t *)S.knn_id.p, (float *)S.knn_d.p,
                                                 (uint8_t *)S.knn_new.p); note_launch();
    CKS(cudaGetLastError());

    GROW(S.indeg, sizeof(int32_t) * (n + 1));
    GROW(S.inoff, sizeof(int64_t) * (n + 1));
    GROW(S.cursor, sizeof(int32_t) * (n + 1));
    GROW(S.in_e, sizeof(int32_t) * nk);
    GROW(S.U, sizeof(int32_t) * (size_t)n * Ucap);
    GROW(S.Uf, sizeof(uint8_t) * (size_t)n * Ucap);
    GROW(S.Udeg, sizeof(int32_t) * n);
    GROW(S.in_last, sizeof(int32_t) * nk);
    GROW(S.in_fresh, sizeof(int32_t) * nk);
    GROW(S.Usym, sizeof(uint8_t) * (size_t)n * Ucap);
    CKS(launch_fill_i32((int32_t *)S.in_last.p, -1, nk, c->stream));
    CKS(launch_fill_i32((int32_t *)S.in_fresh.p, -1, nk, c->stream));
    GROW(S.scan_in, sizeof(int64_t) * (n + 1));
    GROW(S.scan_tmp, sizeof(int64_t) * scan_tmp_elems(n + 1));
    const int raw = Ucap * Ucap;
    int hsize = 1;
    while (hsize < 2 * (raw + k) && hsize < 16384) hsize <<= 1;
    const int lcap = std::min(raw, hsize / 2);
    const size_t per_warp = sizeof(int32_t) * (size_t)(hsize + lcap + 1);
    int warps_per_block = (int)std::max<size_t>(1, std::min<size_t>(8, (96 * 1024) / per_warp));
    const size_t smem_gen = per_warp * warps_per_block;
    if (smem_gen > 48 * 1024)
        CKS(cudaFuncSetAttribute(k_gen, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_gen));
    // node x has at most min(raw, n-1) candidates
    const int64_t cand_cap = std::max<int64_t>(std::min<int64_t>((int64_t)n * lcap, (int64_t)n * (n - 1)), 1);
    GROW(S.cand, sizeof(int32_t) * 2 * cand_cap);
    GROW(S.cand_d, sizeof(float) * cand_cap);
    GROW(S.seg_node, sizeof(int32_t) * n);
    GROW(S.seg_start, sizeof(int64_t) * n);
    GROW(S.seg_count, sizeof(int32_t) * n);

    int max_iters = c->opt.max_knn_iters;
    if (max_iters <= 0) max_iters = 2 * (int)std::ceil(std::log((double)std::max(n, 2)) / std::log(2.0 * k)) + 2;
    // offers: at most two per candidate; beyond the buffer they are dropped (counted)
    const int64_t ocap = std::max<int64_t>(std::min<int64_t>(2 * cand_cap, (int64_t)1 << 30), 1);
    GROW(S.off_t, sizeof(int32_t) * ocap);
    GROW(S.off_v, sizeof(int32_t) * ocap);
    GROW(S.off_d, sizeof(float) * ocap);
    GROW(S.off_sv, sizeof(int32_t) * ocap);
    GROW(S.off_sd, sizeof(float) * ocap);
    GROW(S.iter, sizeof(int) * 4);
    CKS(cudaMemsetAsync(S.iter.p, 0, sizeof(int) * 4, c->stream));
    GROW(S.seed, sizeof(unsigned long long));
    {
        const unsigned long long sh = seed;  // staged by the copy before the call returns
        CKS(cudaMemcpyAsync(S.seed.p, &sh, sizeof sh, cudaMemcpyHostToDevice, c->stream));
    }
    const int threads = c->tuned_threads ? c->tuned_threads : 256;
    const unsigned stride_grid = (unsigned)std::max(1, 8 * c->num_sms);
    cudaEvent_t ea = nullptr, eb = nullptr;
    if (c->opt.timing) {
        if (!c->nnd_ea) CKS(cudaEventCreate(&c->nnd_ea));
        if (!c->nnd_eb) CKS(cudaEventCreate(&c->nnd_eb));
        ea = c->nnd_ea;
        eb = c->nnd_eb;
    }
    // The iterations run on a private non-blocking stream (graph capture is not
    // possible on the legacy default stream), ordered after the work already on
    // the context's stream and before anything enqueued there afterwards.
    const bool use_graph = c->opt.no_graphs == 0;
    cudaStream_t gs = c->stream;
    cudaEvent_t ev_join = nullptr;
    if (use_graph) {
        if (!c->gstream) CKS(cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
        gs = c->gstream;
        CKS(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
        CKS(cudaEventRecord(ev_join, c->stream));
        CKS(cudaStreamWaitEvent(gs, ev_join, 0));
    }
    // One iteration, enqueued with every count kept on the device (so that it can
    // be captured once as a CUDA graph and replayed); ends with one read-back of
    // the candidate, offer and change counts and the error word.
    // timing events inside a capture become record nodes of the graph
    unsigned rec_flags = cudaEventRecordDefault;
    // one iteration; readback: its counts to the host, for the host loop's
    // stopping test (the device loop tests on the device)
    auto enqueue = [&](bool readback) -> cudaError_t {
        cudaError_t e;
        k_next_iter<<<1, 1, 0, gs>>>((int *)S.iter.p);
        note_launch();
        if ((e = cudaMemsetAsync(S.indeg.p, 0, sizeof(int32_t) * (n + 1), gs))) return e;
        k_in_count<<<nblk(nk), 256, 0, gs>>>(nk, (int32_t *)S.knn_id.p, (int32_t *)S.indeg.p);
        note_launch();
        k_i32_to_i64<<<nblk(n + 1), 256, 0, gs>>>((int32_t *)S.indeg.p, (int64_t *)S.scan_in.p, n + 1);
        note_launch();
        if ((e = launch_scan_i64((int64_t *)S.scan_in.p, (int64_t *)S.inoff.p, n + 1, (int64_t *)S.scan_tmp.p,
                                 gs)))
            return e;
        if ((e = cudaMemsetAsync(S.cursor.p, 0, sizeof(int32_t) * (n + 1), gs))) return e;
        k_in_fill<<<nblk(nk), 256, 0, gs>>>(nk, (int32_t *)S.knn_id.p, (int64_t *)S.inoff.p,
                                                   (int32_t *)S.cursor.p, (int32_t *)S.in_e.p);
        note_launch();
        {
            const int wpb = 8;
            size_t smem = sizeof(int32_t) * 2 * Ucap * wpb;
            k_build_U<<<nblk((int64_t)n * 32, 32 * wpb), 32 * wpb, smem, gs>>>(
                n, k, klen, in_cap, Ucap, (const unsigned long long *)S.seed.p, (int *)S.iter.p, (int32_t *)S.knn_id.p,
                (uint8_t *)S.knn_new.p,
                (int64_t *)S.inoff.p, (int32_t *)S.indeg.p, (int32_t *)S.in_e.p, (int32_t *)S.in_last.p,
                (int32_t *)S.in_fresh.p, (int32_t *)S.U.p, (uint8_t *)S.Uf.p,
                (int32_t *)S.Udeg.p);
            note_launch();
        }
        k_U_sym<<<nblk((int64_t)n * 32, 256), 256, 0, gs>>>(n, k, klen, Ucap, (int *)S.iter.p, (int32_t *)S.knn_id.p,
                                                          (uint8_t *)S.knn_new.p, (int32_t *)S.in_fresh.p,
                                                          (int32_t *)S.U.p, (uint8_t *)S.Uf.p, (int32_t *)S.Udeg.p,
                                                          (uint8_t *)S.Usym.p);
        note_launch();
        if ((e = cudaMemsetAsync(c->cnt + CNT_SCRATCH0, 0, sizeof(unsigned long long) * 4, gs))) return e;
        k_gen<<<nblk((int64_t)n * 32, 32 * warps_per_block), 32 * warps_per_block, smem_gen, gs>>>(
            n, k, klen, Ucap, (int32_t *)S.U.p, (uint8_t *)S.Uf.p, (uint8_t *)S.Usym.p, (int32_t *)S.Udeg.p,
            (int32_t *)S.knn_id.p, hsize,
            lcap, (int32_t *)S.cand.p, cand_cap, counter(c, CNT_SCRATCH0), c->cnt, (int32_t *)S.seg_node.p,
            (int64_t *)S.seg_start.p, (int32_t *)S.seg_count.p);
        note_launch();
        if (ea && (e = cudaEventRecordWithFlags(ea, gs, rec_flags))) return e;
        if ((e = launch_seg(c, (int32_t *)S.seg_node.p, (int64_t *)S.seg_start.p, (int32_t *)S.seg_count.p, nullptr,
                            n, (int32_t *)S.cand.p, gid, (float *)S.cand_d.p, threads, gs)))
            return e;
        if (eb && (e = cudaEventRecordWithFlags(eb, gs, rec_flags))) return e;
        k_offer<<<stride_grid, 256, 0, gs>>>(counter(c, CNT_SCRATCH0), cand_cap, (int32_t *)S.cand.p,
                                                    (float *)S.cand_d.p, k, klen, (float *)S.knn_d.p,
                                                    (int32_t *)S.off_t.p, (int32_t *)S.off_v.p, (float *)S.off_d.p,
                                                    counter(c, CNT_SCRATCH1), ocap, counter(c, CNT_SCRATCH3));
        note_launch();
        if ((e = cudaMemsetAsync(S.indeg.p, 0, sizeof(int32_t) * (n + 1), gs))) return e;
        k_count_targets<<<stride_grid, 256, 0, gs>>>(counter(c, CNT_SCRATCH1), ocap, (int32_t *)S.off_t.p,
                                                            (int32_t *)S.indeg.p);
        note_launch();
        k_i32_to_i64<<<nblk(n + 1), 256, 0, gs>>>((int32_t *)S.indeg.p, (int64_t *)S.scan_in.p, n + 1);
        note_launch();
        if ((e = launch_scan_i64((int64_t *)S.scan_in.p, (int64_t *)S.inoff.p, n + 1, (int64_t *)S.scan_tmp.p,
                                 gs)))
            return e;
        if ((e = cudaMemsetAsync(S.cursor.p, 0, sizeof(int32_t) * (n + 1), gs))) return e;
        k_scatter_offers<<<stride_grid, 256, 0, gs>>>(counter(c, CNT_SCRATCH1), ocap, (int32_t *)S.off_t.p,
                                                             (int32_t *)S.off_v.p, (float *)S.off_d.p,
                                                             (int64_t *)S.inoff.p, (int32_t *)S.cursor.p,
                                                             (int32_t *)S.off_sv.p, (float *)S.off_sd.p);
        note_launch();
        k_merge<<<nblk((int64_t)n * 32), 256, 0, gs>>>(n, k, klen, gid, (int32_t *)S.knn_id.p,
                                                              (float *)S.knn_d.p, (uint8_t *)S.knn_new.p,
                                                              (int64_t *)S.inoff.p, (int32_t *)S.off_sv.p,
                                                              (float *)S.off_sd.p, counter(c, CNT_SCRATCH2));
        note_launch();
        if (!readback) return cudaGetLastError();
        // counts back to the host: candidates, offers, changes, drops; and the error word
        if ((e = cudaMemcpyAsync(c->cnt_host + CNT_SCRATCH0, c->cnt + CNT_SCRATCH0, sizeof(unsigned long long) * 4,
                                 cudaMemcpyDeviceToHost, gs)))
            return e;
        if ((e = cudaMemcpyAsync(c->cnt_host + CNT_ERR, c->cnt + CNT_ERR, sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, gs)))
            return e;
        return cudaGetLastError();
    };
    // everything the captured iteration depends on: a graph captured with the
    // same values (a later search of the same shape) is replayed as it is
    std::vector<uint8_t> sig;
    auto put = [&](const void *p, size_t nb) {
        const uint8_t *b = (const uint8_t *)p;
        sig.insert(sig.end(), b, b + nb);
    };
    {
        const int64_t ints[] = {n, k, in_cap, Ucap, hsize, lcap, cand_cap, ocap, (int64_t)smem_gen, warps_per_block,
                                threads, stride_grid, c->model};
        put(ints, sizeof ints);
        const void *ptrs[] = {klen, gid, ea, eb, gs, c->cnt, c->cnt_host, S.knn_id.p, S.knn_d.p, S.knn_new.p,
                              S.indeg.p, S.inoff.p, S.cursor.p, S.in_e.p, S.in_last.p, S.in_fresh.p, S.Usym.p,
                              S.U.p, S.Uf.p, S.Udeg.p, S.scan_in.p,
                              S.scan_tmp.p, S.cand.p, S.cand_d.p, S.seg_node.p, S.seg_start.p, S.seg_count.p,
                              S.off_t.p, S.off_v.p, S.off_d.p, S.off_sv.p, S.off_sd.p, S.iter.p, S.seed.p};
        put(ptrs, sizeof ptrs);
        const ScoreParams sp = c->sp();
        put(&sp, sizeof sp);
        put(&c->W, sizeof c->W);
        if (c->model == RECON_ISING) {
            const IsingView v = c->iv();
            put(&v, sizeof v);
        } else {
            const GaussView v = c->gv();
            put(&v, sizeof v);
        }
    }
    int it = 0;
    recon_status result = RECON_OK;
    bool done = false;  // the device loop ran the iterations
    // Without per-iteration timing, every iteration goes into one graph launch: a
    // WHILE node whose body is an iteration followed by k_nnd_continue, the
    // stopping test on the device.  One launch and one synchronisation per
    // level instead of one of each per iteration; when the conditional graph
    // cannot be built, the host loop below runs instead.
    if (use_graph && !ea && !c->nnd_loop_broken) {
        GROW(S.nnd_acc, sizeof(unsigned long long) * 2);
        std::vector<uint8_t> lsig = sig;
        {
            const double lp[] = {(double)max_iters, (double)S.klen_sum, c->opt.eps_knn,
                                 (double)(uintptr_t)S.nnd_acc.p};
            const uint8_t *b = (const uint8_t *)lp;
            lsig.insert(lsig.end(), b, b + sizeof lp);
        }
        if (c->nnd_loop_exec && lsig != c->nnd_loop_sig) {
            cudaGraphExecDestroy(c->nnd_loop_exec);
            c->nnd_loop_exec = nullptr;
            c->nnd_loop_sig.clear();
        }
        if (!c->nnd_loop_exec) {
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaGraphCreate(&g, 0);
            cudaGraphConditionalHandle h{};
            if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t node = nullptr;
            if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
            if (e == cudaSuccess) {
                cudaGraph_t body = cp.conditional.phGraph_out[0];
                e = cudaStreamBeginCaptureToGraph(gs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    const int64_t l0 = c->stats.kernel_launches;
                    cudaError_t ce = enqueue(false);
                    if (ce == cudaSuccess) {
                        k_nnd_continue<<<1, 1, 0, gs>>>(h, c->cnt, (const int *)S.iter.p, max_iters,
                                                        (double)S.klen_sum, c->opt.eps_knn,
                                                        (unsigned long long)cand_cap,
                                                        (unsigned long long *)S.nnd_acc.p);
                        note_launch();
                        ce = cudaGetLastError();
                    }
                    c->graph_launches_per_iter = c->stats.kernel_launches - l0;
                    c->stats.kernel_launches = l0;
                    cudaGraph_t out = nullptr;
                    const cudaError_t ee = cudaStreamEndCapture(gs, &out);
                    e = ce != cudaSuccess ? ce : ee;
                }
            }
            cudaGraphExec_t ex = nullptr;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e == cudaSuccess) {
                c->nnd_loop_exec = ex;
                c->nnd_loop_sig = std::move(lsig);
            } else {
                (void)cudaGetLastError();
                c->nnd_loop_broken = true;
            }
        }
        if (c->nnd_loop_exec) {
            unsigned long long acc_h[2] = {0, 0};
            int iters_h = 0;
            cudaError_t e = cudaMemsetAsync(S.nnd_acc.p, 0, sizeof(unsigned long long) * 2, gs);
            if (e == cudaSuccess) e = cudaGraphLaunch(c->nnd_loop_exec, gs);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(acc_h, S.nnd_acc.p, sizeof acc_h, cudaMemcpyDeviceToHost, gs);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&iters_h, S.iter.p, sizeof(int), cudaMemcpyDeviceToHost, gs);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(c->cnt_host + CNT_ERR, c->cnt + CNT_ERR, sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, gs);
            if (e == cudaSuccess) e = cudaStreamSynchronize(gs);
            if (e != cudaSuccess) {
                result = cuda_fail(c, e, "NNDescent iterations");
            } else {
                it = iters_h;
                c->stats.kernel_launches += c->graph_launches_per_iter * (int64_t)it;
                c->stats.pair_evals += (int64_t)acc_h[0];
                c->stats.dropped_offers += (int64_t)acc_h[1];
                c->stats.nnd_graph_loops += 1;
                if (c->cnt_host[CNT_ERR]) result = check_err_flags(c, "NNDescent");
            }
            done = true;
        }
    }
    cudaGraphExec_t exec = nullptr;
    if (!done && use_graph && c->nnd_exec && sig == c->nnd_sig) exec = c->nnd_exec;
    if (!done && use_graph && !exec) {
        if (c->nnd_exec) {
            cudaGraphExecDestroy(c->nnd_exec);
            c->nnd_exec = nullptr;
            c->nnd_sig.clear();
        }
        // a capture that fails leaves the launch-by-launch path in use
        cudaGraph_t graph = nullptr;
        const int64_t launches0 = c->stats.kernel_launches;
        cudaError_t e = cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            rec_flags = cudaEventRecordExternal;
            cudaError_t ce = enqueue(true);
            rec_flags = cudaEventRecordDefault;
            cudaError_t ee = cudaStreamEndCapture(gs, &graph);
            e = ce != cudaSuccess ? ce : ee;
        }
        c->graph_launches_per_iter = c->stats.kernel_launches - launches0;
        c->stats.kernel_launches = launches0;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            exec = nullptr;
            cudaGetLastError();
        } else {
            c->nnd_exec = exec;
            c->nnd_sig = std::move(sig);
        }
    }
    while (!done && it < max_iters) {
        ++it;
        cudaError_t e;
        if (exec) {
            e = cudaGraphLaunch(exec, gs);
            c->stats.kernel_launches += c->graph_launches_per_iter;
        } else
            e = enqueue(true);
        if (e == cudaSuccess) e = cudaStreamSynchronize(gs);
        if (e != cudaSuccess) {
            result = cuda_fail(c, e, "NNDescent iteration");
            break;
        }
        const unsigned long long ncand = std::min<unsigned long long>(c->cnt_host[CNT_SCRATCH0], cand_cap);
        const unsigned long long delta = c->cnt_host[CNT_SCRATCH2];
        c->stats.pair_evals += (int64_t)ncand;
        c->stats.dropped_offers += (int64_t)c->cnt_host[CNT_SCRATCH3];
        if (ea) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ea, eb) == cudaSuccess) {
                c->stats.score_ms += ms;
                c->stats.score_launches += 1;
                c->stats.score_pairs += (int64_t)ncand;
            } else
                cudaGetLastError();
        }
        if (c->cnt_host[CNT_ERR]) {
            result = check_err_flags(c, "NNDescent");
            if (result != RECON_OK) break;
        }
        if ((double)delta / (double)S.klen_sum < c->opt.eps_knn) break;
    }
    if (ev_join) {
        cudaEventRecord(ev_join, gs);
        cudaStreamWaitEvent(c->stream, ev_join, 0);
        cudaEventDestroy(ev_join);
    }
    if (result != RECON_OK) return result;
    *iters_out = it;
    return RECON_OK;
}

// final m best of the collected (global) pairs, ordered by (d, i, j), unique
static recon_status finish_results(recon_ctx *c, int64_t m, int64_t *count) {
    SearchBufs &S = SB(c);
    const int64_t P = S.res_n;
    *count = 0;
    if (P == 0) return RECON_OK;
    GROW(S.fk, sizeof(unsigned long long) * P);
    GROW(S.fv, sizeof(uint32_t) * P);
    GROW(S.flag, sizeof(int64_t) * P);
    GROW(S.pos, sizeof(int64_t) * P);
    GROW(S.scan_tmp2, sizeof(int64_t) * scan_tmp_elems(P));
    GROW(S.out_pairs, sizeof(int32_t) * 2 * std::max<int64_t>(m, 1));
    GROW(S.out_d, sizeof(float) * std::max<int64_t>(m, 1));
    if (P <= FIN_SMALL && !c->findbest_sorts) {  // one CTA: sort in shared memory, unique, gather
        int np2 = 1;
        while (np2 < P) np2 <<= 1;
        const size_t smem = sizeof(FinItem) * (size_t)np2;
        static int attr_device = -1;
        if (attr_device != c->device) {
            CKS(cudaFuncSetAttribute(k_finish_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(sizeof(FinItem) * FIN_SMALL)));
            attr_device = c->device;
        }
        k_finish_small<<<1, 1024, smem, c->stream>>>((int)P, np2, m, (int32_t *)S.res_pairs.p, (float *)S.res_d.p,
                                                      (int32_t *)S.out_pairs.p, (float *)S.out_d.p,
                                                      counter(c, CNT_SCRATCH2)); note_launch();
        CKS(cudaGetLastError());
        unsigned long long nout = 0;
        recon_status st = read_counter(c, CNT_SCRATCH2, &nout);
        if (st != RECON_OK) return st;
        *count = (int64_t)nout;
        return RECON_OK;
    }
    k_pair_keys<<<nblk(P), 256, 0, c->stream>>>(P, (int32_t *)S.res_pairs.p, (unsigned long long *)S.fk.p,
                                                (uint32_t *)S.fv.p); note_launch();
    CKS(cudaGetLastError());
    // by (i, j): both ids are below N, so only their low bits need passes (a
    // stable LSD sort over j's bits, then over i's, orders by the full key)
    int idb = 8;
    while (idb < 32 && ((int64_t)1 << idb) < c->N) idb += 8;
    recon_status st = sort_kv(c, (unsigned long long *)S.fk.p, (uint32_t *)S.fv.p, P, 0, idb);
    if (st != RECON_OK) return st;
    st = sort_kv(c, (unsigned long long *)S.fk.p, (uint32_t *)S.fv.p, P, 32, 32 + idb);
    if (st != RECON_OK) return st;
    GROW(S.fk2, sizeof(unsigned long long) * P);
    GROW(S.fv2, sizeof(uint32_t) * P);
    k_d_keys<<<nblk(P), 256, 0, c->stream>>>(P, (uint32_t *)S.fv.p, (float *)S.res_d.p, (unsigned long long *)S.fk2.p,
                                             (uint32_t *)S.fv2.p); note_launch();
    CKS(cudaGetLastError());
    st = sort_kv(c, (unsigned long long *)S.fk2.p, (uint32_t *)S.fv2.p, P, 0, 32);
    if (st != RECON_OK) return st;
    k_unique_flags<<<nblk(P), 256, 0, c->stream>>>(P, (uint32_t *)S.fv2.p, (int32_t *)S.res_pairs.p,
                                                   (int64_t *)S.flag.p); note_launch();
    CKS(cudaGetLastError());
    CKS(launch_scan_i64((int64_t *)S.flag.p, (int64_t *)S.pos.p, P, (int64_t *)S.scan_tmp2.p, c->stream));
    k_unique_gather<<<nblk(P), 256, 0, c->stream>>>(P, m, (uint32_t *)S.fv2.p, (int64_t *)S.flag.p,
                                                    (int64_t *)S.pos.p, (int32_t *)S.res_pairs.p, (float *)S.res_d.p,
                                                    (int32_t *)S.out_pairs.p, (float *)S.out_d.p); note_launch();
    CKS(cudaGetLastError());
    int64_t last_pos = 0, last_flag = 0;
    CKS(cudaMemcpyAsync(&last_pos, (int64_t *)S.pos.p + P - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    CKS(cudaMemcpyAsync(&last_flag, (int64_t *)S.flag.p + P - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    CKS(cudaStreamSynchronize(c->stream));
    *count = std::min(m, last_pos + last_flag);
    return RECON_OK;
}

recon_status findbest_run(recon_ctx *c, int k_cfg, int64_t m, int32_t **pairs_dev, float **d_dev, int64_t *count) {
    if (c->opt.knn_mode == RECON_KNN_SCREEN) {
        c->stats.levels = 0;
        c->stats.knn_iters = 0;
        c->stats.level_size[0] = c->N;
        return screen_run(c, m, pairs_dev, d_dev, count);
    }
    SearchBufs &S = SB(c);
    S.res_n = 0;
    c->stats.levels = 0;
    c->stats.knn_iters = 0;
    for (int t = 0; t < 16; ++t) c->stats.level_k[t] = 0;
    for (int t = 0; t < 17; ++t) c->stats.level_size[t] = 0;
    const int64_t N = c->N;
    GROW(S.gid_a, sizeof(int32_t) * N);
    GROW(S.gid_b, sizeof(int32_t) * N);
    k_iota<<<nblk(N), 256, 0, c->stream>>>((int32_t *)S.gid_a.p, N); note_launch();
    CKS(cudaGetLastError());
    int32_t *gid = (int32_t *)S.gid_a.p, *gid_next = (int32_t *)S.gid_b.p;
    int64_t n = N;
    const uint64_t call_seed = mix64(c->opt.seed ^ mix64(0x9e37ull + (uint64_t)c->stats_calls));
    c->stats_calls++;
    S.g0_n = N;
    S.g0_K = 0;
    S.g0_moved = false;
    for (int level = 0;; ++level) {
        if (level < 17) c->stats.level_size[level] = n;
        if (level == 1 && S.g0_K > 0) {
            // keep the first level's lists (the k-NN graph of all nodes): the
            // buffers change places, nothing is copied
            std::swap(S.knn_id, S.g0_id);
            std::swap(S.knn_d, S.g0_d);
            std::swap(S.klen, S.g0_klen);
            S.g0_moved = true;
        }
        if (n * n <= 4 * m) {
            recon_status st = exhaustive_best_set(c, level == 0 ? nullptr : gid, n, m);
            if (st != RECON_OK) return st;
            break;
        }
        int64_t k64 = (4 * m + n - 1) / n;
        k64 = std::max<int64_t>(k64, k_cfg);
        k64 = std::min<int64_t>(k64, n - 1);
        int k = (int)k64;
        // per-node list lengths (first level only, when the caller set them)
        const bool uneven = level == 0 && (int64_t)c->klen_host.size() == n;
        GROW(S.klen, sizeof(int32_t) * n);
        if (uneven) {
            std::vector<int32_t> kl(n);
            int kmax = 1;
            int64_t sum = 0;
            for (int64_t x = 0; x < n; ++x) {
                kl[x] = (int32_t)std::min<int64_t>(n - 1, std::max<int64_t>(c->klen_host[x], (4 * m + n - 1) / n));
                kmax = std::max(kmax, (int)kl[x]);
                sum += kl[x];
            }
            if (kmax > NND_MAX_K)
                return set_err(c, RECON_EUNSUPPORTED, "per-node list lengths above %d", NND_MAX_K);
            CKS(cudaMemcpyAsync(S.klen.p, kl.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, c->stream));
            CKS(cudaStreamSynchronize(c->stream));
            k = kmax;
            S.klen_sum = sum;
        } else {
            CKS(launch_fill_i32((int32_t *)S.klen.p, k, n, c->stream));
            S.klen_sum = n * (int64_t)k;
        }
        if (level < 16) c->stats.level_k[level] = k;
        c->stats.levels = level + 1;
        const int64_t nk = n * k;
        GROW(S.knn_id, sizeof(int32_t) * nk);
        GROW(S.knn_d, sizeof(float) * nk);
        GROW(S.knn_new, sizeof(uint8_t) * nk);
        bool exhaustive = (c->opt.knn_mode == RECON_KNN_EXHAUSTIVE || k > NND_MAX_K) && !uneven;
        if (c->opt.knn_mode == RECON_KNN_AUTO) {
            // NNDescent scores about |S| (2k)^2 / 2 pairs per iteration
            double nnd = (double)n * 4.0 * k * k / 2.0 * 3.0;
            double exh = (double)n * (n - 1) / 2.0;
            exhaustive = (exhaustive || exh <= nnd) && !uneven;
        }
        if (exhaustive && (double)n * n * 4.0 > 16e9)
            return set_err(c, RECON_EUNSUPPORTED, "level of %lld nodes with k = %d needs NNDescent with k <= %d",
                           (long long)n, k, NND_MAX_K);
        recon_status st;
        if (exhaustive) {
            st = knn_exhaustive(c, gid, (int)n, k);
        } else {
            int iters = 0;
            const bool learned = level == 0 && c->opt.seed_mode == RECON_SEED_LEARNED && c->prop && c->prop->trained;
            st = knn_nndescent(c, gid, (int)n, k, (int32_t *)S.klen.p, mix64(call_seed + (uint64_t)level), &iters,
                               learned);
            c->stats.knn_iters += iters;
        }
        if (st != RECON_OK) return st;
        if (level == 0) S.g0_K = k;
        // D+ : the 2m best directed edges
        GROW(S.ek, sizeof(unsigned long long) * nk);
        GROW(S.ev, sizeof(uint32_t) * nk);
        k_edge_keys<<<nblk(nk), 256, 0, c->stream>>>((int)n, k, gid, (int32_t *)S.knn_id.p, (float *)S.knn_d.p,
                                                     (unsigned long long *)S.ek.p, (uint32_t *)S.ev.p); note_launch();
        CKS(cudaGetLastError());
        const int64_t nDp = std::min<int64_t>(2 * m, S.klen_sum);
        if (nk <= SEL_SMALL && !c->findbest_sorts) {  // one CTA selects the nDp best keys (a set: D+ needs no order)
            if (nDp > 0) {
                k_select_small<<<1, 1024, 0, c->stream>>>(nk, nDp, (unsigned long long *)S.ek.p, (uint32_t *)S.ev.p);
                note_launch();
                CKS(cudaGetLastError());
            }
        } else {
            st = sort_kv(c, (unsigned long long *)S.ek.p, (uint32_t *)S.ev.p, nk, 0, 64);
            if (st != RECON_OK) return st;
        }
        // D : unique pairs of D+
        uint64_t dcap = 1;
        while (dcap < (uint64_t)(4 * nDp + 64)) dcap <<= 1;
        GROW(S.dset, sizeof(unsigned long long) * dcap);
        CKS(launch_fill_u64((unsigned long long *)S.dset.p, RECON_EMPTY_KEY, (int64_t)dcap, c->stream));
        GROW_KEEP(S.res_pairs, sizeof(int32_t) * 2 * (S.res_n + nDp), sizeof(int32_t) * 2 * S.res_n);
        GROW_KEEP(S.res_d, sizeof(float) * (S.res_n + nDp), sizeof(float) * S.res_n);
        CKS(cudaMemsetAsync(counter(c, CNT_SCRATCH3), 0, sizeof(unsigned long long), c->stream));
        k_take_D<<<nblk(nDp), 256, 0, c->stream>>>(nDp, k, gid, (int32_t *)S.knn_id.p, (float *)S.knn_d.p,
                                                   (uint32_t *)S.ev.p, (unsigned long long *)S.dset.p, dcap - 1,
                                                   (int32_t *)S.res_pairs.p + 2 * S.res_n,
                                                   (float *)S.res_d.p + S.res_n, counter(c, CNT_SCRATCH3), c->cnt); note_launch();
        CKS(cudaGetLastError());
        unsigned long long nD = 0;
        st = read_counter(c, CNT_SCRATCH3, &nD);
        if (st != RECON_OK) return st;
        S.res_n += (int64_t)nD;
        // S' : saturated nodes
        GROW(S.flag, sizeof(int64_t) * (n + 1));
        GROW(S.pos, sizeof(int64_t) * (n + 1));
        GROW(S.scan_tmp2, sizeof(int64_t) * scan_tmp_elems(n + 1));
        k_saturated<<<nblk(n), 256, 0, c->stream>>>((int)n, k, (int32_t *)S.klen.p, gid, (int32_t *)S.knn_id.p,
                                                    (unsigned long long *)S.dset.p, dcap - 1, (int64_t *)S.flag.p); note_launch();
        CKS(cudaGetLastError());
        CKS(cudaMemsetAsync((int64_t *)S.flag.p + n, 0, sizeof(int64_t), c->stream));
        CKS(launch_scan_i64((int64_t *)S.flag.p, (int64_t *)S.pos.p, n + 1, (int64_t *)S.scan_tmp2.p, c->stream));
        k_compact_nodes<<<nblk(n), 256, 0, c->stream>>>((int)n, (int64_t *)S.flag.p, (int64_t *)S.pos.p, gid,
                                                        gid_next); note_launch();
        CKS(cudaGetLastError());
        int64_t n2 = 0;
        CKS(cudaMemcpyAsync(&n2, (int64_t *)S.pos.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
        CKS(cudaStreamSynchronize(c->stream));
        st = check_err_flags(c, "FindBest");
        if (st != RECON_OK) return st;
        std::swap(gid, gid_next);
        n = n2;
        if (n < 2) {
            if (level + 1 < 17) c->stats.level_size[level + 1] = n;
            break;
        }
    }
    recon_status st = finish_results(c, m, count);
    if (st != RECON_OK) return st;
    *pairs_dev = (int32_t *)S.out_pairs.p;
    *d_dev = (float *)S.out_d.p;
    return RECON_OK;
}

// The exact m best pairs through the tensor-core screen: every pair that can
// have a nonzero gain survives the screen (see screen.cu); those and the stored
// couplings are scored exactly, and the m best of them are returned.
recon_status screen_run(recon_ctx *c, int64_t m, int32_t **pairs_dev, float **d_dev, int64_t *count) {
    SearchBufs &S = SB(c);
    S.res_n = 0;
    S.g0_K = 0;
    const bool fp8 = c->opt.screen_fp8 != 0;
    const int64_t N = c->N;
    int64_t nnz = 0;
    {
        CKS(cudaMemsetAsync(counter(c, CNT_SCRATCH0), 0, sizeof(unsigned long long), c->stream));
        CKS(launch_table_count(c->W, counter(c, CNT_SCRATCH0), c->stream));
        unsigned long long v = 0;
        recon_status st = read_counter(c, CNT_SCRATCH0, &v);
        if (st != RECON_OK) return st;
        nnz = (int64_t)v;
    }
    // the empty network (no stored coupling): every sample of a node has the same
    // field, and the screen takes its exact rank-one form (E4M3 spins, K = Mp);
    // the prep kernel confirms the constant rows, else the general form runs
    bool rank1 = c->model == RECON_ISING && nnz == 0 && !c->opt.screen_no_rank1;
    if (rank1) {
        GROW(S.scr_A, (size_t)N * screen_k_rank1(c));
        GROW(S.scr_l1, sizeof(float2) * N);
        CKS(cudaMemsetAsync(counter(c, CNT_SCRATCH2), 0, sizeof(unsigned long long), c->stream));
        CKS(launch_screen_prep_rank1(c, S.scr_A.p, (float2 *)S.scr_l1.p, counter(c, CNT_SCRATCH2)));
        unsigned long long nonconst = 0;
        recon_status st = read_counter(c, CNT_SCRATCH2, &nonconst);
        if (st != RECON_OK) return st;
        rank1 = nonconst == 0;
    }
    if (!rank1) {
        const int64_t K = screen_k(c, fp8);
        const size_t esz = fp8 ? 1 : sizeof(uint16_t);
        GROW(S.scr_A, esz * (size_t)N * K);
        GROW(S.scr_B, esz * (size_t)N * K);
        GROW(S.scr_l1, sizeof(float) * N);
        CKS(launch_screen_prep(c, S.scr_A.p, S.scr_B.p, (float *)S.scr_l1.p, fp8));
    }
    int64_t cap = std::max<int64_t>(int64_t(1) << 20, 16 * m);
    const float rel = screen_rel_err(c->model, (int)c->Mp, fp8);
    unsigned long long nsurv = 0;
    for (int attempt = 0; attempt < 3; ++attempt) {
        GROW(S.cand, sizeof(int32_t) * 2 * (cap + nnz + 1));
        CKS(cudaMemsetAsync(counter(c, CNT_SCRATCH1), 0, sizeof(unsigned long long), c->stream));
        cudaEvent_t ea = nullptr, eb = nullptr;
        if (c->opt.timing) {
            for (cudaEvent_t *ev : {&ea, &eb}) {
                if (!c->event_pool.empty()) {
                    *ev = c->event_pool.back();
                    c->event_pool.pop_back();
                } else
                    CKS(cudaEventCreate(ev));
            }
            CKS(cudaEventRecord(ea, c->stream));
        }
        double flop = 0.0;
        if (rank1)
            CKS(launch_screen_ex(c, S.scr_A.p, S.scr_A.p, screen_k_rank1(c), (float)c->opt.lambda, nullptr, 0.f, 0,
                                 true, (int32_t *)S.cand.p, cap, counter(c, CNT_SCRATCH1), &flop, true,
                                 screen_rank1_margin(c), (int)c->Mp, (const float2 *)S.scr_l1.p, true));
        else
            CKS(launch_screen(c, S.scr_A.p, S.scr_B.p, (float *)S.scr_l1.p, (int32_t *)S.cand.p, cap,
                              counter(c, CNT_SCRATCH1), rel, &flop, fp8));
        if (rank1) c->stats.screen_rank1 += 1;
        if (c->opt.timing) {
            CKS(cudaEventRecord(eb, c->stream));
            c->timed.push_back({ea, eb, -1});
            c->stats.screen_flop += flop;
        }
        recon_status st = read_counter(c, CNT_SCRATCH1, &nsurv);
        if (st != RECON_OK) return st;
        st = check_err_flags(c, "screen");
        if (st != RECON_OK) {
            c->broken = true;
            return set_err(c, RECON_ETIMEOUT, "the tensor-core screen gave up waiting");
        }
        if ((int64_t)nsurv <= cap) break;
        cap = (int64_t)nsurv + nsurv / 4 + 1024;
    }
    if ((int64_t)nsurv > cap) return set_err(c, RECON_ENOMEM, "screen survivors exceed the buffer");
    c->stats.screen_survivors += (int64_t)nsurv;
    // the stored couplings, appended after the survivors
    if (nnz > 0) {
        GROW(S.ex_d, sizeof(float) * (nnz + 1));
        CKS(cudaMemsetAsync(counter(c, CNT_SCRATCH2), 0, sizeof(unsigned long long), c->stream));
        CKS(launch_table_dump(c->W, (int32_t *)S.cand.p + 2 * nsurv, (float *)S.ex_d.p, counter(c, CNT_SCRATCH2),
                              c->stream));
    }
    const int64_t P = (int64_t)nsurv + nnz;
    GROW(S.res_pairs, sizeof(int32_t) * 2 * std::max<int64_t>(P, 1));
    GROW(S.res_d, sizeof(float) * std::max<int64_t>(P, 1));
    if (P > 0) {
        recon_status st = score_pairs_device(c, (int32_t *)S.cand.p, P, nullptr, (float *)S.res_d.p, nullptr);
        if (st != RECON_OK) return st;
        CKS(cudaMemcpyAsync(S.res_pairs.p, S.cand.p, sizeof(int32_t) * 2 * P, cudaMemcpyDeviceToDevice, c->stream));
    }
    S.res_n = P;
    recon_status st = finish_results(c, m, count);
    if (st != RECON_OK) return st;
    *pairs_dev = (int32_t *)S.out_pairs.p;
    *d_dev = (float *)S.out_d.p;
    return RECON_OK;
}

// the m best of a scored pair list (device), unique, ordered by (d, i, j):
// the merge of the shards of a split search
recon_status select_run(recon_ctx *c, const int32_t *pairs, const float *d, int64_t P, int64_t m, int32_t **pairs_dev,
                        float **d_dev, int64_t *count) {
    SearchBufs &S = SB(c);
    S.res_n = 0;
    S.g0_K = 0;
    GROW(S.res_pairs, sizeof(int32_t) * 2 * std::max<int64_t>(P, 1));
    GROW(S.res_d, sizeof(float) * std::max<int64_t>(P, 1));
    k_canon_pairs<<<nblk(P), 256, 0, c->stream>>>(P, (int)c->N, pairs, d, (int32_t *)S.res_pairs.p,
                                                  (float *)S.res_d.p, c->cnt);
    note_launch();
    CKS(cudaGetLastError());
    recon_status st = check_err_flags(c, "select");
    if (st != RECON_OK) return st;
    S.res_n = P;
    st = finish_results(c, m, count);
    if (st != RECON_OK) return st;
    *pairs_dev = (int32_t *)S.out_pairs.p;
    *d_dev = (float *)S.out_d.p;
    return RECON_OK;
}

recon_status exhaustive_run(recon_ctx *c, int64_t m, int32_t **pairs_dev, float **d_dev, int64_t *count) {
    SearchBufs &S = SB(c);
    S.res_n = 0;
    recon_status st = exhaustive_best_set(c, nullptr, c->N, m);
    if (st != RECON_OK) return st;
    st = finish_results(c, m, count);
    if (st != RECON_OK) return st;
    *pairs_dev = (int32_t *)S.out_pairs.p;
    *d_dev = (float *)S.out_d.p;
    return RECON_OK;
}

// segments of whole rows: row r of the batch covers columns [0, n) in chunks
// of 512, d of (rows[r], y) at r n + y
__global__ void k_row_segments(int64_t nb, int64_t n, int64_t nch, const int32_t *rows, int32_t *seg_node,
                               int64_t *seg_start, int32_t *seg_count, int32_t *seg_vbase) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nb * nch) return;
    const int64_t r = s / nch, ch = s % nch;
    const int64_t y0 = ch * 512;
    seg_node[s] = rows[r];
    seg_start[s] = r * n + y0;
    seg_count[s] = (int32_t)min((int64_t)512, n - y0);
    seg_vbase[s] = (int32_t)y0;
}

// pairs {rows[r], y}, y != rows[r], with d < cut, appended in canonical order
__global__ void k_row_select(int64_t nb, int64_t n, const int32_t *rows, const float *dd, float cut, int32_t *pairs,
                             float *dout, int64_t cap, unsigned long long *counter) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = e < nb * n;
    int x = 0, y = 0;
    float d = 0.f;
    bool take = false;
    if (in) {
        x = rows[e / n];
        y = (int)(e % n);
        d = dd[e];
        take = y != x && d < cut;
    }
    const unsigned mask = __ballot_sync(0xffffffffu, take);
    if (!mask) return;
    const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (!take) return;
    const int64_t q = (int64_t)base + __popc(mask & ((1u << lane) - 1u));
    if (q >= cap) return;
    pairs[2 * q] = min(x, y);
    pairs[2 * q + 1] = max(x, y);
    dout[q] = d;
}

// every pair incident to the given rows with d < cut, scored exactly (all N
// columns of each row), unique and ordered by (d, i, j): Algorithm 3's
// exhaustive scoring restricted to a node subset
recon_status row_best_run(recon_ctx *c, const int32_t *rows_dev, int64_t nrows, float cut, int32_t **pairs_dev,
                          float **d_dev, int64_t *count) {
    SearchBufs &S = SB(c);
    S.res_n = 0;
    *count = 0;
    const int64_t N = c->N;
    const int64_t nch = (N + 511) / 512;
    const int64_t B = std::max<int64_t>(1, std::min<int64_t>(nrows, ((int64_t)1 << 28) / N));
    GROW(S.seg_node, sizeof(int32_t) * B * nch);
    GROW(S.seg_start, sizeof(int64_t) * B * nch);
    GROW(S.seg_count, sizeof(int32_t) * B * nch);
    GROW(S.seg_vbase, sizeof(int32_t) * B * nch);
    GROW(S.ex_d, sizeof(float) * B * N);
    int64_t rcap = std::max<int64_t>((int64_t)S.res_d.bytes / sizeof(float), 1 << 16);
    GROW_KEEP(S.res_pairs, sizeof(int32_t) * 2 * rcap, 0);
    GROW_KEEP(S.res_d, sizeof(float) * rcap, 0);
    for (int64_t r0 = 0; r0 < nrows; r0 += B) {
        const int64_t nb = std::min(B, nrows - r0);
        k_row_segments<<<nblk(nb * nch), 256, 0, c->stream>>>(nb, N, nch, rows_dev + r0, (int32_t *)S.seg_node.p,
                                                              (int64_t *)S.seg_start.p, (int32_t *)S.seg_count.p,
                                                              (int32_t *)S.seg_vbase.p); note_launch();
        CKS(cudaGetLastError());
        recon_status st = score_segments_device(c, (int32_t *)S.seg_node.p, (int64_t *)S.seg_start.p,
                                                (int32_t *)S.seg_count.p, (int32_t *)S.seg_vbase.p, nb * nch,
                                                nullptr, nb * N, nullptr, (float *)S.ex_d.p);
        if (st != RECON_OK) return st;
        for (int attempt = 0; attempt < 2; ++attempt) {
            CKS(cudaMemsetAsync(counter(c, CNT_SCRATCH3), 0, sizeof(unsigned long long), c->stream));
            k_row_select<<<nblk(nb * N), 256, 0, c->stream>>>(nb, N, rows_dev + r0, (float *)S.ex_d.p, cut,
                                                               (int32_t *)S.res_pairs.p + 2 * S.res_n,
                                                               (float *)S.res_d.p + S.res_n, rcap - S.res_n,
                                                               counter(c, CNT_SCRATCH3)); note_launch();
            CKS(cudaGetLastError());
            unsigned long long got = 0;
            st = read_counter(c, CNT_SCRATCH3, &got);
            if (st != RECON_OK) return st;
            if (S.res_n + (int64_t)got <= rcap) {
                S.res_n += (int64_t)got;
                break;
            }
            // the output did not fit: grow it (keeping what is there) and select again
            rcap = S.res_n + (int64_t)got + (int64_t)got / 4 + 1024;
            GROW_KEEP(S.res_pairs, sizeof(int32_t) * 2 * rcap, sizeof(int32_t) * 2 * S.res_n);
            GROW_KEEP(S.res_d, sizeof(float) * rcap, sizeof(float) * S.res_n);
        }
    }
    recon_status st = check_err_flags(c, "row scoring");
    if (st != RECON_OK) return st;
    st = finish_results(c, std::max<int64_t>(S.res_n, 1), count);
    if (st != RECON_OK) return st;
    *pairs_dev = (int32_t *)S.out_pairs.p;
    *d_dev = (float *)S.out_d.p;
    return RECON_OK;
}

// the first level's lists of the last FindBest search, with global node ids
recon_status knn_graph_copy(recon_ctx *c, int32_t *ids, float *d, int64_t cap, int32_t *k_out, int64_t *n_out) {
    SearchBufs &S = SB(c);
    const int K = S.g0_K;
    const int64_t n = K > 0 ? S.g0_n : 0;
    if (k_out) *k_out = K;
    if (n_out) *n_out = n;
    if (!ids && !d) return RECON_OK;
    if (cap < n * K) return set_err(c, RECON_EINVAL, "cap %lld < N k = %lld", (long long)cap, (long long)(n * K));
    if (n == 0) return RECON_OK;
    const DBuf &bi = S.g0_moved ? S.g0_id : S.knn_id;
    const DBuf &bd = S.g0_moved ? S.g0_d : S.knn_d;
    std::vector<int32_t> hi((size_t)(n * K));
    std::vector<float> hd((size_t)(n * K));
    CKS(cudaMemcpyAsync(hi.data(), bi.p, sizeof(int32_t) * n * K, cudaMemcpyDeviceToHost, c->stream));
    CKS(cudaMemcpyAsync(hd.data(), bd.p, sizeof(float) * n * K, cudaMemcpyDeviceToHost, c->stream));
    CKS(cudaStreamSynchronize(c->stream));
    // NNDescent keeps its rows ascending; the exhaustive k-NN selection does
    // not order them, so rows are put in ascending d here (stable)
    std::vector<int> perm(K);
    for (int64_t x = 0; x < n; ++x) {
        const float *dr = hd.data() + x * K;
        const int32_t *ir = hi.data() + x * K;
        for (int r = 0; r < K; ++r) perm[r] = r;
        std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return dr[a] < dr[b]; });
        for (int r = 0; r < K; ++r) {
            if (ids) ids[x * K + r] = ir[perm[r]];
            if (d) d[x * K + r] = dr[perm[r]];
        }
    }
    return RECON_OK;
}
