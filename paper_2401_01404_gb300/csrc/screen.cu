// screen.cu -- the tensor-core gradient screen: every pair's gradient at
// W_ij = 0 at once, as one dense contraction on the 5th-generation tensor cores
// (tcgen05 MMA, TMA tile loads, TMEM accumulators), with a fused epilogue that
// keeps only the pairs whose exact gain can be nonzero.
//
// Why it is exact.  Under the Laplace prior, a pair at W_ij = 0 has a nonzero
// gain iff |F'(0)| > lambda (the subgradient condition at w = 0), where
//   Ising:    F'(0) = g_ij = sum_m [r_i x_j + x_i r_j],  r = x - tanh(phi)
//   Gaussian: a_ij = -sum_m [e_i x_j + x_i e_j],       e = x + s2 mu
// i.e. G = [R | X] [X | R]^T, a product of two N x 2Mp matrices.  The screen
// computes G with bf16 operands (or, for the Ising model on request, E4M3) and
// f32 accumulation; its error is bounded per pair: for the Ising model, whose
// spins are exact in both types, |dG_ij| <= e_i + e_j with e_i the node's
// actual rounding error sum_m |r~_im - r_im|, plus an accumulation allowance;
// for the Gaussian model (2u + u^2) l_i l_j.  Keeping every pair with
// |G~_ij| > lambda - margin_ij therefore loses none of the pairs with a nonzero
// gain.  The survivors, and every stored coupling, are then scored exactly in
// FP32; the m best of them are the exact m best pairs (the exhaustive base case
// of Algorithm 3 over the whole node set).  The gradient as a cheap proxy for d
// is the paper's own suggestion (App. B, "Gradient as distance").
//
// The empty network (W = 0, where Algorithm 2 starts).  Every sample of node i
// then has the same field, so t_im = tau_i for m < M and, with s_i = sum_m x_im,
//   g_ij = 2 sum_m x_im x_jm - tau_j s_i - tau_i s_j :
// G is the spin product X X^T (K = M instead of 2M) plus a rank-two correction
// applied in the epilogue.  The spins are exact in E4M3 and every partial sum of
// the product is an integer of magnitude <= M, so the tensor-core product is
// exact whatever the accumulator's width; the only error left is the FP32
// rounding of the correction, covered by a margin of Mp / 2048 (several hundred
// times that rounding, and also above the FP32 rounding of the exact scorer's
// own first pass, so that no pair the scorer gives a nonzero gain is dropped).
//
// Kernel layout: a persistent grid; each CTA walks 128x256 units of G: the two
// row halves of each 256x256 super-tile of the upper triangle (super-tiles in
// bands of 8 super-rows, for L2 reuse).  Warp 8 issues TMA loads of 128-row (A)
// and 256-row (B) tiles of 128-byte k-block rows (64 bf16 or 128 E4M3; 128-byte
// swizzle) into a 4-stage ring, warp 9 issues tcgen05.mma (M=128, N=256, K=16
// bf16 / 32 E4M3) into one of two TMEM accumulators of 256 columns, and warps
// 0-7 drain the other accumulator (tcgen05.ld; warp w reads TMEM lanes
// 32 (w % 4) .. + 31, one row per thread, and columns 128 (w / 4) .. + 127)
// and stage the surviving pairs.  With K = Mp (224 at M = 200) a unit's MMAs
// take about half a microsecond, less than the round trip of either handoff
// (a stage: MMA commit -> producer -> TMA -> MMA issuer; an accumulator: MMA
// commit -> epilogue -> MMA issuer), and two 256-column accumulators fill the
// TMEM: the handoffs, not the tensor pipe, set the screen's pace.  So the
// epilogue reads each half of its columns once for a maximum, hands the
// accumulator back at once when no row of the warp can pass (nearly always),
// and reads the passing halves again only otherwise.  Every wait is bounded
// (1 s); on a timeout the kernel sets an error word, lets its own copies
// land, frees TMEM and returns.
//
// The CTA-pair form (recon_options.screen_pair; tcgen05 cta_group::2 in
// clusters of two): one M = 256 MMA covers both CTAs' units of a super-tile,
// each CTA loading its 128 rows of A and half of B (32 KB stages, six of them);
// the commits arrive on both CTAs' barriers, the peer's tile bytes and its
// epilogue's releases on the leader's.  It moves a third less operand data
// per SM, but its accumulator handoff crosses the pair and it measures 5-7 %
// slower, so the one-CTA form is the default.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "common.cuh"

namespace {

// a unit of work is a 128 x 256 block of G: rows BM from A, columns BN from B;
// units are the two 128-row halves of the 256 x 256 super-tiles (SUP) of the
// upper triangle
// BK: elements of a 128-byte k-block row: 64 in bf16, 128 in fp8
constexpr int BM = 128, BN = 256, SUP = 256, BK = 64, BK8 = 128, STAGES = 4;
constexpr int A_BYTES = BM * 128, B_BYTES = BN * 128;
constexpr uint32_t TMEM_COLS = 512;  // two accumulators of 256 f32 columns
// warps 0-7: epilogue (row group w % 4, column half w / 4); 8: TMA producer; 9: MMA issuer
constexpr int EPI_WARPS = 8, PRODUCER_WARP = 8, MMA_WARP = 9, THREADS = 32 * (EPI_WARPS + 2);
// survivors are staged per epilogue warp in shared memory and written out in
// batches: one atomic reservation and one round of stored-coupling lookups per batch
constexpr int SBUF = 128;
// The CTA-pair form (tcgen05 cta_group::2, a cluster of two CTAs on the two SMs
// of a TPC): one MMA of M = 256 covers both CTAs' 128-row units of a super-tile.
// Each CTA holds its own 128 rows of A and one half (128 rows) of the 256 rows of
// B per k-block, and its TMEM holds its 128 x 256 block of the product.  A stage
// is then 32 KB instead of 48, so six stages fit where the single-CTA form has
// four: three units of operands in flight per SM instead of two.
template <bool PAIR>
struct Geo {
    static constexpr int stages = PAIR ? 6 : STAGES;
    static constexpr int b_rows = PAIR ? BN / 2 : BN;  // rows of B held by one CTA
    static constexpr int b_bytes = b_rows * 128;
    static constexpr int m = PAIR ? 2 * BM : BM;       // rows of one MMA
};

// bounded wait (about 1 s of wall time); false on timeout or when another role
// gave up.  The global timer is a slow special-register read, so it is read only
// every 256 failed polls (a completed barrier costs one try_wait and no read).
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t par, volatile int *abort) {
    if (mbar_try(b, par)) return true;
    uint64_t t0 = 0;
    for (uint32_t n = 1;; ++n) {
        if (mbar_try(b, par)) return true;
        if ((n & 255u) == 0) {
            if (*abort) return false;
            const uint64_t now = gtimer();
            if (t0 == 0)
                t0 = now;
            else if (now - t0 > 1000000000ull) {
                *abort = 1;
                return false;
            }
        }
    }
}
__device__ __forceinline__ void tma_2d(void *dst, const CUtensorMap *tm, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            su32(dst)),
        "l"(tm), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t desc_sw128(const void *p) {
    const uint64_t a = su32(p);
    return ((a >> 4) & 0x3FFFull) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
// FP8 (E4M3 x E4M3) operands, K = 32 per instruction, FP32 accumulation
__device__ __forceinline__ void mma_fp8(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// --- the CTA-pair forms (every tcgen05 instruction of a kernel names one CTA group)
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// the shared::cluster address of the same shared-memory location in CTA `rank`
__device__ __forceinline__ uint32_t map_rank(const void *p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(su32(p)), "r"(rank));
    return r;
}
// (default semantics: the arrival only says that this warp's TMEM loads have
// completed; a cluster-scope release would also wait for its outstanding global
// loads, and measured a third slower)
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
// the tile lands in this CTA's shared memory; its bytes count on the mbarrier at
// a shared::cluster address (the leader CTA's)
__device__ __forceinline__ void tma_2d_pair(void *dst, const CUtensorMap *tm, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.cta_group::2 [%0], [%1, {%2, "
        "%3}], [%4];" ::"r"(su32(dst)),
        "l"(tm), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
template <bool PAIR>
__device__ __forceinline__ void mma_f8(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if constexpr (PAIR)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    else
        mma_fp8(d, a, b, idesc, acc);
}
template <bool PAIR>
__device__ __forceinline__ void mma_16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if constexpr (PAIR)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    else
        mma_bf16(d, a, b, idesc, acc);
}
// the commit's arrival reaches the mbarrier at this offset in both CTAs of the pair
template <bool PAIR>
__device__ __forceinline__ void commit(uint64_t *bar) {
    if constexpr (PAIR) {
        const uint16_t both = 3;
        asm volatile(
            "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
                su32(bar)),
            "h"(both)
            : "memory");
    } else {
        mma_commit(bar);
    }
}
// TMEM: in the pair form one warp of each CTA takes part in the allocation
template <bool PAIR>
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t cols) {
    if constexpr (PAIR) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)), "r"(cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
    } else {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)), "r"(cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
}
template <bool PAIR>
__device__ __forceinline__ void tmem_dealloc(uint32_t tmem, uint32_t cols) {
    if constexpr (PAIR)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
    else
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
}

#define TMEM_LD32(r, taddr)                                                                                        \
    asm volatile(                                                                                                  \
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%" \
        "19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                                              \
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),          \
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),    \
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),  \
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])   \
        : "r"(taddr))

// Tile order over the upper triangle (bi <= bj) of a T x T tile grid: bands of
// GROUP tile rows, each band walked column by column (in a column, its rows in
// order).  The tiles that the persistent CTAs hold at one time then form a
// compact block of about GROUP rows x (grid / GROUP) columns: the band's A tiles
// stay in L2 for the whole band, and each B tile is read from memory once per
// band instead of once per tile row.
constexpr int GROUP = 8;
__device__ __forceinline__ int64_t band_start(int64_t g, int64_t T) {
    // tiles before band g; every band before it is full
    return g * GROUP * (GROUP + 1) / 2 + (int64_t)GROUP * (g * T - (int64_t)GROUP * g * (g + 1) / 2);
}
__device__ __forceinline__ void tile_of(int64_t t, int T, int &bi, int &bj) {
    const int64_t nb = ((int64_t)T + GROUP - 1) / GROUP;
    int64_t lo = 0, hi = nb - 1;
    while (lo < hi) {  // the last band that starts at or before t
        const int64_t mid = (lo + hi + 1) / 2;
        if (band_start(mid, T) <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    const int64_t r0 = lo * GROUP;
    const int64_t Gb = min((int64_t)GROUP, (int64_t)T - r0);
    int64_t u = t - band_start(lo, T);
    const int64_t tri = Gb * (Gb + 1) / 2;
    if (u < tri) {  // the band's own triangle: column c holds rows r0 .. r0 + c
        int64_t c = 0;
        while ((c + 1) * (c + 2) / 2 <= u) ++c;
        bi = (int)(r0 + u - c * (c + 1) / 2);
        bj = (int)(r0 + c);
        return;
    }
    u -= tri;
    bi = (int)(r0 + u % Gb);
    bj = (int)(r0 + Gb + u / Gb);
}

// Unit u is half u & 1 of super-tile u >> 1.  Each role of a CTA visits its
// units in increasing order, so the band only moves forward: the walker keeps
// the current band and its start, and maps a unit with 32-bit arithmetic
// (tile_of above is the same order in closed form).
struct UnitWalker {
    int T;
    int64_t nb, g = -1, g_start = 0, g_next = 0;
    __device__ explicit UnitWalker(int T_) : T(T_), nb(((int64_t)T_ + GROUP - 1) / GROUP) {}
    // first row of A and of B of unit u
    __device__ __forceinline__ void map(int64_t u, int &ra, int &rb) {
        const int64_t st = u >> 1;
        if (g < 0) {
            int bi, bj;
            tile_of(st, T, bi, bj);
            g = bi / GROUP;
            g_start = band_start(g, T);
            g_next = g + 1 < nb ? band_start(g + 1, T) : INT64_MAX;
        }
        while (st >= g_next) {
            ++g;
            g_start = g_next;
            g_next = g + 1 < nb ? band_start(g + 1, T) : INT64_MAX;
        }
        const int r0 = (int)(g * GROUP);
        const int Gb = min(GROUP, T - r0);
        uint32_t v = (uint32_t)(st - g_start);
        const uint32_t tri = (uint32_t)(Gb * (Gb + 1) / 2);
        int bi, bj;
        if (v < tri) {
            uint32_t c = 0;
            while ((c + 1) * (c + 2) / 2 <= v) ++c;
            bi = r0 + (int)(v - c * (c + 1) / 2);
            bj = r0 + (int)c;
        } else {
            v -= tri;
            if (Gb == GROUP) {
                bi = r0 + (int)(v % GROUP);
                bj = r0 + Gb + (int)(v / GROUP);
            } else {
                bi = r0 + (int)(v % (uint32_t)Gb);
                bj = r0 + Gb + (int)(v / (uint32_t)Gb);
            }
        }
        ra = bi * SUP + (int)(u & 1) * BM;
        rb = bj * SUP;
    }
};

struct ScreenArgs {
    int n;              // nodes
    int T;              // super-tiles per side
    int64_t ntiles;     // units: 2 T (T + 1) / 2
    int nk;             // K / BK (K / BK8 for fp8)
    int last_mma;       // MMAs issued for the last k-block (trailing zero padding skipped)
    float lambda;
    float rel_err;      // margin per unit of the per-node norms
    float abs_margin;   // plus this much
    int product_margin; // margin rel_err * l_i * l_j (Gaussian) instead of rel_err * (l_i + l_j)
    const float *l1;    // per-node norms of the margin
    const float2 *r1;   // rank-one form: per node (s_i, tau_i)
    WTable W;           // pairs with a stored coupling are left to the caller
    int skip_stored;    // leave out pairs that hold a stored coupling
    int32_t *out;       // survivors (i, j), i < j
    int64_t cap;
    unsigned long long *count;
    unsigned long long *err;
    int stall;          // fault injection: issue no loads, so the bounded waits run out
    int shard, nshard;  // this launch covers work items shard, shard + nshard, ... (a shard of the screen)
    int64_t nlocal;     // work items of this shard: units, or in the pair form super-tiles
};

// PAIR: the CTA-pair form, launched in clusters of two; CTA rank r of a pair
// works on unit 2 st + r of super-tile st (its 128 rows), rank 0 issues the MMAs
template <bool F8, bool R1, bool PAIR>
__global__ void __launch_bounds__(THREADS, 1) k_screen(const __grid_constant__ CUtensorMap tA,
                                                       const __grid_constant__ CUtensorMap tB, ScreenArgs a) {
    using G = Geo<PAIR>;
    // k-blocks per stage: the rank-one form (K = Mp, two k-blocks at M = 200) keeps a
    // unit's k-blocks in one stage, so that its MMA thread polls one full barrier and
    // commits one empty barrier per unit instead of one per k-block; at K = 224 that
    // thread's polls and commits take as long as the tensor pipe's work.  The same
    // bytes in flight: two stages of two k-blocks instead of four of one.
    constexpr int KPS = (R1 && !PAIR) ? 2 : 1;
    constexpr int NST = G::stages / KPS;
    static_assert(NST * KPS == G::stages, "stages hold whole k-block groups");
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem, *sB = smem + NST * KPS * A_BYTES;
    uint64_t *full = (uint64_t *)(sB + NST * KPS * G::b_bytes);
    uint64_t *empty = full + NST;
    uint64_t *acc_full = empty + NST;      // [2]
    uint64_t *acc_empty = acc_full + 2;    // [2]
    uint32_t *tmem_slot = (uint32_t *)(acc_empty + 2);
    int *abort = (int *)(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // the pair form: rank 0 (the leader) issues the MMAs; its full barriers count
    // both CTAs' tile bytes and its accumulator-empty barriers both CTAs' epilogues
    const uint32_t rank = PAIR ? cluster_rank() : 0u;
    // One stage per unit (the rank-one form with K <= 2 k-blocks): the producer also
    // waits for the unit's accumulator to be free and then adds a second arrival to
    // the stage's full barrier, so the MMA thread polls one barrier per unit (each
    // poll costs that thread about 80 ns, and its polls, MMA issues and commits are
    // what bound the screen at K = 224).
    const bool unit_stage = KPS > 1 && a.nk <= KPS;
    const int64_t wi0 = PAIR ? (int64_t)(blockIdx.x >> 1) : (int64_t)blockIdx.x;  // first work item
    const int64_t wstep = PAIR ? (int64_t)(gridDim.x >> 1) : (int64_t)gridDim.x;
    // the unit this CTA works on for work item t
    auto unit_of = [&](int64_t t) -> int64_t {
        const int64_t g = a.shard + a.nshard * t;
        return PAIR ? 2 * g + rank : g;
    };
    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(full + s, unit_stage ? 2 : 1);
            mbar_init(empty + s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(acc_full + b, 1);
            mbar_init(acc_empty + b, (PAIR ? 2 : 1) * EPI_WARPS);  // one arrival per epilogue warp
        }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == MMA_WARP) tmem_alloc<PAIR>(tmem_slot, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    if constexpr (PAIR) cluster_sync();  // the peer's barriers exist before anything arrives on them
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == PRODUCER_WARP) {
        if (lane == 0) {  // TMA producer
            UnitWalker walk(a.T);
            int64_t kb_all = 0;  // stages filled so far
            for (int64_t t = wi0; t < a.nlocal && !a.stall && !*(volatile int *)abort; t += wstep) {
                int ra, rb;
                walk.map(unit_of(t), ra, rb);
                for (int kb = 0; kb < a.nk; kb += KPS, ++kb_all) {
                    const int s = (int)(kb_all % NST);
                    if (!mbar_wait(empty + s, (uint32_t)(((kb_all / NST) & 1) ^ 1), abort)) break;
                    const int x = kb * (F8 ? BK8 : BK);
                    if constexpr (KPS > 1) {
                        const int nkb = min(KPS, a.nk - kb);
                        mbar_expect_tx(full + s, (uint32_t)nkb * (A_BYTES + B_BYTES));
                        for (int j = 0; j < nkb; ++j) {
                            const int xj = (kb + j) * (F8 ? BK8 : BK);
                            tma_2d(sA + (s * KPS + j) * A_BYTES, &tA, xj, ra, full + s);
                            tma_2d(sB + (s * KPS + j) * B_BYTES, &tB, xj, rb, full + s);
                        }
                        if (unit_stage) {  // unit kb_all's accumulator, then the second arrival
                            if (!mbar_wait(acc_empty + (kb_all & 1), (uint32_t)(((kb_all >> 1) & 1) ^ 1), abort))
                                break;
                            mbar_arrive(full + s);
                        }
                    } else if constexpr (PAIR) {
                        // both CTAs' tiles count on the leader's full barrier
                        if (rank == 0) mbar_expect_tx(full + s, 2 * (A_BYTES + G::b_bytes));
                        const uint32_t fb = map_rank(full + s, 0);
                        tma_2d_pair(sA + s * A_BYTES, &tA, x, ra, fb);
                        tma_2d_pair(sB + s * G::b_bytes, &tB, x, rb + (int)rank * G::b_rows, fb);
                    } else {
                        mbar_expect_tx(full + s, A_BYTES + B_BYTES);
                        tma_2d(sA + s * A_BYTES, &tA, x, ra, full + s);
                        tma_2d(sB + s * B_BYTES, &tB, x, rb, full + s);
                    }
                }
            }
            // let every copy issued above land before the CTA can leave (the leader's
            // full barriers count the peer's copies too); in the pair form each CTA
            // also waits for the MMAs' last reads of its stages (their commits arrive
            // on its empty barriers), unless the screen gave up
            if (kb_all > 0) {
                const int64_t first = kb_all > NST ? kb_all - NST : 0;
                for (int64_t q = first; q < kb_all; ++q) {
                    if (!PAIR || rank == 0) {
                        const uint64_t t0 = gtimer();
                        while (!mbar_try(full + (q % NST), (uint32_t)((q / NST) & 1)))
                            if (gtimer() - t0 > 1000000000ull) break;
                    }
                    if (PAIR && !*(volatile int *)abort) {
                        const uint64_t t0 = gtimer();
                        while (!mbar_try(empty + (q % NST), (uint32_t)((q / NST) & 1)))
                            if (gtimer() - t0 > 1000000000ull) break;
                    }
                }
            }
        }
    } else if (warp == MMA_WARP) {
        if (lane == 0 && rank == 0) {  // MMA issuer (in the pair form, the leader's only)
            // F32 accumulator; A and B bf16 (kind::f16: type 1) or E4M3 (kind::f8f6f4: type 0);
            // M = 256 in the pair form (128 rows per CTA), N = 256
            const uint32_t ab = F8 ? 0u : 1u;
            const uint32_t idesc = (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(BN >> 3) << 17) |
                                   ((uint32_t)(G::m >> 4) << 24);
            int64_t kb_all = 0, it = 0, last_it = -1;  // last_it: the unit of the last accumulator commit
            for (int64_t t = wi0; t < a.nlocal && !*(volatile int *)abort; t += wstep, ++it) {
                const int b = (int)(it & 1);
                // (one stage per unit: the stage's full barrier already includes this)
                if (!unit_stage && !mbar_wait(acc_empty + b, (uint32_t)(((it >> 1) & 1) ^ 1), abort)) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * BN);
                bool ok = true;
                for (int kb0 = 0; kb0 < a.nk; kb0 += KPS, ++kb_all) {
                    const int s = (int)(kb_all % NST);
                    if (!mbar_wait(full + s, (uint32_t)((kb_all / NST) & 1), abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int j = 0; j < KPS; ++j) {
                    const int kb = kb0 + j;
                    if (KPS > 1 && kb >= a.nk) break;
                    const uint64_t da = desc_sw128(sA + (s * KPS + j) * A_BYTES),
                                   db = desc_sw128(sB + (s * KPS + j) * G::b_bytes);
                    // four MMAs per 128-byte k-block row (K = 16 bf16 or 32 fp8 each, 32 bytes
                    // apart: +2 in the descriptor's 16-byte address units)
                    // (straight-line issue: a data-dependent branch between the MMAs of a
                    // k-block cost the bf16 path about a tenth of its throughput)
                    if constexpr (F8) {
                        // the k-block's MMA count is chosen once, before the first MMA:
                        // each count issues its MMAs in straight line
                        const int nm = kb + 1 < a.nk ? 4 : a.last_mma;
                        if (nm == 4) {
#pragma unroll
                            for (int k = 0; k < 4; ++k) mma_f8<PAIR>(d, da + 2 * k, db + 2 * k, idesc, (kb | k) != 0);
                        } else if (nm == 3) {
#pragma unroll
                            for (int k = 0; k < 3; ++k) mma_f8<PAIR>(d, da + 2 * k, db + 2 * k, idesc, (kb | k) != 0);
                        } else if (nm == 2) {
#pragma unroll
                            for (int k = 0; k < 2; ++k) mma_f8<PAIR>(d, da + 2 * k, db + 2 * k, idesc, (kb | k) != 0);
                        } else {
                            mma_f8<PAIR>(d, da, db, idesc, kb != 0);
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < 4; ++k) mma_16<PAIR>(d, da + 2 * k, db + 2 * k, idesc, (kb | k) != 0);
                    }
                    }  // k-blocks of the stage
                    commit<PAIR>(empty + s);
                }
                commit<PAIR>(acc_full + b);
                last_it = it;
                if (!ok) break;
            }
            // after an abort, the MMAs already issued may still be reading the stages and
            // writing TMEM: wait (bounded) for the last commit, which tracks all of them,
            // before the CTA frees TMEM and leaves
            if (last_it >= 0 && *(volatile int *)abort) {
                const uint64_t t0 = gtimer();
                while (!mbar_try(acc_full + (last_it & 1), (uint32_t)((last_it >> 1) & 1)))
                    if (gtimer() - t0 > 1000000000ull) break;
            }
        }
    } else {  // epilogue warps: row 32 (warp % 4) + lane, columns 128 (warp / 4) .. + 127 of each unit
        const int rg = warp & 3, ch = warp >> 2;
        // per-warp copy of its 128 column norms (the margin's l_j), or in the
        // rank-one form of its columns' s_j (first 128) and tau_j (next 128), read
        // as 128-bit broadcasts
        float *cn = (float *)(smem + STAGES * (A_BYTES + B_BYTES) + 256) + warp * BN;
        int2 *sbuf = (int2 *)(smem + STAGES * (A_BYTES + B_BYTES) + 256 + EPI_WARPS * BN * sizeof(float)) +
                     warp * SBUF;
        int nbuf = 0;  // warp-uniform fill of sbuf
        // write the staged survivors: each lane checks up to SBUF / 32 entries against
        // the stored couplings (independent loads), then one reservation for the warp
        auto flush = [&]() {
            uint32_t keep = 0;
#pragma unroll
            for (int u = 0; u < SBUF / 32; ++u) {
                const int e = 32 * u + lane;
                if (e < nbuf) {
                    const int2 pr = sbuf[e];
                    if (!(a.skip_stored && wt_contains(a.W, pair_key(pr.x, pr.y)))) keep |= 1u << u;
                }
            }
            int kc = __popc(keep), incl = kc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            unsigned long long base = 0;
            if (lane == 0 && total) base = atomicAdd(a.count, (unsigned long long)total);
            base = __shfl_sync(0xffffffffu, base, 0);
            int64_t pos = (int64_t)base + incl - kc;
#pragma unroll
            for (int u = 0; u < SBUF / 32; ++u) {
                if (keep >> u & 1u) {
                    if (pos < a.cap) {
                        const int2 pr = sbuf[32 * u + lane];
                        a.out[2 * pos] = pr.x;
                        a.out[2 * pos + 1] = pr.y;
                    }
                    ++pos;
                }
            }
            __syncwarp();
            nbuf = 0;
        };
        UnitWalker walk(a.T);
        // the column norms l_j of a unit: lane holds columns 4 lane .. 4 lane + 3 of
        // the warp's half, loaded one unit ahead so that their latency hides
        // behind the compare
        // (rank-one form: n0 = s_j and n1 = tau_j of the four columns)
        auto load_norms = [&](int jt, float4 &n0, float4 &n1) {
            const int j = jt + (BN / 2) * ch + 4 * lane;
            if constexpr (R1) {
                if (j + 3 < a.n) {
                    const float4 p0 = *(const float4 *)(a.r1 + j), p1 = *(const float4 *)(a.r1 + j + 2);
                    n0 = make_float4(p0.x, p0.z, p1.x, p1.z);
                    n1 = make_float4(p0.y, p0.w, p1.y, p1.w);
                } else {
                    float q[4], w[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float2 e = j + u < a.n ? a.r1[j + u] : make_float2(0.f, 0.f);
                        q[u] = e.x;
                        w[u] = e.y;
                    }
                    n0 = make_float4(q[0], q[1], q[2], q[3]);
                    n1 = make_float4(w[0], w[1], w[2], w[3]);
                }
            } else if (a.l1 && j + 3 < a.n) {
                n0 = *(const float4 *)(a.l1 + j);
            } else {
                float q[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) q[u] = (a.l1 && j + u < a.n) ? a.l1[j + u] : 0.f;
                n0 = make_float4(q[0], q[1], q[2], q[3]);
            }
        };
        // the row's l_i, or in the rank-one form its (s_i, tau_i)
        auto load_row = [&](int ra_) {
            const int i_ = ra_ + 32 * rg + lane;
            if constexpr (R1) return i_ < a.n ? a.r1[i_] : make_float2(0.f, 0.f);
            else return make_float2((a.l1 && i_ < a.n) ? a.l1[i_] : 0.f, 0.f);
        };
        int ra = 0, jt = 0;
        float4 n0 = make_float4(0.f, 0.f, 0.f, 0.f), n1 = n0;
        float2 li_n = make_float2(0.f, 0.f);
        if (wi0 < a.nlocal) {
            walk.map(unit_of(wi0), ra, jt);
            load_norms(jt, n0, n1);
            li_n = load_row(ra);
        }
        int64_t it = 0;
        for (int64_t t = wi0; t < a.nlocal; t += wstep, ++it) {
            const int b = (int)(it & 1);
            const int i = ra + 32 * rg + lane;
            const int jt_cur = jt + (BN / 2) * ch;
            // keep iff |g| > lambda - margin, written |g| + s c_j > thr:
            //   sum margin     rel (l_i + l_j):  c_j = rel l_j, s = 1,        thr = lambda - rel l_i
            //   product margin rel l_i l_j:      c_j = l_j,     s = rel l_i,  thr = lambda
            // rank-one form: g = 2 S_ij - (tau_j s_i + tau_i s_j), thr = lambda - abs_margin,
            //   and |tau_j s_i + tau_i s_j| <= cb = |s_i| max |tau_j| + |tau_i| max |s_j|
            const float li = li_n.x;
            float sc, thr, cmax, thr_q;  // thr_q: the unit-level test's threshold
            if constexpr (R1) {
                ((float4 *)cn)[lane] = n0;
                ((float4 *)(cn + BN / 2))[lane] = n1;
                // abs values order like their bit patterns: one reduction each
                const float umax = __uint_as_float(__reduce_max_sync(
                    0xffffffffu, __float_as_uint(fmaxf(fmaxf(fabsf(n0.x), fabsf(n0.y)), fmaxf(fabsf(n0.z), fabsf(n0.w))))));
                const float vmax = __uint_as_float(__reduce_max_sync(
                    0xffffffffu, __float_as_uint(fmaxf(fmaxf(fabsf(n1.x), fabsf(n1.y)), fmaxf(fabsf(n1.z), fabsf(n1.w))))));
                sc = 1.f;
                cmax = fabsf(li) * vmax + fabsf(li_n.y) * umax;
                thr = a.lambda - a.abs_margin;
                // the unit-level test is a bound with its own FP32 roundings (a few
                // units of 2^-24 of 4 Mp): a sixteenth of the margin absorbs them
                thr_q = thr - 0.0625f * a.abs_margin;
            } else {
                sc = a.product_margin ? a.rel_err * li : 1.f;
                thr = (a.product_margin ? a.lambda : a.lambda - a.rel_err * li) - a.abs_margin;
                const float f = a.product_margin ? 1.f : a.rel_err;
                const float4 c0 = make_float4(f * n0.x, f * n0.y, f * n0.z, f * n0.w);
                ((float4 *)cn)[lane] = c0;
                // the warp's largest c_j in one reduction: c_j >= +0, whose bit patterns
                // order like the values
                cmax = __uint_as_float(
                    __reduce_max_sync(0xffffffffu, __float_as_uint(fmaxf(fmaxf(c0.x, c0.y), fmaxf(c0.z, c0.w)))));
                thr_q = thr;
            }
            const float ui = li, vi = li_n.y;
            // the next unit's mapping and norms, in flight during this unit's compare
            if (t + wstep < a.nlocal) {
                walk.map(unit_of(t + wstep), ra, jt);
                load_norms(jt, n0, n1);
                li_n = load_row(ra);
            }
            __syncwarp();
            // all lanes leave together: the loads and shuffles below are warp-wide
            if (!__all_sync(0xffffffffu, mbar_wait(acc_full + b, (uint32_t)((it >> 1) & 1), abort))) break;
            tc_fence_after();
            const uint32_t taddr = tmem + ((uint32_t)(32 * rg) << 16) + (uint32_t)(b * BN + (BN / 2) * ch);
            // First pass: max |g| of each 64-column half (eight independent running
            // maxima: one chain would serialise 64 dependent max operations) against
            // the unit's loosest threshold thr - s max c_j.  When no row of the warp
            // passes (the common case), the accumulator goes back to the MMA issuer at
            // once and the next unit's MMAs run while the warp moves on; otherwise
            // the passing halves are read again for the exact test, and the
            // accumulator is released after it.
            static_assert(BN == 256, "two 64-column halves per epilogue warp");
            bool pass[BN / 128];
#pragma unroll
            for (int hf = 0; hf < BN / 128; ++hf) {
                uint32_t r[64];
                TMEM_LD32(r, taddr + (uint32_t)(64 * hf));
                TMEM_LD32((r + 32), taddr + (uint32_t)(64 * hf + 32));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                float m8[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) m8[u] = fabsf(__uint_as_float(r[u]));
#pragma unroll
                for (int q = 8; q < 64; ++q) m8[q & 7] = fmaxf(m8[q & 7], fabsf(__uint_as_float(r[q])));
                const float m = fmaxf(fmaxf(fmaxf(m8[0], m8[1]), fmaxf(m8[2], m8[3])),
                                      fmaxf(fmaxf(m8[4], m8[5]), fmaxf(m8[6], m8[7])));
                pass[hf] = (R1 ? 2.f * m : m) + sc * cmax > thr_q;
            }
            auto release = [&]() {
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    if constexpr (PAIR)
                        mbar_arrive_cluster(map_rank(acc_empty + b, 0));  // the leader's barrier
                    else
                        mbar_arrive(acc_empty + b);
                }
            };
            bool hold = false;
#pragma unroll
            for (int hf = 0; hf < BN / 128; ++hf) hold |= pass[hf];
            if (!__any_sync(0xffffffffu, hold)) {
                release();
                continue;
            }
            // the exact test of the passing halves, 64 columns at a time; the warp
            // then stages its survivors
#pragma unroll 1
            for (int hf = 0; hf < BN / 128; ++hf) {
                const bool ph = hf == 0 ? pass[0] : pass[1];
                if (!__any_sync(0xffffffffu, ph)) continue;
                uint32_t r[64];
                TMEM_LD32(r, taddr + (uint32_t)(64 * hf));
                TMEM_LD32((r + 32), taddr + (uint32_t)(64 * hf + 32));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                unsigned long long mk = 0;
                const int j0 = jt_cur + 64 * hf;
                if (ph) {
                    // exact test of the 64 columns as a bit mask (branch-free), then
                    // j > i, j < n and the stored couplings, then one reservation
                    const float4 *c4p = (const float4 *)(cn + 64 * hf);
                    // two 32-bit halves, four partial masks each: short dependency chains
                    uint32_t mw[2][4] = {{0u, 0u, 0u, 0u}, {0u, 0u, 0u, 0u}};
                    if constexpr (R1) {
                        const float4 *v4p = (const float4 *)(cn + BN / 2 + 64 * hf);
#pragma unroll
                        for (int q4 = 0; q4 < 16; ++q4) {
                            const float4 u4 = c4p[q4], v4 = v4p[q4];
                            const int h = q4 >> 3, sh = 4 * (q4 & 7);
                            // g = 2 S - (tau_j s_i + tau_i s_j)
#define R1_BIT(k, uu, vv)                                                                                       \
    mw[h][k] |= (uint32_t)(fabsf(fmaf(2.f, __uint_as_float(r[4 * q4 + k]), -fmaf(vv, ui, vi * uu))) > thr)      \
                << (sh + k)
                            R1_BIT(0, u4.x, v4.x);
                            R1_BIT(1, u4.y, v4.y);
                            R1_BIT(2, u4.z, v4.z);
                            R1_BIT(3, u4.w, v4.w);
#undef R1_BIT
                        }
                    } else {
#pragma unroll
                        for (int q4 = 0; q4 < 16; ++q4) {
                            const float4 c4 = c4p[q4];
                            const int h = q4 >> 3, sh = 4 * (q4 & 7);
                            mw[h][0] |= (uint32_t)(fabsf(__uint_as_float(r[4 * q4 + 0])) + sc * c4.x > thr) << (sh + 0);
                            mw[h][1] |= (uint32_t)(fabsf(__uint_as_float(r[4 * q4 + 1])) + sc * c4.y > thr) << (sh + 1);
                            mw[h][2] |= (uint32_t)(fabsf(__uint_as_float(r[4 * q4 + 2])) + sc * c4.z > thr) << (sh + 2);
                            mw[h][3] |= (uint32_t)(fabsf(__uint_as_float(r[4 * q4 + 3])) + sc * c4.w > thr) << (sh + 3);
                        }
                    }
                    mk = (unsigned long long)((mw[0][0] | mw[0][1]) | (mw[0][2] | mw[0][3])) |
                         ((unsigned long long)((mw[1][0] | mw[1][1]) | (mw[1][2] | mw[1][3])) << 32);
                    const int below = i - j0;  // columns q <= below have j <= i
                    if (below >= 63)
                        mk = 0;
                    else if (below >= 0)
                        mk &= ~0ull << (below + 1);
                    const int valid = a.n - j0;  // columns q < valid have j < n
                    if (valid <= 0)
                        mk = 0;
                    else if (valid < 64)
                        mk &= ~0ull >> (64 - valid);
                }
                if (!__any_sync(0xffffffffu, mk != 0)) continue;  // the common case: no survivor in the warp
                const int cnt = __popcll(mk);
                int incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const int total = __shfl_sync(0xffffffffu, incl, 31);
                if (total > SBUF) {
                    // more than a batch at once (a penalty the screen cannot cut):
                    // each thread filters and reserves for itself
                    if (a.skip_stored) {  // stored couplings come separately
                        for (unsigned long long mm = mk; mm; mm &= mm - 1) {
                            const int q = __ffsll((long long)mm) - 1;
                            if (wt_contains(a.W, pair_key(i, j0 + q))) mk &= ~(1ull << q);
                        }
                    }
                    if (mk) {
                        int64_t pos = (int64_t)atomicAdd(a.count, (unsigned long long)__popcll(mk));
                        for (; mk; mk &= mk - 1, ++pos) {
                            const int q = __ffsll((long long)mk) - 1;
                            if (pos < a.cap) {
                                a.out[2 * pos] = i;
                                a.out[2 * pos + 1] = j0 + q;
                            }
                        }
                    }
                } else if (total > 0) {
                    if (nbuf + total > SBUF) flush();
                    int e = nbuf + incl - cnt;
                    for (; mk; mk &= mk - 1, ++e) sbuf[e] = make_int2(i, j0 + (__ffsll((long long)mk) - 1));
                    __syncwarp();
                    nbuf += total;
                }
            }
            release();
        }
        if (nbuf) flush();
    }
    tc_fence_before();
    __syncthreads();
    // the pair form: neither CTA leaves (or frees TMEM) while the other's MMAs,
    // copies or arrivals may still reach its shared memory
    if constexpr (PAIR) cluster_sync();
    if (warp == MMA_WARP) {
        tc_fence_after();
        tmem_dealloc<PAIR>(tmem, TMEM_COLS);
    }
    if (threadIdx.x == 0 && *abort) atomicOr(a.err + CNT_ERR, (unsigned long long)ERR_TIMEOUT);
}

// Ising operands: A_i = [r_i | x_i], B_i = [x_i | r_i] (bf16), r = x - t;
// padding samples have r = 0.  The spins are exact, so the product's error
// is |G~_ij - G_ij| <= sum_m |r~_im - r_im| + sum_m |r~_jm - r_jm| plus the
// accumulation's; each node's share q_i = (e_i + acc sum_m |r_im|)(1 + 2^-10)
// is written to q (e_i the node's actual rounding error, summed in FP32; the
// last factor covers that sum's own rounding), and the margin is q_i + q_j.
__global__ void k_prep_ising(IsingView v, __nv_bfloat16 *A, __nv_bfloat16 *B, float acc, float *q) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= v.N) return;
    const int K = 2 * v.Mp;
    float s = 0.f, e = 0.f;
    for (int m = lane; m < v.Mp; m += 32) {
        const float x = ((v.xbits[i * v.Mw + (m >> 5)] >> (m & 31)) & 1u) ? -1.f : 1.f;
        const float r = m < v.M ? x - v.t[i * v.Mp + m] : 0.f;
        const __nv_bfloat16 rb = __float2bfloat16_rn(r), xb = __float2bfloat16_rn(x);
        A[i * K + m] = rb;
        A[i * K + v.Mp + m] = xb;
        B[i * K + m] = xb;
        B[i * K + v.Mp + m] = rb;
        s += fabsf(r);
        e += fabsf(__bfloat162float(rb) - r);  // exact: both are floats within a factor 2
    }
    s = warp_sum(s);
    e = warp_sum(e);
    if (lane == 0) q[i] = (e + acc * s) * (1.f + 1.f / 1024.f);
}

// Gaussian operands: A_i = [e_i | x_i], B_i = [x_i | e_i] (bf16), and the
// margin's per-node norm l_i = |e_i|_2 + |x_i|_2
__global__ void k_prep_gauss(GaussView v, __nv_bfloat16 *A, __nv_bfloat16 *B, float *l1) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= v.N) return;
    const int K = 2 * v.Mp;
    float se = 0.f, sx = 0.f;
    for (int m = lane; m < v.Mp; m += 32) {
        const float x = v.xg[i * v.Mp + m], e = m < v.M ? v.e[i * v.Mp + m] : 0.f;
        const __nv_bfloat16 eb = __float2bfloat16_rn(e), xb = __float2bfloat16_rn(x);
        A[i * K + m] = eb;
        A[i * K + v.Mp + m] = xb;
        B[i * K + m] = xb;
        B[i * K + v.Mp + m] = eb;
        se += e * e;
        sx += x * x;
    }
    se = warp_sum(se);
    sx = warp_sum(sx);
    if (lane == 0) l1[i] = sqrtf(se) + sqrtf(sx);  // |e|_2 + |x|_2, combined with the partner's by the margin
}

// Ising operands in FP8 E4M3 (uint8 codes): the same rows, each padded with
// zeros to K8 = a multiple of 128 entries; spins are exact, residuals rounded
// to nearest (saturating, |r| < 2 anyway); q as for bf16, with the E4M3
// rounding errors
__global__ void k_prep_ising_fp8(IsingView v, int K8, uint8_t *A, uint8_t *B, float acc, float *q) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= v.N) return;
    float s = 0.f, e = 0.f;
    for (int m = 2 * v.Mp + lane; m < K8; m += 32) {
        A[i * K8 + m] = 0;
        B[i * K8 + m] = 0;
    }
    for (int m = lane; m < v.Mp; m += 32) {
        const float x = ((v.xbits[i * v.Mw + (m >> 5)] >> (m & 31)) & 1u) ? -1.f : 1.f;
        const float r = m < v.M ? x - v.t[i * v.Mp + m] : 0.f;
        const __nv_fp8_storage_t rb = __nv_cvt_float_to_fp8(r, __NV_SATFINITE, __NV_E4M3);
        const uint8_t xb = (uint8_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
        A[i * K8 + m] = (uint8_t)rb;
        A[i * K8 + v.Mp + m] = xb;
        B[i * K8 + m] = xb;
        B[i * K8 + v.Mp + m] = (uint8_t)rb;
        s += fabsf(r);
        // the code's value (E4M3 -> half is exact), minus r: exact in FP32
        e += fabsf(__half2float(__half(__nv_cvt_fp8_to_halfraw(rb, __NV_E4M3))) - r);
    }
    s = warp_sum(s);
    e = warp_sum(e);
    if (lane == 0) q[i] = (e + acc * s) * (1.f + 1.f / 1024.f);
}

// Operands of the rank-one form at the empty network: E4M3 spin rows (+-1 for
// the M samples, zero past them, K8 = Mp rounded up to 128 entries) and per node
// (s_i, tau_i) with s_i = sum_m x_im (exact) and tau_i = t_i of its first sample.
// A node whose t differs between its samples sets *flag (the caller then uses
// the general form).
__global__ void k_prep_ising_rank1(IsingView v, int K8, uint8_t *A, float2 *r1, unsigned long long *flag) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= v.N) return;
    const float tau = v.t[i * v.Mp];
    int s = 0;
    bool same = true;
    for (int m = lane; m < K8; m += 32) {
        float x = 0.f;
        if (m < v.M) {
            x = ((v.xbits[i * v.Mw + (m >> 5)] >> (m & 31)) & 1u) ? -1.f : 1.f;
            same &= v.t[i * v.Mp + m] == tau;
        }
        A[i * K8 + m] = (uint8_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
        s += (int)x;
    }
    s = warp_sum_i(s);
    const bool all_same = __all_sync(0xffffffffu, same);
    if (lane == 0) {
        r1[i] = make_float2((float)s, tau);
        if (!all_same) atomicOr(flag, 1ull);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

}  // namespace

// operand row length: 2 Mp bf16 entries, or 2 Mp fp8 entries padded to 128
int screen_k(recon_ctx *c, bool fp8) {
    const int k = 2 * (int)c->Mp;
    return fp8 ? (k + BK8 - 1) / BK8 * BK8 : k;
}

// operand row length of the rank-one form: Mp E4M3 entries padded to 128
int screen_k_rank1(recon_ctx *c) { return ((int)c->Mp + BK8 - 1) / BK8 * BK8; }

// the margin of the rank-one form (see the header)
float screen_rank1_margin(recon_ctx *c) { return (float)c->Mp / 2048.f; }

cudaError_t launch_screen_prep_rank1(recon_ctx *c, void *A, float2 *r1, unsigned long long *flag) {
    if (c->model != RECON_ISING) return cudaErrorInvalidValue;
    const unsigned grid = (unsigned)((c->N * 32 + 255) / 256);
    k_prep_ising_rank1<<<grid, 256, 0, c->stream>>>(c->iv(), screen_k_rank1(c), (uint8_t *)A, r1, flag);
    note_launch();
    return cudaGetLastError();
}

// bf16 (or, for the Ising model, fp8) operand rows and the margin's norms
cudaError_t launch_screen_prep(recon_ctx *c, void *A, void *B, float *l1, bool fp8) {
    const int64_t warps = c->N;
    const unsigned grid = (unsigned)((warps * 32 + 255) / 256);
    if (fp8) {
        if (c->model != RECON_ISING) return cudaErrorInvalidValue;
        k_prep_ising_fp8<<<grid, 256, 0, c->stream>>>(c->iv(), screen_k(c, true), (uint8_t *)A, (uint8_t *)B,
                                                       screen_acc_err(c, true), l1);
        note_launch();
        return cudaGetLastError();
    }
    if (c->model == RECON_ISING)
        k_prep_ising<<<grid, 256, 0, c->stream>>>(c->iv(), (__nv_bfloat16 *)A, (__nv_bfloat16 *)B,
                                                  screen_acc_err(c, false), l1);
    else
        k_prep_gauss<<<grid, 256, 0, c->stream>>>(c->gv(), (__nv_bfloat16 *)A, (__nv_bfloat16 *)B, l1);
    note_launch();
    return cudaGetLastError();
}

// The screen keeps (i, j) when |G~_ij| + margin_ij > lambda, with margin_ij
// at least the error of the tensor-core product G~ against the exact G.
// Ising: the prep kernel writes each node's share q_i of the margin (its
//   residuals' actual rounding error plus the accumulation allowance), and the
//   margin is 1 * (q_i + q_j).
// Gaussian: both operands are rounded to bf16 (unit roundoff u = 2^-8),
//   |dg_ij| <= (2u + u^2) sum_m (|e_i x_j| + |x_i e_j|)
//   <= (2u + u^2)(|e_i|_2 |x_j|_2 + |x_i|_2 |e_j|_2) <= (2u + u^2) l_i l_j with
//   l = |e|_2 + |x|_2 (Cauchy-Schwarz), plus the accumulation error.
float screen_rel_err(int model, int Mp, bool fp8) {
    (void)fp8;
    if (model == RECON_ISING) return 1.f;
    const double u = 1.0 / 256.0, acc = 2.0 * Mp * 1.2e-7;
    return (float)(2 * u + u * u + acc);
}

// The accumulation allowance per unit of sum_m |r_im| (the products r~ x are
// exact): bf16, K = 2 Mp FP32 additions, each off by at most 2^-24 of the
// running magnitude (charged 2^-23); E4M3, 2^-12 of the running magnitude per
// MMA (K = 32), which also covers an accumulator narrower than FP32.
float screen_acc_err(recon_ctx *c, bool fp8) {
    const double Mp = (double)c->Mp;
    return fp8 ? (float)((2.0 * Mp / 32.0 + 1.0) / 4096.0) : (float)(2.0 * Mp * 1.2e-7);
}

namespace {
template <bool PAIR>
constexpr size_t screen_smem() {
    return 1024 + (size_t)Geo<PAIR>::stages * (A_BYTES + Geo<PAIR>::b_bytes) + 256 + EPI_WARPS * BN * sizeof(float) +
           EPI_WARPS * SBUF * sizeof(int2);
}
template <class Kern>
cudaError_t set_smem(Kern k, size_t smem) {
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}
// the dynamic shared-memory size of each variant, set once per device
cudaError_t screen_set_smem(recon_ctx *c, int variant, bool pair) {
    static int attr_device[2][3] = {{-1, -1, -1}, {-1, -1, -1}};
    int &dev = attr_device[pair ? 1 : 0][variant];
    if (dev == c->device) return cudaSuccess;
    cudaError_t e;
    if (pair) {
        const size_t sm = screen_smem<true>();
        e = variant == 2   ? set_smem(k_screen<true, true, true>, sm)
            : variant == 1 ? set_smem(k_screen<true, false, true>, sm)
                           : set_smem(k_screen<false, false, true>, sm);
    } else {
        const size_t sm = screen_smem<false>();
        e = variant == 2   ? set_smem(k_screen<true, true, false>, sm)
            : variant == 1 ? set_smem(k_screen<true, false, false>, sm)
                           : set_smem(k_screen<false, false, false>, sm);
    }
    if (e == cudaSuccess) dev = c->device;
    return e;
}
cudaLaunchConfig_t pair_config(unsigned grid, size_t smem, cudaStream_t st, cudaLaunchAttribute *at) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}
template <class Kern>
cudaError_t launch_pair(Kern k, unsigned grid, size_t smem, cudaStream_t st, const CUtensorMap &ta,
                        const CUtensorMap &tb, const ScreenArgs &a) {
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = pair_config(grid, smem, st, at);
    return cudaLaunchKernelEx(&cfg, k, ta, tb, a);
}
// clusters of two that fit on the device at once (0: the pair form cannot run),
// per device and variant
int screen_pair_clusters(recon_ctx *c, int variant) {
    static int cached_dev[3] = {-1, -1, -1}, cached_n[3] = {0, 0, 0};
    if (cached_dev[variant] == c->device) return cached_n[variant];
    if (screen_set_smem(c, variant, true) != cudaSuccess) return 0;
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = pair_config(2u * (unsigned)c->num_sms, screen_smem<true>(), c->stream, at);
    int n = 0;
    cudaError_t e = variant == 2   ? cudaOccupancyMaxActiveClusters(&n, k_screen<true, true, true>, &cfg)
                    : variant == 1 ? cudaOccupancyMaxActiveClusters(&n, k_screen<true, false, true>, &cfg)
                                   : cudaOccupancyMaxActiveClusters(&n, k_screen<false, false, true>, &cfg);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        n = 0;
    }
    cached_dev[variant] = c->device;
    cached_n[variant] = n;
    return n;
}
}  // namespace

cudaError_t launch_screen_ex(recon_ctx *c, const void *A, const void *B, int K, float thr, const float *l1,
                             float rel, int product_margin, bool skip_stored, int32_t *out, int64_t cap,
                             unsigned long long *count, double *flop_out, bool fp8, float abs_margin,
                             int k_valid, const float2 *r1, bool use_shard) {
    if (r1 && !fp8) return cudaErrorInvalidValue;  // the rank-one form reads E4M3 spins
    const int bke = fp8 ? BK8 : BK;  // elements per 128-byte k-block row
    const int kchunk = fp8 ? 32 : 16;  // elements per MMA
    if (K % bke || k_valid <= K - bke || k_valid > K || k_valid % kchunk) return cudaErrorInvalidValue;
    if (!fp8 && k_valid != K) return cudaErrorInvalidValue;  // the bf16 path issues whole k-blocks
    if (!g_encode) {
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void **)&g_encode, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess || !g_encode) return e != cudaSuccess ? e : cudaErrorNotSupported;
    }
    // the pair form (on request): needs clusters of two co-resident CTAs at one per SM
    const int variant = r1 ? 2 : fp8 ? 1 : 0;
    bool pair = c->opt.screen_pair != 0;
    int pair_clusters = 0;
    if (pair) {
        pair_clusters = screen_pair_clusters(c, variant);
        pair = pair_clusters > 0;
    }
    CUtensorMap ta, tb;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)c->N};
    const CUtensorMapDataType dt = fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    cuuint64_t strides[1] = {(cuuint64_t)K * (fp8 ? 1 : 2)};
    cuuint32_t box_a[2] = {(cuuint32_t)bke, BM}, box_b[2] = {(cuuint32_t)bke, (cuuint32_t)(pair ? BN / 2 : BN)};
    cuuint32_t es[2] = {1, 1};
    if (g_encode(&ta, dt, 2, const_cast<void *>(A), dims, strides, box_a, es,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
        g_encode(&tb, dt, 2, const_cast<void *>(B), dims, strides, box_b, es,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const size_t smem = pair ? screen_smem<true>() : screen_smem<false>();
    if (cudaError_t e = screen_set_smem(c, variant, pair); e != cudaSuccess) return e;
    ScreenArgs a;
    a.n = (int)c->N;
    a.T = (int)((c->N + SUP - 1) / SUP);
    a.ntiles = (int64_t)a.T * (a.T + 1);  // two units per super-tile
    a.nk = K / bke;
    a.last_mma = (k_valid - (a.nk - 1) * bke) / kchunk;
    a.lambda = thr;
    a.rel_err = rel;
    a.abs_margin = abs_margin;
    a.product_margin = product_margin;
    a.l1 = l1;
    a.r1 = r1;
    a.W = c->W;
    a.skip_stored = skip_stored ? 1 : 0;
    a.out = out;
    a.cap = cap;
    a.count = count;
    a.err = c->cnt;
    a.stall = c->fault_screen_stall ? 1 : 0;
    // a shard of the screen: every nshard-th work item (unit, or in the pair form
    // super-tile), starting at item `shard`
    const int64_t items = pair ? a.ntiles / 2 : a.ntiles;
    a.nshard = use_shard && c->opt.shard_count > 1 ? c->opt.shard_count : 1;
    a.shard = a.nshard > 1 ? c->opt.shard_index : 0;
    a.nlocal = items > a.shard ? (items - a.shard + a.nshard - 1) / a.nshard : 0;
    cudaError_t e;
    if (pair) {
        // persistent: one cluster of two CTAs per pair of SMs
        const unsigned g = 2u * (unsigned)std::max<int64_t>(std::min<int64_t>(a.nlocal, pair_clusters), 1);
        e = variant == 2   ? launch_pair(k_screen<true, true, true>, g, smem, c->stream, ta, tb, a)
            : variant == 1 ? launch_pair(k_screen<true, false, true>, g, smem, c->stream, ta, tb, a)
                           : launch_pair(k_screen<false, false, true>, g, smem, c->stream, ta, tb, a);
    } else {
        const int64_t grid = std::min<int64_t>(a.nlocal, (int64_t)c->num_sms);  // persistent: one CTA per SM
        const unsigned g = (unsigned)std::max<int64_t>(grid, 1);
        if (r1)
            k_screen<true, true, false><<<g, THREADS, smem, c->stream>>>(ta, tb, a);
        else if (fp8)
            k_screen<true, false, false><<<g, THREADS, smem, c->stream>>>(ta, tb, a);
        else
            k_screen<false, false, false><<<g, THREADS, smem, c->stream>>>(ta, tb, a);
        e = cudaGetLastError();
    }
    note_launch();
    if (flop_out) *flop_out = 2.0 * BM * BN * (double)k_valid * (double)(pair ? 2 * a.nlocal : a.nlocal);
    return e;
}

cudaError_t launch_screen(recon_ctx *c, const void *A, const void *B, const float *l1, int32_t *out, int64_t cap,
                          unsigned long long *count, float margin_scale, double *flop_out, bool fp8) {
    return launch_screen_ex(c, A, B, screen_k(c, fp8), (float)c->opt.lambda, l1, margin_scale,
                            c->model == RECON_GAUSSIAN, true, out, cap, count, flop_out, fp8, 0.f,
                            2 * (int)c->Mp, nullptr, true);
}
