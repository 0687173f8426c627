// noalloc.cu -- recon_score_noalloc: pair scoring that performs no device
// allocation at call time.
//
// Who needs it: callers that may not allocate device memory while they run.
// A process that shares the GPU with PyTorch or JAX usually finds most of HBM
// already reserved by that framework's caching allocator, so a cudaMalloc from
// another library can fail or fragment it; serving and real-time loops often
// forbid allocation after start-up; and recon_score's own staging buffers grow
// with cudaMalloc/cudaFree, and cudaFree waits for the whole device.  This entry
// point stages the caller's pairs and results in one fixed array in device
// global memory that the library reserves statically, so a call never
// allocates, whatever P is (up to the limit below).
//
// The array is shared by every call in the process on a given device and keeps
// the contents of the last call: the per-call error and counter words are
// cleared at the start of each call, and calls whose work overlaps on the GPU
// (from several host threads or streams) race on it.
#include <mutex>

#include "common.cuh"

namespace {

constexpr int64_t kMaxPairs = 1 << 16;  // pairs per call
constexpr size_t kWords = 16;            // error / counter words
constexpr size_t kPairBytes = sizeof(int32_t) * 2 * kMaxPairs;
constexpr size_t kOutBytes = sizeof(float) * kMaxPairs;
constexpr size_t kScratchBytes = sizeof(unsigned long long) * kWords + kPairBytes + 2 * kOutBytes;  // 1 MiB + 128 B
static_assert(kWords >= CNT_N, "the scorer's error and counter words must fit in the array");

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the array, one per device.  In host code the array's name
// is only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress while that device is current.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

cudaError_t scratch_on_device(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = (unsigned char *)g_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" recon_status recon_score_noalloc(recon_ctx *c, const int32_t *pairs, int64_t P, float *d_out,
                                            float *w_out) {
    if (!c) return set_err(nullptr, RECON_EINVAL, "null context");
    tl_ctx = c;
    if (c->broken) return set_err(c, RECON_ESTATE, "context unusable after an earlier error: %s", c->err.c_str());
    if (P < 0) return set_err(c, RECON_EINVAL, "P < 0");
    if (P > kMaxPairs)
        return set_err(c, RECON_EINVAL, "recon_score_noalloc takes at most %lld pairs per call (got %lld)",
                       (long long)kMaxPairs, (long long)P);
    if (P == 0) return RECON_OK;
    if (!pairs || !d_out) return set_err(c, RECON_EINVAL, "pairs or d_out is NULL");
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetDevice");
    if (cur != c->device) {
        e = cudaSetDevice(c->device);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    }
    unsigned char *base = nullptr;
    e = scratch_on_device(c->device, &base);
    if (e == cudaSuccess) {
        unsigned long long *words = (unsigned long long *)base;
        int32_t *dp = (int32_t *)(base + sizeof(unsigned long long) * kWords);
        float *dd = (float *)(base + sizeof(unsigned long long) * kWords + kPairBytes);
        float *dw = dd + kMaxPairs;
        unsigned long long flags = 0;
        // the error and counter words must start at zero on every call
        e = cudaMemsetAsync(words, 0, sizeof(unsigned long long) * kWords, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dp, pairs, sizeof(int32_t) * 2 * P, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = launch_check_pairs(dp, P, (int)c->N, words, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&flags, words + CNT_ERR, sizeof flags, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e == cudaSuccess && flags) {
            if (cur != c->device) cudaSetDevice(cur);
            return set_err(c, RECON_EINVAL, "a pair has an id outside [0, N) or i == j");
        }
        if (e == cudaSuccess) {
            if (c->model == RECON_ISING)
                e = launch_ising_score(c->iv(), c->W, c->sp(), dp, P, nullptr, dd, dw, words, c->stream);
            else
                e = launch_gauss_score(c->gv(), c->W, c->sp(), dp, P, nullptr, dd, dw, words, c->stream);
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_out, dd, sizeof(float) * P, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess && w_out)
            e = cudaMemcpyAsync(w_out, dw, sizeof(float) * P, cudaMemcpyDeviceToHost, c->stream);
        // the scorer counts its Newton passes in the array's words: carried over to
        // the context's statistics
        unsigned long long npass = 0;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&npass, words + CNT_NEWTON, sizeof npass, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e == cudaSuccess) {
            c->stats.pair_evals += P;
            c->newton_extra += (int64_t)npass;
        }
    }
    if (cur != c->device) cudaSetDevice(cur);
    if (e != cudaSuccess) return cuda_fail(c, e, "recon_score_noalloc");
    return RECON_OK;
}
