// peaks.cu -- the device ceilings that the kernels' rooflines are stated
// against, measured on the device itself: FP32 and FP64 fused multiply-add
// rates, the special-function unit's reciprocal, exp2, log2 and tanh rates, and
// the read bandwidth from an L2-resident buffer into the SMs.  The paper has no
// counterpart: this is measurement support for the pair scorer (FP32 + MUFU
// arithmetic on rows that sit in L2) and the update kernels.
//
// Each kernel runs a fixed amount of independent work per thread (eight
// independent chains, so that issue rather than latency limits it) on a grid
// of several CTAs per SM, timed with CUDA events on a private stream after one
// untimed launch.  Nothing here changes a device setting.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"

namespace {

constexpr int CHAINS = 8;

__global__ void __launch_bounds__(256) k_peak_ffma(int iters, float b, float c, float *out) {
    float a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = (float)(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[k]) : "f"(b), "f"(c));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    if (s == 1234.5f) out[0] = s;  // keeps the chains live
}

__global__ void __launch_bounds__(256) k_peak_dfma(int iters, double b, double c, double *out) {
    double a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = (double)(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(a[k]) : "d"(b), "d"(c));
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    if (s == 1234.5) out[0] = s;
}

// op 0: rcp.approx   x <- 1 / (x + 1)       (one FP32 add per call besides the MUFU op)
// op 1: ex2.approx   x <- 2^(-x)            (bounded: the fixed point is about 0.64)
// op 2: lg2.approx   x <- log2(|x| + 1.5)   (one FP32 add per call besides the MUFU op)
// op 3: tanh.approx  x <- tanh(x)
template <int OP>
__global__ void __launch_bounds__(256) k_peak_mufu(int iters, float *out) {
    float a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = 0.5f + 0.01f * (float)((threadIdx.x + k) & 31);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) {
            if constexpr (OP == 0)
                asm volatile("{.reg .f32 t; add.f32 t, %0, 0f3F800000; rcp.approx.ftz.f32 %0, t;}" : "+f"(a[k]));
            if constexpr (OP == 1) asm volatile("{.reg .f32 t; neg.f32 t, %0; ex2.approx.ftz.f32 %0, t;}" : "+f"(a[k]));
            if constexpr (OP == 2)
                asm volatile("{.reg .f32 t; abs.f32 t, %0; add.f32 t, t, 0f3FC00000; lg2.approx.ftz.f32 %0, t;}"
                             : "+f"(a[k]));
            if constexpr (OP == 3) asm volatile("tanh.approx.f32 %0, %0;" : "+f"(a[k]));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    if (s == 1234.5f) out[0] = s;
}

// the grid reads the whole buffer `passes` times (16-byte loads cached in L2
// only); after the untimed launch the buffer is L2-resident
__global__ void __launch_bounds__(256) k_peak_l2(const float4 *buf, int64_t n4, int passes, float *out) {
    float acc = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int p = 0; p < passes; ++p)
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n4; e += stride) {
            const float4 v = __ldcg(buf + e);
            acc += (v.x + v.y) + (v.z + v.w);
        }
    if (acc == 1234.5f) out[0] = acc;
}

}  // namespace

extern "C" recon_status recon_device_peaks(int32_t device, recon_peaks *out) {
    if (!out) return RECON_EINVAL;
    std::memset(out, 0, sizeof *out);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return RECON_ECUDA;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return RECON_ECUDA;
    int clk_khz = 0;
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, device);
    out->sm_count = prop.multiProcessorCount;
    out->sm_clock_mhz = clk_khz / 1000.0;
    out->l2_bytes = prop.l2CacheSize;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float *sink = nullptr;
    float4 *l2buf = nullptr;
    recon_status st = RECON_OK;
    const int64_t l2n = (int64_t)prop.l2CacheSize / 4 / (int64_t)sizeof(float4);  // a quarter of L2
    do {
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
            cudaEventCreate(&e1) != cudaSuccess || cudaMalloc(&sink, 64) != cudaSuccess ||
            cudaMalloc(&l2buf, (size_t)l2n * sizeof(float4)) != cudaSuccess) {
            st = RECON_ECUDA;
            break;
        }
        cudaMemsetAsync(l2buf, 0, (size_t)l2n * sizeof(float4), s);
        const unsigned grid = (unsigned)(prop.multiProcessorCount * 8);
        const double threads = (double)grid * 256.0;
        // one untimed launch, then one timed; returns milliseconds
        auto timed = [&](auto launch) -> float {
            launch();
            cudaEventRecord(e0, s);
            launch();
            cudaEventRecord(e1, s);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return -1.f;
            return ms;
        };
        const int it32 = 4096, it64 = 256, itm = 1024;
        float ms = timed([&] { k_peak_ffma<<<grid, 256, 0, s>>>(it32, 1.0000001f, 1e-7f, sink); });
        out->fp32_tflops = 2.0 * threads * it32 * CHAINS / (ms * 1e-3) / 1e12;
        ms = timed([&] { k_peak_dfma<<<grid, 256, 0, s>>>(it64, 1.0000001, 1e-7, (double *)sink); });
        out->fp64_tflops = 2.0 * threads * it64 * CHAINS / (ms * 1e-3) / 1e12;
        ms = timed([&] { k_peak_mufu<0><<<grid, 256, 0, s>>>(itm, sink); });
        out->mufu_rcp_gops = threads * itm * CHAINS / (ms * 1e-3) / 1e9;
        ms = timed([&] { k_peak_mufu<1><<<grid, 256, 0, s>>>(itm, sink); });
        out->mufu_ex2_gops = threads * itm * CHAINS / (ms * 1e-3) / 1e9;
        ms = timed([&] { k_peak_mufu<2><<<grid, 256, 0, s>>>(itm, sink); });
        out->mufu_lg2_gops = threads * itm * CHAINS / (ms * 1e-3) / 1e9;
        ms = timed([&] { k_peak_mufu<3><<<grid, 256, 0, s>>>(itm, sink); });
        out->mufu_tanh_gops = threads * itm * CHAINS / (ms * 1e-3) / 1e9;
        const int passes = 64;
        ms = timed([&] { k_peak_l2<<<grid, 256, 0, s>>>(l2buf, l2n, passes, sink); });
        out->l2_read_gbs = (double)passes * (double)l2n * sizeof(float4) / (ms * 1e-3) / 1e9;
        out->l2_buffer_bytes = (double)l2n * sizeof(float4);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) st = RECON_ECUDA;
    } while (false);
    if (l2buf) cudaFree(l2buf);
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    return st;
}
