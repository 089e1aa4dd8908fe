// Measured FP32 fused multiply-add throughput of the current GPU: the peak the
// FP32 pair kernels are compared with (the vendor figure counts units and the
// maximum clock; this one is what the SMs sustain under the clocks and power
// cap of the moment).
#include <algorithm>

#include "rc_internal.cuh"

namespace {

constexpr int PROBE_THREADS = 256, PROBE_CHAINS = 8, PROBE_UNROLL = 16, PROBE_MAX_BLOCKS = 4096;
__device__ float g_probe_sink[PROBE_MAX_BLOCKS];

// PROBE_CHAINS independent FMA chains per thread, so that every FP32 lane has
// work in every cycle whatever the FMA latency
__global__ void __launch_bounds__(PROBE_THREADS) k_ffma_probe(int iters, float seed) {
    float a[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; k++) a[k] = seed + 1e-7f * (float)threadIdx.x + (float)k;
    const float m = 0.9999999f, b = 1e-7f;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; u++) {
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; k++) a[k] = fmaf(a[k], m, b);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; k++) s += a[k];
    if (s == 1234.5678f) g_probe_sink[blockIdx.x] = s;  // keeps the chains live; never true in practice
}

}  // namespace

extern "C" int rcell_fp32_peak(void *stream, double *tflops) {
    if (!tflops) return RC_EINVAL;
    *tflops = 0.0;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RC_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RC_ECUDA;
    const int blocks = std::min(sms * (2048 / PROBE_THREADS), PROBE_MAX_BLOCKS);
    const int iters = 4096;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return RC_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return RC_ECUDA; }
    k_ffma_probe<<<blocks, PROBE_THREADS, 0, st>>>(iters / 8, 1.0f);  // warm-up (clocks up)
    cudaEventRecord(e0, st);
    k_ffma_probe<<<blocks, PROBE_THREADS, 0, st>>>(iters, 1.0f);
    cudaEventRecord(e1, st);
    float ms = 0.0f;
    const bool ok = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok || cudaGetLastError() != cudaSuccess || ms <= 0.0f) return RC_ECUDA;
    const double fma = (double)blocks * PROBE_THREADS * iters * PROBE_UNROLL * PROBE_CHAINS;
    *tflops = 2.0 * fma / ((double)ms * 1e-3) / 1e12;
    return RC_OK;
}
