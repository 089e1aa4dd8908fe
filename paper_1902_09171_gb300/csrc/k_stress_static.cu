// Stress reduction that allocates nothing.
//
// Some callers cannot call cudaMalloc at the moment they need the
// time-averaged stress: a host program that reserves the GPU's memory up front
// for its own pool and forbids any later device allocation, or a latency-bound
// loop that must not take the implicit device-wide synchronisation that
// cudaFree (and, when it has to grow the heap, cudaMalloc) performs.
// rcell_stress_reduce_static gives them the stress reduction of rcell_stress
// (rotation to the FE frame, mean, blocking standard error, first
// Piola-Kirchhoff stress) with its only scratch -- the rotated sample series --
// in a fixed-size array that lives in this library's device image.  The caller
// passes inputs and outputs; the call allocates nothing and calls no
// allocating library routine.
//
// Limits and sharing:
//   * The scratch holds RC_STATIC_SCRATCH_SAMPLES six-component samples
//     (3 MiB of FP64); n_cells * n_avg above that is rejected with RC_EINVAL
//     before any GPU work.  Every GPU that loads the library holds the array
//     until the process exits.
//   * All calls share the one array, which keeps the last call's contents.
//     Each call writes every scratch entry it reads before reading it, so
//     leftovers of an earlier call never matter, but two calls whose kernels
//     overlap on the GPU (different streams, no ordering between them) race on
//     the array and give wrong results.
//   * The first call on a device looks up the array's device address with
//     cudaGetSymbolAddress while that device is current; make that first call
//     before any stream capture.
#include <mutex>

#include "rc_internal.cuh"

#define RC_STATIC_SCRATCH_SAMPLES 65536
#define RC_STATIC_MAX_DEVICES 64

// the scratch: one FE-frame stress sample (6 doubles) per entry
static __device__ __align__(256) double g_rot_static[RC_STATIC_SCRATCH_SAMPLES * 6];

namespace {

std::mutex g_mtx;
double *g_rot_ptr[RC_STATIC_MAX_DEVICES] = {nullptr};

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

// One CTA per cell: rotate every MD-frame sample to the FE frame into the
// scratch, then warp k < 6 forms the mean and the blocking standard error of
// component k, then thread 0 forms P = J sigma F^{-T}.
constexpr int ST_THREADS = 256;
__global__ void __launch_bounds__(ST_THREADS) k_stress_static(const double *__restrict__ series, int n_avg,
                                                               const double *__restrict__ Qall,
                                                               const double *__restrict__ Fall, double *rot_all,
                                                               double *sig, double *se_out, double *P) {
    const int c = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ double s_mean[6];
    const double *Q = Qall + 9 * c;
    const double *ser = series + (size_t)c * n_avg * 6;
    double *rot = rot_all + (size_t)c * n_avg * 6;
    const int vi[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    for (int t = tid; t < n_avg; t += ST_THREADS) {
        double S[9];
        for (int k = 0; k < 6; k++) {
            const double s = ser[(size_t)t * 6 + k];
            S[3 * vi[k][0] + vi[k][1]] = s;
            S[3 * vi[k][1] + vi[k][0]] = s;
        }
        for (int k = 0; k < 6; k++) {
            const int a = vi[k][0], b = vi[k][1];
            double r = 0.0;
            for (int u = 0; u < 3; u++)
                for (int v = 0; v < 3; v++) r += Q[3 * a + u] * S[3 * u + v] * Q[3 * b + v];
            rot[(size_t)t * 6 + k] = r;
        }
    }
    __syncthreads();
    if (warp < 6) {
        const int k = warp;
        double sum = 0.0;
        for (int t = lane; t < n_avg; t += 32) sum += rot[(size_t)t * 6 + k];
        const double mean = wsum(sum) / n_avg;
        double best = 0.0;
        for (int lvl = 0;; lvl++) {
            const int bs = 1 << lvl, nk = n_avg / bs;
            if (nk < 2 || (lvl > 0 && nk < 16)) break;
            double mb = 0.0;
            for (int b = lane; b < nk; b += 32) {
                double m = 0.0;
                for (int t = 0; t < bs; t++) m += rot[(size_t)(b * bs + t) * 6 + k];
                mb += m / bs;
            }
            mb = wsum(mb) / nk;
            double v = 0.0;
            for (int b = lane; b < nk; b += 32) {
                double m = 0.0;
                for (int t = 0; t < bs; t++) m += rot[(size_t)(b * bs + t) * 6 + k];
                m /= bs;
                v += (m - mb) * (m - mb);
            }
            v = wsum(v);
            const double e = sqrt(v / ((double)nk * (nk - 1)));
            if (e > best) best = e;
        }
        if (lane == 0) {
            sig[6 * c + k] = mean;
            if (se_out) se_out[6 * c + k] = best;
            s_mean[k] = mean;
        }
    }
    __syncthreads();
    if (tid == 0 && P) {
        const double *F = Fall + 9 * c;
        const double J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                         F[2] * (F[3] * F[7] - F[4] * F[6]);
        double Fi[9];
        Fi[0] = (F[4] * F[8] - F[5] * F[7]) / J;
        Fi[1] = (F[2] * F[7] - F[1] * F[8]) / J;
        Fi[2] = (F[1] * F[5] - F[2] * F[4]) / J;
        Fi[3] = (F[5] * F[6] - F[3] * F[8]) / J;
        Fi[4] = (F[0] * F[8] - F[2] * F[6]) / J;
        Fi[5] = (F[2] * F[3] - F[0] * F[5]) / J;
        Fi[6] = (F[3] * F[7] - F[4] * F[6]) / J;
        Fi[7] = (F[1] * F[6] - F[0] * F[7]) / J;
        Fi[8] = (F[0] * F[4] - F[1] * F[3]) / J;
        const double S[9] = {s_mean[0], s_mean[3], s_mean[4], s_mean[3], s_mean[1], s_mean[5],
                             s_mean[4], s_mean[5], s_mean[2]};
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double s = 0.0;
                for (int l = 0; l < 3; l++) s += S[3 * i + l] * Fi[3 * j + l];
                P[9 * c + 3 * i + j] = J * s;
            }
    }
}

}  // namespace

extern "C" int rcell_stress_reduce_static(const double *series, int n_cells, int n_avg, const double *Q,
                                          const double *F, double *sigma, double *sigma_stderr, double *P,
                                          void *stream) {
    if (!series || !Q || !F || !sigma || n_cells <= 0 || n_avg <= 0) return RC_EINVAL;
    if ((long long)n_cells * n_avg > RC_STATIC_SCRATCH_SAMPLES) return RC_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RC_ECUDA;
    if (dev < 0 || dev >= RC_STATIC_MAX_DEVICES) return RC_EINVAL;
    double *rot = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mtx);
        if (!g_rot_ptr[dev]) {
            // set-up, once per device with that device current: the device
            // address of the scratch array (its host-side name is not one)
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_rot_static) != cudaSuccess || !ptr) return RC_ECUDA;
            g_rot_ptr[dev] = static_cast<double *>(ptr);
        }
        rot = g_rot_ptr[dev];
    }
    // the launch's own return code: an error left behind by an unrelated
    // earlier call is neither reported nor cleared here
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)n_cells);
    cfg.blockDim = dim3(ST_THREADS);
    cfg.stream = (cudaStream_t)stream;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_stress_static, series, n_avg, Q, F, rot, sigma, sigma_stderr, P);
    return e == cudaSuccess ? RC_OK : RC_ECUDA;
}
