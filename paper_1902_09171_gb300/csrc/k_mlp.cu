// Recurrent-MLP stress surrogate on tensor cores: BF16 operands, FP32
// accumulation, fused epilogues, BPTT and AdamW.  The default engine runs on
// tcgen05 (5th-generation tensor cores, accumulators in tensor memory): the
// whole forward and the whole BPTT data-gradient chain each in one
// warp-specialised kernel (k_forward_ws, k_backward_ws), the weight and bias
// gradients in k_wgrad_tc05, all members side by side.  The alternative
// engines run one GEMM per layer and step, on tcgen05 (k_gemm_tc05) or on
// warp-level mma.sync m16n8k16 (k_gemm).
//
// mma.sync GEMM: C[M x N] = op(A)[M x K] * B[K x N], op(A) = A (row-major, lda) or A^T
// (A stored K x M).  CTA tile 64 x 64 x 32, four warps of 32 x 32; operand
// tiles staged in shared memory (A as [m][k], B as [n][k], k contiguous, so
// every fragment register is one aligned 32-bit shared load).  Epilogues fuse
// bias + GELU (forward), the head (stress output + tanh state written straight
// into the next step's input row), GELU' (backward) and split-K FP32 weight
// gradient accumulation.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/surrogate.h"
#include "rc_internal.cuh"

namespace {

constexpr int K0 = 144, WID = 256, N4 = 144, NIN = SUR_N_IN, NH = SUR_N_H, NOUT = SUR_N_OUT;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + K0 * WID, OFF_W2 = OFF_B1 + WID, OFF_B2 = OFF_W2 + WID * WID,
              OFF_W3 = OFF_B2 + WID, OFF_B3 = OFF_W3 + WID * WID, OFF_W4 = OFF_B3 + WID, OFF_B4 = OFF_W4 + WID * N4,
              NPAR = OFF_B4 + N4;
static_assert(NPAR == SUR_N_PARAMS, "parameter layout");

constexpr int BM = 64, BN = 64, BK = 32, PADK = 8, GEMM_THREADS = 128;

enum { EPI_GELU = 0, EPI_HEAD = 1, EPI_DGELU = 2, EPI_F32 = 3, EPI_WGRAD = 4 };

struct Epi {
    const float *bias;       // GELU, HEAD
    __nv_bfloat16 *y_out;    // GELU: pre-activation
    __nv_bfloat16 *a_out;    // GELU: activation; DGELU: dy out
    int ld_out;
    const __nv_bfloat16 *y_in;  // DGELU: pre-activation
    int ld_in;
    float *s_out;            // HEAD: stress (row stride s_ld), F32/WGRAD: C
    int s_ld;
    __nv_bfloat16 *h_next;   // HEAD: next step's input row block (columns NIN..NIN+NH), may be null
    float *h_f32;            // HEAD: FP32 copy of h (ld NH), may be null
    const float *s_mul;      // HEAD: per-component stress scale (null: network units)
    long ms_in, ms_out;      // member strides (elements) of y_in and of the outputs, for member-batched launches
};

// the epilogue pointers of member z of a member-batched launch
__device__ __forceinline__ void epi_member(Epi &e, int z) {
    if (z == 0) return;
    if (e.y_in) e.y_in += z * e.ms_in;
    if (e.y_out) e.y_out += z * e.ms_out;
    if (e.a_out) e.a_out += z * e.ms_out;
    if (e.s_out) e.s_out += z * e.ms_out;
}

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.3989422804014327f * expf(-0.5f * x * x);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int EPI>
__device__ __forceinline__ void epilogue(const Epi &e, int m, int n, int M, int N, float acc) {
    if (m >= M || n >= N) return;
    if (EPI == EPI_GELU) {
        const float y = acc + e.bias[n];
        e.y_out[(size_t)m * e.ld_out + n] = __float2bfloat16(y);
        e.a_out[(size_t)m * e.ld_out + n] = __float2bfloat16(gelu_f(y));
    } else if (EPI == EPI_HEAD) {
        const float o = acc + e.bias[n];
        if (n < NOUT) {
            e.s_out[(size_t)m * e.s_ld + n] = e.s_mul ? o * e.s_mul[n] : o;
        } else if (n < NOUT + NH) {
            const float h = tanhf(o);
            if (e.h_next) e.h_next[(size_t)m * K0 + NIN + (n - NOUT)] = __float2bfloat16(h);
            if (e.h_f32) e.h_f32[(size_t)m * NH + (n - NOUT)] = h;
        }
    } else if (EPI == EPI_DGELU) {
        const float y = __bfloat162float(e.y_in[(size_t)m * e.ld_in + n]);
        e.a_out[(size_t)m * e.ld_out + n] = __float2bfloat16(acc * gelu_d(y));
    } else if (EPI == EPI_F32) {
        e.s_out[(size_t)m * e.s_ld + n] = acc;
    } else {  // EPI_WGRAD: split-K partial sums
        atomicAdd(&e.s_out[(size_t)m * e.s_ld + n], acc);
    }
}

// Sixteen consecutive columns n..n+15 of row m (n a multiple of 16, N a
// multiple of 16) with 16-byte loads and stores; the head epilogue, whose
// outputs are not 16-byte aligned, goes element by element.
template <int EPI>
__device__ __forceinline__ void epilogue16(const Epi &e, int m, int n, int M, int N, const float (&acc)[16]) {
    if (m >= M || n >= N) return;
    if (EPI == EPI_GELU) {
        __align__(16) __nv_bfloat16 y[16], a[16];
#pragma unroll
        for (int j = 0; j < 16; j++) {
            const float v = acc[j] + e.bias[n + j];
            y[j] = __float2bfloat16(v);
            a[j] = __float2bfloat16(gelu_f(v));
        }
        uint4 *py = reinterpret_cast<uint4 *>(e.y_out + (size_t)m * e.ld_out + n);
        uint4 *pa = reinterpret_cast<uint4 *>(e.a_out + (size_t)m * e.ld_out + n);
        py[0] = reinterpret_cast<const uint4 *>(y)[0];
        py[1] = reinterpret_cast<const uint4 *>(y)[1];
        pa[0] = reinterpret_cast<const uint4 *>(a)[0];
        pa[1] = reinterpret_cast<const uint4 *>(a)[1];
    } else if (EPI == EPI_DGELU) {
        __align__(16) __nv_bfloat16 y[16], d[16];
        const uint4 *py = reinterpret_cast<const uint4 *>(e.y_in + (size_t)m * e.ld_in + n);
        reinterpret_cast<uint4 *>(y)[0] = py[0];
        reinterpret_cast<uint4 *>(y)[1] = py[1];
#pragma unroll
        for (int j = 0; j < 16; j++) d[j] = __float2bfloat16(acc[j] * gelu_d(__bfloat162float(y[j])));
        uint4 *pd = reinterpret_cast<uint4 *>(e.a_out + (size_t)m * e.ld_out + n);
        pd[0] = reinterpret_cast<const uint4 *>(d)[0];
        pd[1] = reinterpret_cast<const uint4 *>(d)[1];
    } else if (EPI == EPI_F32) {
        float4 *p = reinterpret_cast<float4 *>(e.s_out + (size_t)m * e.s_ld + n);
#pragma unroll
        for (int j = 0; j < 4; j++) p[j] = make_float4(acc[4 * j], acc[4 * j + 1], acc[4 * j + 2], acc[4 * j + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < 16; j++) epilogue<EPI>(e, m, n + j, M, N, acc[j]);
    }
}

template <int EPI, bool TRANS_A>
__global__ void __launch_bounds__(GEMM_THREADS) k_gemm(const __nv_bfloat16 *__restrict__ A, int lda,
                                                       const __nv_bfloat16 *__restrict__ B, int ldb, int M, int N,
                                                       int K, int k_chunk, Epi e, int nz, long a_ms, long b_ms) {
    __shared__ __align__(16) __nv_bfloat16 As[BM][BK + PADK];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][BK + PADK];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1, g = lane >> 2, q = lane & 3;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int mb = blockIdx.z / nz;  // member of a member-batched launch, then the split-K part
    A += mb * a_ms;
    B += mb * b_ms;
    epi_member(e, mb);
    const int kb = (blockIdx.z - mb * nz) * k_chunk, ke = min(K, kb + k_chunk);
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
            for (int r = 0; r < 4; r++) acc[i][j][r] = 0.f;
    const uint4 zero4 = make_uint4(0, 0, 0, 0);
    for (int k0 = kb; k0 < ke; k0 += BK) {
        // ---- stage op(A) tile [BM][BK] ----
#pragma unroll
        for (int it = 0; it < 2; it++) {
            const int idx = tid + it * GEMM_THREADS;  // 256 chunks of 8 elements
            if (!TRANS_A) {
                const int r = idx >> 2, kc = (idx & 3) * 8;
                uint4 v = zero4;
                if (m0 + r < M && k0 + kc < ke) v = *reinterpret_cast<const uint4 *>(A + (size_t)(m0 + r) * lda + k0 + kc);
                *reinterpret_cast<uint4 *>(&As[r][kc]) = v;
            } else {
                const int kr = idx >> 3, mc = (idx & 7) * 8;
                uint4 v = zero4;
                if (k0 + kr < ke && m0 + mc < M) v = *reinterpret_cast<const uint4 *>(A + (size_t)(k0 + kr) * lda + m0 + mc);
                const __nv_bfloat16 *pv = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
                for (int i = 0; i < 8; i++) As[mc + i][kr] = pv[i];
            }
        }
        // ---- stage B tile as [BN][BK] ----
#pragma unroll
        for (int it = 0; it < 2; it++) {
            const int idx = tid + it * GEMM_THREADS;
            const int kr = idx >> 3, nc = (idx & 7) * 8;
            uint4 v = zero4;
            if (k0 + kr < ke && n0 + nc < N) v = *reinterpret_cast<const uint4 *>(B + (size_t)(k0 + kr) * ldb + n0 + nc);
            const __nv_bfloat16 *pv = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
            for (int i = 0; i < 8; i++) Bs[nc + i][kr] = pv[i];
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            unsigned a[2][4], b[4][2];
#pragma unroll
            for (int mi = 0; mi < 2; mi++) {
                const int r = wm * 32 + mi * 16 + g;
                a[mi][0] = *reinterpret_cast<const unsigned *>(&As[r][kk + 2 * q]);
                a[mi][1] = *reinterpret_cast<const unsigned *>(&As[r + 8][kk + 2 * q]);
                a[mi][2] = *reinterpret_cast<const unsigned *>(&As[r][kk + 8 + 2 * q]);
                a[mi][3] = *reinterpret_cast<const unsigned *>(&As[r + 8][kk + 8 + 2 * q]);
            }
#pragma unroll
            for (int ni = 0; ni < 4; ni++) {
                const int c = wn * 32 + ni * 8 + g;
                b[ni][0] = *reinterpret_cast<const unsigned *>(&Bs[c][kk + 2 * q]);
                b[ni][1] = *reinterpret_cast<const unsigned *>(&Bs[c][kk + 8 + 2 * q]);
            }
#pragma unroll
            for (int mi = 0; mi < 2; mi++)
#pragma unroll
                for (int ni = 0; ni < 4; ni++) mma_bf16(acc[mi][ni], a[mi], b[ni]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int mi = 0; mi < 2; mi++)
#pragma unroll
        for (int ni = 0; ni < 4; ni++) {
            const int m = m0 + wm * 32 + mi * 16 + g, n = n0 + wn * 32 + ni * 8 + 2 * q;
            epilogue<EPI>(e, m, n, M, N, acc[mi][ni][0]);
            epilogue<EPI>(e, m, n + 1, M, N, acc[mi][ni][1]);
            epilogue<EPI>(e, m + 8, n, M, N, acc[mi][ni][2]);
            epilogue<EPI>(e, m + 8, n + 1, M, N, acc[mi][ni][3]);
        }
}

// nb members at once (operand strides a_ms, b_ms; epilogue strides in e)
template <int EPI, bool TRANS_A>
void gemm(cudaStream_t s, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, int M, int N, int K,
          const Epi &e, int split_k = 1, int nb = 1, long a_ms = 0, long b_ms = 0) {
    int chunk = (K + split_k - 1) / split_k;
    chunk = (chunk + BK - 1) / BK * BK;
    const int nz = (K + chunk - 1) / chunk;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, nz * nb);
    k_gemm<EPI, TRANS_A><<<grid, GEMM_THREADS, 0, s>>>(A, lda, B, ldb, M, N, K, chunk, e, nz, a_ms, b_ms);
}

// ---------------------------------------------------------------------------
// The same GEMM on the 5th-generation tensor cores (tcgen05): C[M x N] =
// A[M x K] * Bk[N x K]^T with both operands K-major.  One CTA computes a
// 128 x 256 tile (every output column of this network: the A rows are read
// once) with the whole K (<= 256) resident in shared memory:
//   * operands are copied (cp.async, 16 bytes per copy) into shared memory in
//     the K-major "core matrix" layout (8 rows x 16 bytes per core matrix, no
//     swizzle): core (r/8, k/8) at byte (k/8 * rows/8 + r/8) * 128, row r%8 at
//     +16 (r%8);
//   * one elected thread issues K/16 tcgen05.mma (kind::f16, BF16 inputs,
//     FP32 accumulator in tensor memory) and a tcgen05.commit onto an mbarrier;
//   * every warp waits on the mbarrier (bounded), reads its 32 accumulator rows
//     (its lane quarter) of one 64-column part with tcgen05.ld and runs the
//     fused epilogue sixteen columns at a time with 16-byte stores (sixteen
//     warps); tensor memory is freed on every path.
// ---------------------------------------------------------------------------
constexpr int TC_M = 128, TC_N = 256, TC_THREADS = 512, TC_SPIN = 1 << 22;

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of the 5th-generation tensor cores; no swizzle
    return d;
}

template <int EPI>
__global__ void __launch_bounds__(TC_THREADS) k_gemm_tc05(const __nv_bfloat16 *__restrict__ A, int lda,
                                                          const __nv_bfloat16 *__restrict__ Bk, int ldb, int M, int N,
                                                          int K, Epi e, int *err, long a_ms, long b_ms) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) unsigned long long s_bar;
    __shared__ unsigned s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TC_M, n0 = blockIdx.x * TC_N;
    A += blockIdx.z * a_ms;  // member of a member-batched launch
    Bk += blockIdx.z * b_ms;
    epi_member(e, blockIdx.z);
    const int KC = K >> 3;  // 16-byte chunks along K
    unsigned char *sA = tc_smem, *sB = tc_smem + (size_t)TC_M * K * 2;
    // tensor memory: 256 columns x 128 lanes of FP32 for the 128 x 256 accumulator
    if (warp == 0) {
        const unsigned dst = (unsigned)__cvta_generic_to_shared(&s_tmem);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(TC_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // operands into the core-matrix layout with asynchronous 16-byte copies (all
    // of a thread's copies in flight at once; rows past the matrix are zero-filled)
    for (int idx = tid; idx < TC_M * KC; idx += TC_THREADS) {
        const int r = idx / KC, kc = idx - r * KC;
        const bool in = m0 + r < M;
        const __nv_bfloat16 *src = A + (size_t)(in ? m0 + r : 0) * lda + kc * 8;
        const unsigned dst =
            (unsigned)__cvta_generic_to_shared(sA + ((size_t)kc * (TC_M / 8) + (r >> 3)) * 128 + (r & 7) * 16);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(in ? 16 : 0)
                     : "memory");
    }
    for (int idx = tid; idx < TC_N * KC; idx += TC_THREADS) {
        const int r = idx / KC, kc = idx - r * KC;
        const bool in = n0 + r < N;
        const __nv_bfloat16 *src = Bk + (size_t)(in ? n0 + r : 0) * ldb + kc * 8;
        const unsigned dst =
            (unsigned)__cvta_generic_to_shared(sB + ((size_t)kc * (TC_N / 8) + (r >> 3)) * 128 + (r & 7) * 16);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(in ? 16 : 0)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const unsigned bar = (unsigned)__cvta_generic_to_shared(&s_bar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = s_tmem;
    if (tid == 0) {
        // instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, N/8, M/16
        const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(TC_N >> 3) << 17) |
                               ((unsigned)(TC_M >> 4) << 24);
        const unsigned a0 = (unsigned)__cvta_generic_to_shared(sA), b0 = (unsigned)__cvta_generic_to_shared(sB);
        const unsigned lboA = (TC_M / 8) * 128, lboB = (TC_N / 8) * 128;
        for (int kk = 0; kk < (K >> 4); kk++) {
            const uint64_t ad = tc_desc(a0 + kk * 2 * lboA, lboA, 128);
            const uint64_t bd = tc_desc(b0 + kk * 2 * lboB, lboB, 128);
            const unsigned acc = kk > 0;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                     : "memory");
    }
    unsigned done = 0;
    for (int it = 0; it < TC_SPIN && !done; it++)
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar)
            : "memory");
    const int ok = __syncthreads_and(done);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        // warp w: accumulator rows 32 (w % 4) .. (its lane quarter), columns 64 (w / 4) ..
        const int quarter = warp & 3, part = warp >> 2;
        const int row = m0 + quarter * 32 + lane;
#pragma unroll
        for (int c0 = part * 64; c0 < part * 64 + 64; c0 += 16) {
            if (n0 + c0 >= N) break;
            unsigned r[16];
            const unsigned taddr = tmem + ((unsigned)(quarter * 32) << 16) + (unsigned)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];\n"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; j++) v[j] = __uint_as_float(r[j]);
            epilogue16<EPI>(e, row, n0 + c0, M, N, v);
        }
    } else if (tid == 0) {
        atomicExch(err, RC_ETIMEOUT);
        // let the tensor-core work in flight finish before its memory is released
        for (int it = 0; it < TC_SPIN && !done; it++)
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(bar)
                : "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N) : "memory");
    }
}

// C = A[M x K] * Bk[N x K]^T on tcgen05 (K a multiple of 16, K <= 256), for nb
// members at once (operand strides a_ms, b_ms; epilogue strides in e)
template <int EPI>
void gemm_tc05(cudaStream_t s, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *Bk, int ldb, int M, int N, int K,
               const Epi &e, int *err, int nb = 1, long a_ms = 0, long b_ms = 0) {
    dim3 grid((N + TC_N - 1) / TC_N, (M + TC_M - 1) / TC_M, nb);
    const size_t smem = (size_t)(TC_M + TC_N) * K * 2;
    k_gemm_tc05<EPI><<<grid, TC_THREADS, smem, s>>>(A, lda, Bk, ldb, M, N, K, e, err, a_ms, b_ms);
}

void prepare_tc05() {
    const int bytes = (TC_M + TC_N) * 256 * 2;
    cudaFuncSetAttribute(k_gemm_tc05<EPI_GELU>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(k_gemm_tc05<EPI_HEAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(k_gemm_tc05<EPI_DGELU>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(k_gemm_tc05<EPI_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// ---------------------------------------------------------------------------
// The whole recurrent forward in one kernel (tcgen05).  A CTA owns 128 rows of
// the batch (one member: blockIdx.y) and walks all T steps: per step the four
// layers run back to back on the tensor cores, with the activations kept in
// shared memory (BF16, K-major core-matrix layout) and the layer accumulators
// (128 x 256 FP32) in tensor memory, two of them (512 columns), so that a
// layer's MMAs can write one while the epilogue still reads the other.  The
// roles are split between warps: one producer thread streams the weights
// through four shared buffers, one 64-column K slice of a layer (all its output
// rows) per buffer, with bulk copies (cp.async.bulk, one per chunk, completing
// on a per-buffer mbarrier; the weights are pre-arranged per member by
// k_pack_weights so that each chunk is one contiguous block in the buffer's
// layout), and issues the MMAs slice by slice; sixteen epilogue warps (warp w:
// accumulator rows 32 (w % 4).., columns 16 (w / 4).. of every slice) wait for
// a layer's accumulator and run its epilogue (bias + GELU into the next
// operand, slice after slice; the head writes the stress and the new state
// h = tanh(.) straight into the next step's input rows).  The MMAs of slice s
// of the next layer start as soon as all warps have written slice s of its
// operand, under the rest of the epilogue.  The two sides meet only at
// mbarriers, all waits bounded:
//   full[b]  : chunk in buffer b has landed          (bulk copy -> producer)
//   empty[b] : the MMAs reading buffer b are done     (tcgen05.commit -> producer)
//   acc      : a layer's accumulator is complete      (tcgen05.commit -> epilogue)
//   slice[s] : the epilogue warps have written slice s of a hidden layer's
//              output (16 warp arrivals -> producer)
//   epi      : the epilogue warps have written the next step's input rows
//              (16 warp arrivals -> producer, and -> the epilogue warps
//              before they copy the rows to the tape)
// With a tape (training) every step's z, y and a rows also go to global memory
// for the backward pass, in the layout the layer-wise kernels use.
// ---------------------------------------------------------------------------
constexpr int FT_PARTS = 4, FT_M = 128, FT_MAXK = 8;
// The input rows z (128 x 144) and the activations (128 x 256) share one
// buffer: z is dead once layer 1's MMAs have read it, and the head writes the
// next step's state after the last layer's MMAs have read the activations.
constexpr int FT_NBUF = 4;   // weight buffers
constexpr int FT_KS = 64;    // K columns of a weight chunk: one 64-column slice of the layer's operand
constexpr int FT_SA = FT_M * WID * 2, FT_SW = WID * FT_KS * 2;
constexpr int FT_SMEM = FT_SA + FT_NBUF * FT_SW;
constexpr int FT_CHUNKS = 3 + 4 + 4 + 4;  // weight chunks per step: K slices of the four layers (K = 144, 256, 256, 256)
constexpr int FT_TMEM_COLS = 2 * WID;     // two accumulators: layer l uses columns (l % 2) * 256 ..
static_assert(FT_KS * 4 == WID && FT_KS * 2 < K0 && K0 <= FT_KS * 3, "slices per layer: 3 (K0) or 4 (WID)");

struct FusedArgs {
    const float *U;      // (B, T, NIN) raw features (row b, step t at (b * T + t) * NIN)
    int B, T;
    const float *u_inv;  // NIN feature scales
    const float *s_mul;  // NOUT output scales, or null (network units)
    float *S;            // stress: member k, row b, step t at S + k * s_mstride + b * s_ld + t * NOUT
    long s_mstride;
    int s_ld;
    float *h;            // FP32 state (member k, row b at h + k * h_mstride + b * NH): read at step 0 and
    long h_mstride;      // overwritten with the final state; null: zero initial state, not written
    __nv_bfloat16 *tZ, *tY[3], *tA[3];  // tape of the launch's first member, or null
    long tz_ms, ty_ms;                   // member strides (elements) of tZ and of tY / tA
    const float *theta[FT_MAXK];
    const unsigned char *Wp[FT_MAXK];  // packed weight chunks (k_pack_weights)
    int *err;
};

// byte offset of element (r, k) in a K-major core-matrix tile with `rows` rows
__device__ __forceinline__ unsigned cm_off(int r, int k, int rows) {
    return (unsigned)((((k >> 3) * (rows >> 3) + (r >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ unsigned short bf16_bits(float v) {
    const __nv_bfloat16 b = __float2bfloat16(v);
    return *reinterpret_cast<const unsigned short *>(&b);
}

// two floats to a BF16 pair (round to nearest even), low half = first
__device__ __forceinline__ unsigned bf16x2_bits(float lo, float hi) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned *>(&p);
}

// 32-byte global store / read-only load of 16 BF16 values (one whole sector per
// lane); the address must be 32-byte aligned
__device__ __forceinline__ void st_v8(void *p, const uint4 &lo, const uint4 &hi) {
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(lo.x), "r"(lo.y),
                 "r"(lo.z), "r"(lo.w), "r"(hi.x), "r"(hi.y), "r"(hi.z), "r"(hi.w)
                 : "memory");
}
__device__ __forceinline__ void ld_v8(const void *p, uint4 &lo, uint4 &hi) {
    asm volatile("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(lo.x), "=r"(lo.y), "=r"(lo.z), "=r"(lo.w), "=r"(hi.x), "=r"(hi.y), "=r"(hi.z), "=r"(hi.w)
                 : "l"(p));
}

// GELU in the fused kernels: the tanh approximation of Hendrycks & Gimpel,
// "Gaussian Error Linear Units" (2016), x/2 (1 + tanh(u)) with
// u = sqrt(2/pi) (x + 0.044715 x^3), evaluated as x s with the logistic form
// s = 1 / (1 + 2^(-2 u log2 e)) of the same function (one exponential and one
// reciprocal on the special-function unit, no cancellation in 1 + tanh for
// large negative x).  Its largest deviation from x/2 (1 + erf(x / sqrt 2)) is
// 4.7e-4 (at x = 2.7, a sixteenth of the BF16 rounding of the stored
// activation there); the derivative's is 8.7e-4.
constexpr float GT_K0 = 0.7978845608028654f;             // sqrt(2 / pi)
constexpr float GT_K1 = 0.7978845608028654f * 0.044715f;  // sqrt(2 / pi) 0.044715
constexpr float GT_L = -2.0f * 1.4426950408889634f;       // -2 log2 e

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// s(x) = (1 + tanh(u)) / 2, the smoothed step of the approximation
__device__ __forceinline__ float gelu_step(float x) {
    const float x2 = x * x;
    return rcp_approx(1.0f + ex2_approx(x * fmaf(GT_L * GT_K1, x2, GT_L * GT_K0)));
}
__device__ __forceinline__ float gelu_fast(float x) { return x * gelu_step(x); }

constexpr int WS_EPI_WARPS = 16, WS_THREADS = (WS_EPI_WARPS + 1) * 32;
static_assert(WS_EPI_WARPS == 4 * FT_PARTS, "epilogue warps cover 4 lane quarters x FT_PARTS column parts");

// Chunk j (0..14) of one step's weight sequence: layer l, K slice s (columns
// 64 s .. 64 s + kw - 1 of the layer's input), all N output rows of the layer:
// layer 1 (K = 144) in slices of 64, 64 and 16 columns, the others (K = 256)
// in four of 64; N = 256 for the hidden layers and 144 for the head.
__host__ __device__ constexpr int ws_chunk_layer(int j) { return j < 3 ? 0 : (j - 3) / 4 + 1; }
__host__ __device__ constexpr int ws_chunk_slice(int j) { return j < 3 ? j : (j - 3) % 4; }
__host__ __device__ constexpr int ws_layer_n(int l) { return l == 3 ? N4 : WID; }
__host__ __device__ constexpr int ws_slice_kw(int l, int sl) {
    return (l == 0 ? K0 : WID) - sl * FT_KS < FT_KS ? (l == 0 ? K0 : WID) - sl * FT_KS : FT_KS;
}
__host__ __device__ constexpr int ws_chunk_bytes(int j) {
    return ws_layer_n(ws_chunk_layer(j)) * ws_slice_kw(ws_chunk_layer(j), ws_chunk_slice(j)) * 2;
}
__host__ __device__ constexpr int ws_chunk_off(int j) { return j == 0 ? 0 : ws_chunk_off(j - 1) + ws_chunk_bytes(j - 1); }
constexpr int WS_WP_BYTES = ws_chunk_off(FT_CHUNKS);  // packed weights per member
static_assert(WS_WP_BYTES == (K0 * WID + 2 * WID * WID + WID * N4) * 2, "every weight once");
static_assert(ws_chunk_bytes(0) <= FT_SW && ws_chunk_bytes(3) <= FT_SW && ws_chunk_bytes(11) <= FT_SW, "chunk fits");

// Wt (N x K row-major, per layer) -> the 15 chunk images: chunk j holds
// element (n, k) of its layer at cm_off(n, k - 64 s, N), the K-major
// core-matrix layout of an N-row operand with kw columns.
__global__ void k_pack_weights(const __nv_bfloat16 *__restrict__ W0, const __nv_bfloat16 *__restrict__ W1,
                               const __nv_bfloat16 *__restrict__ W2, const __nv_bfloat16 *__restrict__ W3,
                               unsigned char *Wp) {
    int u = blockIdx.x * blockDim.x + threadIdx.x;  // one 16-byte unit (8 columns of one row)
    if (u >= WS_WP_BYTES / 16) return;
    int j = 0;
    while (u >= ws_chunk_bytes(j) / 16) {
        u -= ws_chunk_bytes(j) / 16;
        j++;
    }
    const int l = ws_chunk_layer(j), sl = ws_chunk_slice(j), kw = ws_slice_kw(l, sl);
    const int K = l == 0 ? K0 : WID, N = ws_layer_n(l), KC = kw / 8;
    const __nv_bfloat16 *Wt = l == 0 ? W0 : (l == 1 ? W1 : (l == 2 ? W2 : W3));
    const int n = u / KC, kc = u - n * KC;
    const uint4 v = *reinterpret_cast<const uint4 *>(Wt + (size_t)n * K + sl * FT_KS + kc * 8);
    *reinterpret_cast<uint4 *>(Wp + ws_chunk_off(j) + cm_off(n, kc * 8, N)) = v;
}

// Bounded wait that lets the hardware park the thread (up to WS_SUSPEND_NS per
// try) instead of spinning, so that waiting warps leave the issue slots to the
// producer and to the warps that have work: at most WS_TRIES tries (~2 s).
constexpr unsigned WS_SUSPEND_NS = 100000;
constexpr int WS_TRIES = 20000;

__device__ __forceinline__ bool ws_wait(unsigned bar, unsigned parity) {
    unsigned done = 0;
    for (int it = 0; it < WS_TRIES && !done; it++)
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity), "r"(WS_SUSPEND_NS)
            : "memory");
    return done != 0;
}

__device__ __forceinline__ void ws_bulk(unsigned char *sW, const unsigned char *Wp, long c, unsigned bar_full) {
    const int j = (int)(c % FT_CHUNKS), b = (int)(c % FT_NBUF), bytes = ws_chunk_bytes(j);
    const unsigned bar = bar_full + 8u * (unsigned)b;
    const unsigned dst = (unsigned)__cvta_generic_to_shared(sW + (size_t)b * FT_SW);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(Wp + ws_chunk_off(j)), "r"(bytes), "r"(bar)
                 : "memory");
}

// Input rows of step t: columns 0..14 (u_t * u_inv) and the pad column, by the
// WS_EPI_WARPS * 32 epilogue threads, WS_U_PER thread each.  ws_load_u reads
// the features into registers (issued before the head layer's accumulator is
// ready, so that the global-memory latency runs under its MMAs); ws_store_u
// writes them into the operand.
constexpr int WS_U_PER = FT_M * 16 / (WS_EPI_WARPS * 32);
static_assert(WS_U_PER * WS_EPI_WARPS * 32 == FT_M * 16, "input columns per epilogue thread");
__device__ __forceinline__ void ws_load_u(const FusedArgs &a, int m0, int t, int tid, float (&v)[WS_U_PER]) {
#pragma unroll
    for (int k = 0; k < WS_U_PER; k++) {
        const int idx = tid + k * WS_EPI_WARPS * 32, r = idx >> 4, j = idx & 15, bb = m0 + r;
        v[k] = (j < NIN && bb < a.B) ? a.U[((size_t)bb * a.T + t) * NIN + j] * a.u_inv[j] : 0.0f;
    }
}
__device__ __forceinline__ void ws_store_u(unsigned char *sZ, int tid, const float (&v)[WS_U_PER]) {
#pragma unroll
    for (int k = 0; k < WS_U_PER; k++) {
        const int idx = tid + k * WS_EPI_WARPS * 32, r = idx >> 4, j = idx & 15, col = j < NIN ? j : K0 - 1;
        *reinterpret_cast<unsigned short *>(sZ + cm_off(r, col, FT_M)) = bf16_bits(v[k]);
    }
}

// the state columns of step 0 (given h, or zero)
__device__ __forceinline__ void ws_build_h0(const FusedArgs &a, unsigned char *sZ, const float *h, int m0, int tid,
                                            int nthr) {
    for (int idx = tid; idx < FT_M * NH; idx += nthr) {
        const int r = idx / NH, j = idx - r * NH, bb = m0 + r;
        const float v = (h && bb < a.B) ? h[(size_t)bb * NH + j] : 0.0f;
        *reinterpret_cast<unsigned short *>(sZ + cm_off(r, NIN + j, FT_M)) = bf16_bits(v);
    }
}

// The 144-column operand rows of a step (the forward's input rows z_t =
// [u_t, h_{t-1}, 0], the backward's dO_{t-1}), complete in shared memory once
// every epilogue warp has arrived on the hand-over barrier, copied to the tape
// in pieces of 8 columns (16 bytes; 18 pieces a row; row bb of the batch at
// dst + bb * K0).  Each warp copies the pieces that its own next epilogue
// overwrites -- the rows of its lane quarter, columns 64 s + 16 part .. + 15 of
// each slice s, i.e. pieces 8 s + 2 part and 8 s + 2 part + 1 -- so that no
// other warp can overwrite a piece before it has been copied.
__device__ __forceinline__ void ws_tape_rows(__nv_bfloat16 *dst, int B, const unsigned char *sZA, int m0, int quarter,
                                             int part, int lane) {
    constexpr int KG = K0 / 8;
    static_assert(KG * 8 == K0 && KG <= 3 * 8, "whole pieces per row, in three slices");
    for (int i = lane; i < 32 * 6; i += 32) {  // 32 rows x (3 slices x 2 pieces)
        const int r = quarter * 32 + i / 6, e = i % 6, kg = 8 * (e >> 1) + 2 * part + (e & 1), bb = m0 + r;
        if (kg < KG && bb < B)
            *reinterpret_cast<uint4 *>(dst + (size_t)bb * K0 + kg * 8) =
                *reinterpret_cast<const uint4 *>(sZA + cm_off(r, kg * 8, FT_M));
    }
}

// 16 accumulator columns of the warp's lane quarter (32 rows, one per lane)
// from tensor memory into r.  The load is asynchronous: r may be read only
// after tmem_wait16(r).
__device__ __forceinline__ void tmem_ld16(unsigned (&r)[16], unsigned taddr) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

// Waits for every tensor-memory load this thread has issued.  The registers of
// r pass through the statement, so no use of the loaded values can be
// scheduled above the wait.
__device__ __forceinline__ void tmem_wait16(unsigned (&r)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

// hidden layer l < 3, columns n0 .. n0 + 15 of row `row`: bias, GELU, the BF16
// operand of the next layer in shared memory, and the tape (y, a) if recorded
__device__ __forceinline__ void ws_act16(const FusedArgs &a, long tyo, int l, int t, int row, int b, int n0,
                                         const unsigned (&r)[16], unsigned char *sZA, const float *s_bias) {
    const float4 *bias = reinterpret_cast<const float4 *>(s_bias + l * WID + n0);
    unsigned yp[8], ap[8];
#pragma unroll
    for (int j = 0; j < 16; j += 4) {
        const float4 bv = bias[j >> 2];
        const float v0 = __uint_as_float(r[j]) + bv.x, v1 = __uint_as_float(r[j + 1]) + bv.y;
        const float v2 = __uint_as_float(r[j + 2]) + bv.z, v3 = __uint_as_float(r[j + 3]) + bv.w;
        yp[j >> 1] = bf16x2_bits(v0, v1);
        yp[(j >> 1) + 1] = bf16x2_bits(v2, v3);
        ap[j >> 1] = bf16x2_bits(gelu_fast(v0), gelu_fast(v1));
        ap[(j >> 1) + 1] = bf16x2_bits(gelu_fast(v2), gelu_fast(v3));
    }
    const uint4 a0 = make_uint4(ap[0], ap[1], ap[2], ap[3]), a1 = make_uint4(ap[4], ap[5], ap[6], ap[7]);
    *reinterpret_cast<uint4 *>(sZA + cm_off(row, n0, FT_M)) = a0;
    *reinterpret_cast<uint4 *>(sZA + cm_off(row, n0 + 8, FT_M)) = a1;
    if (a.tZ != nullptr && b < a.B) {
        const size_t o = tyo + ((size_t)t * a.B + b) * WID + n0;
        st_v8(a.tY[l] + o, make_uint4(yp[0], yp[1], yp[2], yp[3]), make_uint4(yp[4], yp[5], yp[6], yp[7]));
        st_v8(a.tA[l] + o, a0, a1);
    }
}

// State columns of an operand row: value v[j] of accumulator column n0 + j
// (kept where LO <= n0 + j < LO + NH) goes to operand column n0 + j + SHIFT of
// row `row`.  The shift is odd and n0 even, so the pairs (j, j + 1) with odd j
// land on an aligned column pair and go as one 4-byte store; j = 0 and 15 alone.
template <int LO, int SHIFT>
__device__ __forceinline__ void st_state16(unsigned char *sZA, int row, int n0, const float (&v)[16]) {
    static_assert(SHIFT & 1, "odd column shift");
    const auto ok = [&](int j) { return n0 + j >= LO && n0 + j < LO + NH; };
    const auto one = [&](int j) {
        *reinterpret_cast<unsigned short *>(sZA + cm_off(row, n0 + j + SHIFT, FT_M)) = bf16_bits(v[j]);
    };
    if (ok(0)) one(0);
#pragma unroll
    for (int j = 1; j < 15; j += 2) {
        const bool a0 = ok(j), a1 = ok(j + 1);
        if (a0 && a1) {
            *reinterpret_cast<unsigned *>(sZA + cm_off(row, n0 + j + SHIFT, FT_M)) = bf16x2_bits(v[j], v[j + 1]);
        } else {
            if (a0) one(j);
            if (a1) one(j + 1);
        }
    }
    if (ok(15)) one(15);
}

// tanh on the special-function unit (tanh.approx.f32, maximum relative error
// about 2^-11, a quarter of the BF16 rounding of the stored state)
__device__ __forceinline__ float tanh_approx(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// head layer, columns n0 .. n0 + 15 of row `row`: the stress outputs and the
// next state (tanh) into the state columns of the next step's input rows
__device__ __forceinline__ void ws_head16(const FusedArgs &a, int t, int row, int b, int n0, const unsigned (&r)[16],
                                          unsigned char *sZA, const float *s_bias, float *S, float *h) {
    float hv[16];
#pragma unroll
    for (int j = 0; j < 16; j++) {
        const int n = n0 + j;
        const float o = __uint_as_float(r[j]) + s_bias[3 * WID + n];
        hv[j] = tanh_approx(o);  // used for the state columns only
        if (n < NOUT) {
            if (b < a.B) S[(size_t)b * a.s_ld + t * NOUT + n] = a.s_mul ? o * a.s_mul[n] : o;
        } else if (n < NOUT + NH) {
            if (h && b < a.B && t + 1 == a.T) h[(size_t)b * NH + n - NOUT] = hv[j];
        }
    }
    st_state16<NOUT, NIN - NOUT>(sZA, row, n0, hv);
}

// Hands the epilogue's operand writes to the producer: shared-memory writes
// made visible to the tensor core's proxy, tensor-memory reads ordered before
// the synchronisation, then one arrival per warp on `bar`.
__device__ __forceinline__ void ws_hand_over(unsigned bar, int lane) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncwarp();
    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Epilogue of hidden layer l < 3 at step t for one warp: its 32 accumulator
// rows (lane quarter), 16 columns in each of the four 64-column slices (column
// part * 16 of the slice), slice by slice, handing each slice of the next
// operand over on `slice[s]` as soon as the sixteen warps have written it.  The
// load of the next 16 columns from tensor memory is in flight while the current
// ones are processed (two register sets, straight-line code: no register that
// a load is still filling is copied or read before its wait).
static_assert(WID / 16 == 4 * FT_PARTS, "a hidden layer's part is four 16-column chunks");
static_assert(N4 / 16 == 9 && FT_PARTS == 4, "the head's parts are 2, 2, 2 and 3 chunks");
static_assert(N4 == K0, "the head's output rows and the input rows have the same width");
__device__ __forceinline__ void ws_epilogue_hidden(const FusedArgs &a, long tyo, int l, int t, int quarter, int part,
                                                   int lane, unsigned tmem, unsigned char *sZA, const float *s_bias,
                                                   unsigned bar_slice, int m0) {
    const int row = quarter * 32 + lane, b = m0 + row, c = part * 16;
    const unsigned tq = tmem + ((unsigned)(quarter * 32) << 16) + (unsigned)((l & 1) * WID) + (unsigned)c;
    unsigned ra[16], rb[16];
    tmem_ld16(ra, tq);
    tmem_wait16(ra);
    tmem_ld16(rb, tq + FT_KS);
    ws_act16(a, tyo, l, t, row, b, c, ra, sZA, s_bias);
    ws_hand_over(bar_slice, lane);
    tmem_wait16(rb);
    tmem_ld16(ra, tq + 2 * FT_KS);
    ws_act16(a, tyo, l, t, row, b, FT_KS + c, rb, sZA, s_bias);
    ws_hand_over(bar_slice + 8u, lane);
    tmem_wait16(ra);
    tmem_ld16(rb, tq + 3 * FT_KS);
    ws_act16(a, tyo, l, t, row, b, 2 * FT_KS + c, ra, sZA, s_bias);
    ws_hand_over(bar_slice + 16u, lane);
    tmem_wait16(rb);
    ws_act16(a, tyo, l, t, row, b, 3 * FT_KS + c, rb, sZA, s_bias);
    ws_hand_over(bar_slice + 24u, lane);
}

// Epilogue of the head at step t for one warp: its lane quarter, the 2, 2, 2
// or 3 16-column chunks of its part (the accumulator of layer 3: columns 256 ..)
__device__ __forceinline__ void ws_epilogue_head(const FusedArgs &a, int t, int quarter, int part, int lane,
                                                 unsigned tmem, unsigned char *sZA, const float *s_bias, float *S,
                                                 float *h, int m0) {
    const int row = quarter * 32 + lane, b = m0 + row;
    const unsigned tq = tmem + ((unsigned)(quarter * 32) << 16) + (unsigned)WID;
    unsigned ra[16], rb[16];
    const int c = part * 32;  // chunks 2 part, 2 part + 1 (and 8 for the last part)
    tmem_ld16(ra, tq + c);
    tmem_wait16(ra);
    tmem_ld16(rb, tq + c + 16);
    ws_head16(a, t, row, b, c, ra, sZA, s_bias, S, h);
    tmem_wait16(rb);
    if (part == FT_PARTS - 1) {
        tmem_ld16(ra, tq + c + 32);
        ws_head16(a, t, row, b, c + 16, rb, sZA, s_bias, S, h);
        tmem_wait16(ra);
        ws_head16(a, t, row, b, c + 32, ra, sZA, s_bias, S, h);
    } else {
        ws_head16(a, t, row, b, c + 16, rb, sZA, s_bias, S, h);
    }
}

// The producer thread of the warp-specialised kernels: streams T x FT_CHUNKS
// weight chunks (per step the K slices of the four layers, see ws_chunk_*)
// through the FT_NBUF buffers and issues the MMAs slice by slice: slice s of
// layer l (its K columns 64 s ..) goes as soon as its operand columns are in
// place -- for the first layer when the whole input rows are (the `epi`
// barrier), for the others when the epilogue warps have finished slice s of
// the previous layer (`slice[s]`) -- so that the MMAs of a layer run under
// the epilogue of the previous one.  Layer l accumulates into tensor-memory
// columns (l % 2) * 256 .., the other half from the epilogue still reading the
// previous layer.  False on a timeout.
__device__ __forceinline__ bool ws_produce(const unsigned char *Wp, int T, unsigned char *sZA, unsigned char *sW,
                                           unsigned tmem, unsigned bar_full, unsigned bar_empty, unsigned bar_acc,
                                           unsigned bar_epi, unsigned bar_slice) {
    bool ok = true;
    const long n_chunks = (long)T * FT_CHUNKS;
    for (long c0 = 0; c0 < FT_NBUF && c0 < n_chunks; c0++) ws_bulk(sW, Wp, c0, bar_full);
    const unsigned aBase = (unsigned)__cvta_generic_to_shared(sZA);
    const unsigned lboA = (FT_M / 8) * 128;
    long c = 0;
    for (int t = 0; t < T && ok; t++)
        for (int l = 0; l < 4 && ok; l++) {
            const int N = ws_layer_n(l), ns = l == 0 ? 3 : 4;
            const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) |
                                   ((unsigned)(FT_M >> 4) << 24);
            const unsigned lboB = (unsigned)(N / 8) * 128;
            const unsigned dcol = tmem + (unsigned)((l & 1) * WID);
            for (int sl = 0; sl < ns && ok; sl++, c++) {
                // operand columns of slice sl in place: the input rows of step t
                // (completion t of `epi`), or slice sl of the previous layer's
                // epilogue (completion 3 t + l - 1 of `slice[sl]`)
                if (l == 0) {
                    if (sl == 0) ok = ws_wait(bar_epi, (unsigned)(t & 1));
                } else {
                    ok = ws_wait(bar_slice + 8u * sl, (unsigned)((3 * t + l - 1) & 1));
                }
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int b = (int)(c % FT_NBUF);
                ok = ws_wait(bar_full + 8u * b, (unsigned)((c / FT_NBUF) & 1));
                if (!ok) break;
                const unsigned wb = (unsigned)__cvta_generic_to_shared(sW + (size_t)b * FT_SW);
                const int nkk = ws_slice_kw(l, sl) >> 4;
                for (int kk = 0; kk < nkk; kk++) {
                    const uint64_t ad = tc_desc(aBase + (sl * (FT_KS / 16) + kk) * 2 * lboA, lboA, 128);
                    const uint64_t bd = tc_desc(wb + kk * 2 * lboB, lboB, 128);
                    const unsigned acc = (sl > 0 || kk > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dcol),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                        : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 bar_empty + 8u * b)
                             : "memory");
                // refill the buffer of chunk c - 1 once the MMAs that read it are done
                if (c >= 1 && c - 1 + FT_NBUF < n_chunks) {
                    const int pb = (int)((c - 1) % FT_NBUF);
                    ok = ws_wait(bar_empty + 8u * pb, (unsigned)(((c - 1) / FT_NBUF) & 1));
                    if (!ok) break;
                    ws_bulk(sW, Wp, c - 1 + FT_NBUF, bar_full);
                }
            }
            if (!ok) break;
            // the accumulator is complete once every MMA issued so far is
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_acc)
                         : "memory");
        }
    return ok;
}

__global__ void __launch_bounds__(WS_THREADS, 1) k_forward_ws(FusedArgs a) {
    extern __shared__ __align__(1024) unsigned char ft_smem[];
    __shared__ __align__(8) unsigned long long s_full[FT_NBUF], s_empty[FT_NBUF], s_acc, s_epi, s_slice[4];
    __shared__ unsigned s_tmem;
    __shared__ __align__(16) float s_bias[3 * WID + N4];  // b1, b2, b3, b4
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mk = blockIdx.y, m0 = blockIdx.x * FT_M;
    const long tzo = mk * a.tz_ms, tyo = mk * a.ty_ms;  // this member's tape
    unsigned char *sZA = ft_smem, *sW = ft_smem + FT_SA;  // input rows and activations share the first 64 KB
    const float *theta = a.theta[mk];
    float *S = a.S + mk * a.s_mstride;
    float *h = a.h ? a.h + mk * a.h_mstride : nullptr;
    const int T = a.T;

    if (warp == 0) {
        const unsigned dst = (unsigned)__cvta_generic_to_shared(&s_tmem);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst),
                     "r"(FT_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int i = tid; i < 3 * WID + N4; i += WS_THREADS)
        s_bias[i] = theta[i < WID ? OFF_B1 + i
                                  : (i < 2 * WID ? OFF_B2 + i - WID
                                                 : (i < 3 * WID ? OFF_B3 + i - 2 * WID : OFF_B4 + i - 3 * WID))];
    const unsigned bar_full = (unsigned)__cvta_generic_to_shared(&s_full[0]);
    const unsigned bar_empty = (unsigned)__cvta_generic_to_shared(&s_empty[0]);
    const unsigned bar_acc = (unsigned)__cvta_generic_to_shared(&s_acc);
    const unsigned bar_epi = (unsigned)__cvta_generic_to_shared(&s_epi);
    const unsigned bar_slice = (unsigned)__cvta_generic_to_shared(&s_slice[0]);
    if (tid == 0) {
        for (int i = 0; i < FT_NBUF; i++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_full + 8 * i) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_empty + 8 * i) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_acc) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_epi), "r"(WS_EPI_WARPS) : "memory");
        for (int i = 0; i < 4; i++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_slice + 8 * i), "r"(WS_EPI_WARPS)
                         : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = s_tmem;
    bool ok = true;

    if (warp == WS_EPI_WARPS) {
        // ---- producer: weight chunks and MMAs (one thread) ----
        if (lane == 0) {
            ok = ws_produce(a.Wp[mk], T, sZA, sW, tmem, bar_full, bar_empty, bar_acc, bar_epi, bar_slice);
            if (!ok) atomicExch(a.err, RC_ETIMEOUT);
        }
    } else {
        // ---- epilogue warps ----
        const int etid = tid, nthr = WS_EPI_WARPS * 32, quarter = warp & 3, part = warp >> 2;
        const bool tape = a.tZ != nullptr;
        float uv[WS_U_PER];
        ws_load_u(a, m0, 0, etid, uv);
        ws_store_u(sZA, etid, uv);
        ws_build_h0(a, sZA, h, m0, etid, nthr);
        ws_hand_over(bar_epi, lane);
        // z rows to the tape once all warps have written them: completion 0 of
        // `epi` (the initial rows), completion t + 1 (after the head of step t)
        if (tape) {
            ok = __all_sync(0xffffffffu, ws_wait(bar_epi, 0u));
            if (ok) ws_tape_rows(a.tZ + tzo, a.B, sZA, m0, quarter, part, lane);
            __syncwarp();
        }
        for (int t = 0; t < T && ok; t++)
            for (int l = 0; l < 4 && ok; l++) {
                if (l == 3 && t + 1 < T) ws_load_u(a, m0, t + 1, etid, uv);
                ok = __all_sync(0xffffffffu, ws_wait(bar_acc, (unsigned)((t * 4 + l) & 1)));
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (l < 3) {
                    ws_epilogue_hidden(a, tyo, l, t, quarter, part, lane, tmem, sZA, s_bias, bar_slice, m0);
                    continue;
                }
                ws_epilogue_head(a, t, quarter, part, lane, tmem, sZA, s_bias, S, h, m0);
                if (t + 1 < T) ws_store_u(sZA, etid, uv);
                ws_hand_over(bar_epi, lane);
                if (tape && t + 1 < T) {
                    ok = __all_sync(0xffffffffu, ws_wait(bar_epi, (unsigned)((t + 1) & 1)));
                    if (ok) ws_tape_rows(a.tZ + tzo + (size_t)(t + 1) * a.B * K0, a.B, sZA, m0, quarter, part, lane);
                    __syncwarp();
                }
            }
        if (!ok && lane == 0) atomicExch(a.err, RC_ETIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(FT_TMEM_COLS)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// Weight gradients on tcgen05: G[Kd x Nd] += sum over rows r of X[r][m] D[r][n]
// (X: the layer inputs of every step, rows x Kd; D: the output gradients,
// rows x Nd; both row-major, Kd, Nd <= 256 and multiples of 16).  Both
// operands are the transposed (MN-major) kind for the tensor core: a 16-byte
// piece of a row (8 consecutive m, or n) is one row of a core matrix, so the
// rows stream into shared memory with plain 16-byte asynchronous copies.
// Core matrix (mn/8, r/8) of a stage sits at byte (r/8 * MN/8 + mn/8) * 128,
// piece r%8 at +16 (r%8); the descriptors take the stride between core
// matrices along r as the leading and along mn as the stride byte offset, as
// for the K-major operands of the other kernels.  A CTA owns a range of rows
// and the whole output: two 128-row accumulators (m < 128, m >= 128) of up to
// 256 FP32 columns each fill the 512 columns of tensor memory; a three-stage
// pipeline of 64-row chunks (X 32 KB + D 32 KB per stage) keeps the copies of
// the next chunks in flight while the MMAs of the current one run; the partial
// sums are added into G (FP32 atomics).  With Gb, the column sums of D (the
// bias gradient) are formed from the same staged chunks: lanes 8p .. 8p+7 read
// the eight rows of one core matrix (128 contiguous bytes) and keep eight
// running sums each.  Member blockIdx.y of a member-batched launch reads
// X + y x_ms, D + y d_ms and adds into G + y g_ms, Gb + y g_ms.
// ---------------------------------------------------------------------------
constexpr int WG_ROWS = 64, WG_STAGES = 3, WG_THREADS = 128;
constexpr int WG_SX = 256 * WG_ROWS * 2, WG_SD = 256 * WG_ROWS * 2, WG_STAGE = WG_SX + WG_SD;
constexpr int WG_SMEM = WG_STAGES * WG_STAGE;

__global__ void __launch_bounds__(WG_THREADS, 1)
    k_wgrad_tc05(const __nv_bfloat16 *__restrict__ X, long x_ms, int Kd, const __nv_bfloat16 *__restrict__ D,
                 long d_ms, int Nd, long rows, long rows_per_cta, float *G, float *Gb, long g_ms, int *err) {
    extern __shared__ __align__(1024) unsigned char wg_smem[];
    __shared__ __align__(8) unsigned long long s_done[WG_STAGES];
    __shared__ unsigned s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    X += blockIdx.y * x_ms;
    D += blockIdx.y * d_ms;
    G += blockIdx.y * g_ms;
    if (Gb) Gb += blockIdx.y * g_ms;
    float csum[2][8];  // column sums: pieces tid / 8 and tid / 8 + 16, row tid % 8 of each core matrix
#pragma unroll
    for (int q = 0; q < 2; q++)
#pragma unroll
        for (int e = 0; e < 8; e++) csum[q][e] = 0.0f;
    const long r_begin = (long)blockIdx.x * rows_per_cta;
    const long r_end = r_begin + rows_per_cta < rows ? r_begin + rows_per_cta : rows;
    const int n_chunks = r_end > r_begin ? (int)((r_end - r_begin + WG_ROWS - 1) / WG_ROWS) : 0;
    const int MH = Kd > 128 ? 2 : 1;  // accumulators (m < 128, m >= 128)
    const int XC = Kd >> 3, DC = Nd >> 3;  // 16-byte pieces per row

    if (warp == 0) {
        const unsigned dst = (unsigned)__cvta_generic_to_shared(&s_tmem);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < WG_STAGES; i++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((unsigned)__cvta_generic_to_shared(&s_done[i]))
                         : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // chunk c into its stage: X rows as 128-row halves [MH][...], D rows; pieces
    // past the matrix (rows, columns) are zero-filled
    auto load_chunk = [&](int c) {
        unsigned char *sx = wg_smem + (size_t)(c % WG_STAGES) * WG_STAGE, *sd = sx + WG_SX;
        const long r0 = r_begin + (long)c * WG_ROWS;
        for (int idx = tid; idx < WG_ROWS * 32; idx += WG_THREADS) {  // X: 64 rows x 32 pieces (256 columns)
            const int rr = idx >> 5, pc = idx & 31, m = pc * 8, h = m >> 7, mm = m & 127;
            if (h >= MH) continue;
            const long r = r0 + rr;
            const bool in = r < r_end && pc < XC;
            const __nv_bfloat16 *src = X + (in ? r * Kd + m : 0);
            const unsigned dst = (unsigned)__cvta_generic_to_shared(
                sx + (size_t)h * (128 * WG_ROWS * 2) + ((rr >> 3) * 16 + (mm >> 3)) * 128 + (rr & 7) * 16);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(in ? 16 : 0)
                         : "memory");
        }
        for (int idx = tid; idx < WG_ROWS * DC; idx += WG_THREADS) {  // D: 64 rows x Nd/8 pieces
            const int rr = idx / DC, pc = idx - rr * DC;
            const long r = r0 + rr;
            const bool in = r < r_end;
            const __nv_bfloat16 *src = D + (in ? r * Nd + pc * 8 : 0);
            const unsigned dst = (unsigned)__cvta_generic_to_shared(sd + ((rr >> 3) * DC + pc) * 128 + (rr & 7) * 16);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(in ? 16 : 0)
                         : "memory");
        }
    };
    for (int c = 0; c < WG_STAGES - 1; c++) {
        if (c < n_chunks) load_chunk(c);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = s_tmem;
    // instruction descriptor: FP32 accumulator, BF16 A and B, both transposed (MN-major), N/8, M/16
    const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                           ((unsigned)(Nd >> 3) << 17) | ((unsigned)(128 >> 4) << 24);
    const unsigned lboX = 16 * 128, lboD = (unsigned)DC * 128;  // between core matrices along r
    bool ok = true;
    int issued = -1;  // last chunk whose MMAs were issued
    for (int c = 0; c < n_chunks && ok; c++) {
        asm volatile("cp.async.wait_group %0;" ::"n"(WG_STAGES - 2) : "memory");
        __syncthreads();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned sx = (unsigned)__cvta_generic_to_shared(wg_smem + (size_t)(c % WG_STAGES) * WG_STAGE);
            const unsigned sd = sx + WG_SX;
            for (int h = 0; h < MH; h++)
                for (int ks = 0; ks < WG_ROWS / 16; ks++) {
                    const uint64_t ad = tc_desc(sx + h * (128 * WG_ROWS * 2) + ks * 2 * lboX, lboX, 128);
                    const uint64_t bd = tc_desc(sd + ks * 2 * lboD, lboD, 128);
                    const unsigned acc = (c > 0 || ks > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + (unsigned)(h * 256)),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                        : "memory");
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             (unsigned)__cvta_generic_to_shared(&s_done[c % WG_STAGES]))
                         : "memory");
        }
        issued = c;
        if (Gb) {  // this chunk's rows into the column sums (rows past the matrix are zero)
            const unsigned char *sd = wg_smem + (size_t)(c % WG_STAGES) * WG_STAGE + WG_SX;
            const int j = tid & 7, p = tid >> 3;
#pragma unroll
            for (int q = 0; q < 2; q++) {
                const int pc = p + 16 * q;
                if (pc < DC)
                    for (int rg = 0; rg < WG_ROWS / 8; rg++) {
                        const uint4 v = *reinterpret_cast<const uint4 *>(sd + ((rg * DC + pc) * 128 + j * 16));
                        const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int e = 0; e < 4; e++) {
                            const __nv_bfloat162 x2 = *reinterpret_cast<const __nv_bfloat162 *>(&w[e]);
                            csum[q][2 * e] += __low2float(x2);
                            csum[q][2 * e + 1] += __high2float(x2);
                        }
                    }
            }
        }
        // the stage of chunk c - 1 takes chunk c + STAGES - 1 once its MMAs are done
        const int cn = c + WG_STAGES - 1;
        if (cn < n_chunks) {
            if (c >= 1) {
                const int cp = c - 1;
                ok = ws_wait((unsigned)__cvta_generic_to_shared(&s_done[cp % WG_STAGES]),
                             (unsigned)((cp / WG_STAGES) & 1));
            }
            if (ok) load_chunk(cn);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        ok = __syncthreads_and(ok);
    }
    // the accumulators are complete once the last chunk's MMAs are
    if (ok && n_chunks > 0) {
        const int cl = n_chunks - 1;
        ok = ws_wait((unsigned)__cvta_generic_to_shared(&s_done[cl % WG_STAGES]), (unsigned)((cl / WG_STAGES) & 1));
    }
    ok = __syncthreads_and(ok);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok && n_chunks > 0 && Gb) {
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int pc = (tid >> 3) + 16 * q;
#pragma unroll
            for (int e = 0; e < 8; e++) {
                float v = csum[q][e];
                v += __shfl_xor_sync(0xffffffffu, v, 1);
                v += __shfl_xor_sync(0xffffffffu, v, 2);
                v += __shfl_xor_sync(0xffffffffu, v, 4);
                if ((tid & 7) == 0 && pc < DC) atomicAdd(&Gb[pc * 8 + e], v);
            }
        }
    }
    if (ok && n_chunks > 0) {
        for (int h = 0; h < MH; h++) {
            const int m = h * 128 + warp * 32 + lane;
            for (int c0 = 0; c0 < Nd; c0 += 16) {
                unsigned r[16];
                const unsigned taddr = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)(h * 256 + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];\n"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15])
                    : "r"(taddr)
                    : "memory");
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (m < Kd) {
#pragma unroll
                    for (int j = 0; j < 16; j++) atomicAdd(&G[(size_t)m * Nd + c0 + j], __uint_as_float(r[j]));
                }
            }
        }
    }
    if (!ok) {
        if (tid == 0) atomicExch(err, RC_ETIMEOUT);
        // let the copies and MMAs in flight finish before the memory is released
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        if (tid == 0)
            for (int c = issued >= WG_STAGES ? issued - WG_STAGES + 1 : 0; c <= issued; c++)
                ws_wait((unsigned)__cvta_generic_to_shared(&s_done[c % WG_STAGES]), (unsigned)((c / WG_STAGES) & 1));
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

// ---------------------------------------------------------------------------
// The whole BPTT data-gradient chain in one kernel (tcgen05), the mirror of
// k_forward_ws: a CTA owns 128 rows of one member and walks the steps
// t = T-1 .. 0; per step the four products
//   dY3 = (dO_t W4^T) * gelu'(Y3_t),  dY2 = (dY3 W3^T) * gelu'(Y2_t),
//   dY1 = (dY2 W2^T) * gelu'(Y1_t),   dZ_t = dY1 W1^T
// run back to back on the tensor cores with the operand in shared memory and
// the accumulator in tensor memory.  They have the forward's shapes in the
// reverse order, so the same producer streams the members' backward weight
// images (W4, W3, W2, W1 packed by k_pack_weights as the forward packs W1^T ..
// W4^T).  The epilogue warps read Y_l from the tape, write dY_l into shared
// memory (the next operand) and to global memory (for the weight gradients);
// after dZ_t they build dO_{t-1} = [gscale (s - y / s_scale), dZ_t(state) *
// (1 - h_{t-1}^2), 0] from the predictions, the targets and the state row of
// the tape.  GELU' is the derivative of the forward's tanh approximation
// (gelu_grad_fast), the function the fused forward evaluates.
// ---------------------------------------------------------------------------
struct BwdArgs {
    int B, T;
    const float *S;  // predictions in network units: member k, row b, step t at S + k s_mstride + (b T + t) NOUT
    long s_mstride;
    const float *Y;  // targets, (b T + t) NOUT
    const float *s_inv;
    float gscale;
    const __nv_bfloat16 *Z, *Yt[3];  // tape of the launch's first member: Z rows (t B + b) K0, Y1..Y3 rows WID
    __nv_bfloat16 *dO, *dY[3];       // outputs, rows (t B + b): dO N4 wide, dY1..dY3 WID wide
    long z_ms, y_ms, o_ms;           // member strides (elements)
    const unsigned char *Wb[FT_MAXK];
    int *err;
};

// derivative of the fused kernels' GELU: s + x s (1 - s) 2 (sqrt(2/pi) + 3
// sqrt(2/pi) 0.044715 x^2), with s = gelu_step(x)
__device__ __forceinline__ float gelu_grad_fast(float x) {
    const float sx = gelu_step(x);
    return fmaf(x * sx * (1.0f - sx), 2.0f * fmaf(3.0f * GT_K1, x * x, GT_K0), sx);
}

// dO of step tp = t - 1 (or T - 1 at the start, with no state part): stress
// columns and zero padding of row `row` (the state columns come from dZ)
__device__ __forceinline__ float wb_stress_grad(const BwdArgs &a, const float *S, int b, int tp, int n) {
    const size_t i = ((size_t)b * a.T + tp) * NOUT + n;
    return a.gscale * (S[i] - a.Y[i] * a.s_inv[n]);
}

// Columns c0 .. c0 + 15 and c0 + 64 .. c0 + 79 of the tape row Y_{3-l} of
// step t (row b) into registers (zero past the batch): the warp's 16 columns
// in two consecutive slices.  The first two slices are loaded before the
// layer's accumulator is ready, so that the global-memory latency runs under
// the layer's MMAs; the other two while the first is processed.
__device__ __forceinline__ void wb_load_y(const BwdArgs &a, long yo, int l, int t, int c0, int b, uint4 (&y)[4]) {
#pragma unroll
    for (int k = 0; k < 4; k++) y[k] = make_uint4(0u, 0u, 0u, 0u);
    if (l < 3 && b < a.B) {
        const __nv_bfloat16 *Yg = a.Yt[2 - l] + yo + ((size_t)t * a.B + b) * WID + c0;
        ld_v8(Yg, y[0], y[1]);
        ld_v8(Yg + FT_KS, y[2], y[3]);
    }
}

// What the warp's epilogue of product l at step t reads from the tape, loaded
// before the accumulator is ready: for a hidden layer its columns of the first
// two slices of Y_{3-l}, for dZ columns part * 32 .. part * 32 + 31 of the Z row.
__device__ __forceinline__ void wb_prefetch(const BwdArgs &a, long yo, long zo, int l, int t, int part, int b,
                                            uint4 (&y)[4]) {
    if (l < 3) {
        wb_load_y(a, yo, l, t, part * 16, b, y);
        return;
    }
#pragma unroll
    for (int k = 0; k < 4; k++) y[k] = make_uint4(0u, 0u, 0u, 0u);
    if (t > 0 && b < a.B) {
        const __nv_bfloat16 *Zg = a.Z + zo + ((size_t)t * a.B + b) * K0 + part * 32;
        ld_v8(Zg, y[0], y[1]);
        ld_v8(Zg + 16, y[2], y[3]);
    }
}

// dY = acc * gelu'(Y) for columns n0 .. n0 + 15 of row `row`: the next
// operand in shared memory and the dY rows in global memory
__device__ __forceinline__ void wb_dy16(const BwdArgs &a, long yo, int l, int t, int row, int b, int n0,
                                        const unsigned (&r)[16], const uint4 &y0, const uint4 &y1,
                                        unsigned char *sZA) {
    const unsigned yw[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
    unsigned dp[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const __nv_bfloat162 yy = *reinterpret_cast<const __nv_bfloat162 *>(&yw[j]);
        const float g0 = __uint_as_float(r[2 * j]) * gelu_grad_fast(__low2float(yy));
        const float g1 = __uint_as_float(r[2 * j + 1]) * gelu_grad_fast(__high2float(yy));
        dp[j] = bf16x2_bits(g0, g1);
    }
    const uint4 d0 = make_uint4(dp[0], dp[1], dp[2], dp[3]), d1 = make_uint4(dp[4], dp[5], dp[6], dp[7]);
    *reinterpret_cast<uint4 *>(sZA + cm_off(row, n0, FT_M)) = d0;
    *reinterpret_cast<uint4 *>(sZA + cm_off(row, n0 + 8, FT_M)) = d1;
    if (b < a.B) st_v8(a.dY[2 - l] + yo + ((size_t)t * a.B + b) * WID + n0, d0, d1);
}

// dO state columns from dZ for accumulator columns n0 .. n0 + 15 of row
// `row`, into the next operand: dZ(h) * (1 - h^2) (the tanh of the state), h
// from the Z tape words z
__device__ __forceinline__ void wb_dz16(int row, int n0, const unsigned (&r)[16], const uint4 &z0, const uint4 &z1,
                                        unsigned char *sZA) {
    const unsigned zw[8] = {z0.x, z0.y, z0.z, z0.w, z1.x, z1.y, z1.z, z1.w};
    float v[16];
#pragma unroll
    for (int j = 0; j < 16; j++) {
        const __nv_bfloat162 hh = *reinterpret_cast<const __nv_bfloat162 *>(&zw[j >> 1]);
        const float h = (j & 1) ? __high2float(hh) : __low2float(hh);
        v[j] = __uint_as_float(r[j]) * (1.0f - h * h);
    }
    st_state16<NIN, NOUT - NIN>(sZA, row, n0, v);
}

// Epilogue of backward product l at step t for one warp (lane quarter, column
// part); y holds what wb_prefetch loaded.  Hidden layers go slice by slice as
// the forward's do (16 columns of each 64-column slice, each slice handed over
// on `slice[s]`, the next tensor-memory load in flight); dZ (l = 3, the
// accumulator in columns 256 ..) by the part's 2, 2, 2 or 3 chunks.
__device__ __forceinline__ void wb_epilogue(const BwdArgs &a, long zo, long yo, long oo, int l, int t, int quarter,
                                            int part, int lane, unsigned tmem, unsigned char *sZA, const float *S,
                                            int m0, const uint4 (&y)[4], unsigned bar_slice, const float (&g)[NOUT]) {
    const int B = a.B, row = quarter * 32 + lane, b = m0 + row;
    const bool live = b < B;
    if (l < 3) {  // dY_{3-l} = acc * gelu'(Y_{3-l})
        const int c = part * 16;
        const unsigned tq = tmem + ((unsigned)(quarter * 32) << 16) + (unsigned)((l & 1) * WID) + (unsigned)c;
        unsigned ra[16], rb[16];
        uint4 y2[4];
        tmem_ld16(ra, tq);
        wb_load_y(a, yo, l, t, 2 * FT_KS + c, b, y2);
        tmem_wait16(ra);
        tmem_ld16(rb, tq + FT_KS);
        wb_dy16(a, yo, l, t, row, b, c, ra, y[0], y[1], sZA);
        ws_hand_over(bar_slice, lane);
        tmem_wait16(rb);
        tmem_ld16(ra, tq + 2 * FT_KS);
        wb_dy16(a, yo, l, t, row, b, FT_KS + c, rb, y[2], y[3], sZA);
        ws_hand_over(bar_slice + 8u, lane);
        tmem_wait16(ra);
        tmem_ld16(rb, tq + 3 * FT_KS);
        wb_dy16(a, yo, l, t, row, b, 2 * FT_KS + c, ra, y2[0], y2[1], sZA);
        ws_hand_over(bar_slice + 16u, lane);
        tmem_wait16(rb);
        wb_dy16(a, yo, l, t, row, b, 3 * FT_KS + c, rb, y2[2], y2[3], sZA);
        ws_hand_over(bar_slice + 24u, lane);
        return;
    }
    // dZ_t -> dO_{t-1}; nothing to hand on after step 0.  y holds columns
    // part * 32 .. part * 32 + 31 of the Z tape row [u_t, h_{t-1}, 0]
    // (wb_prefetch); the last part's third chunk is loaded here.
    if (t == 0) return;
    const unsigned tq = tmem + ((unsigned)(quarter * 32) << 16) + (unsigned)WID;
    const int c = part * 32;
    unsigned ra[16], rb[16];
    uint4 z2[2] = {make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u)};
    tmem_ld16(ra, tq + c);
    if (part == FT_PARTS - 1 && live) ld_v8(a.Z + zo + ((size_t)t * B + b) * K0 + c + 32, z2[0], z2[1]);
    tmem_wait16(ra);
    tmem_ld16(rb, tq + c + 16);
    wb_dz16(row, c, ra, y[0], y[1], sZA);
    tmem_wait16(rb);
    if (part == FT_PARTS - 1) {
        tmem_ld16(ra, tq + c + 32);
        wb_dz16(row, c + 16, rb, y[2], y[3], sZA);
        tmem_wait16(ra);
        wb_dz16(row, c + 32, ra, z2[0], z2[1], sZA);
    } else {
        wb_dz16(row, c + 16, rb, y[2], y[3], sZA);
    }
    if (part == 0) {  // the stress columns (g, formed two products earlier) and the padding of dO_{t-1}
#pragma unroll
        for (int n = 0; n < NOUT; n++) *reinterpret_cast<unsigned short *>(sZA + cm_off(row, n, FT_M)) = bf16_bits(g[n]);
        for (int n = NOUT + NH; n < K0; n++) *reinterpret_cast<unsigned short *>(sZA + cm_off(row, n, FT_M)) = 0;
    }
}

__global__ void __launch_bounds__(WS_THREADS, 1) k_backward_ws(BwdArgs a) {
    extern __shared__ __align__(1024) unsigned char ft_smem[];
    __shared__ __align__(8) unsigned long long s_full[FT_NBUF], s_empty[FT_NBUF], s_acc, s_epi, s_slice[4];
    __shared__ unsigned s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mk = blockIdx.y, m0 = blockIdx.x * FT_M;
    const long zo = mk * a.z_ms, yo = mk * a.y_ms, oo = mk * a.o_ms;
    unsigned char *sZA = ft_smem, *sW = ft_smem + FT_SA;
    const float *S = a.S + mk * a.s_mstride;
    const int T = a.T;

    if (warp == 0) {
        const unsigned dst = (unsigned)__cvta_generic_to_shared(&s_tmem);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst),
                     "r"(FT_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    const unsigned bar_full = (unsigned)__cvta_generic_to_shared(&s_full[0]);
    const unsigned bar_empty = (unsigned)__cvta_generic_to_shared(&s_empty[0]);
    const unsigned bar_acc = (unsigned)__cvta_generic_to_shared(&s_acc);
    const unsigned bar_epi = (unsigned)__cvta_generic_to_shared(&s_epi);
    const unsigned bar_slice = (unsigned)__cvta_generic_to_shared(&s_slice[0]);
    if (tid == 0) {
        for (int i = 0; i < FT_NBUF; i++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_full + 8 * i) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_empty + 8 * i) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_acc) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_epi), "r"(WS_EPI_WARPS) : "memory");
        for (int i = 0; i < 4; i++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_slice + 8 * i), "r"(WS_EPI_WARPS)
                         : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = s_tmem;
    bool ok = true;

    if (warp == WS_EPI_WARPS) {
        if (lane == 0) {
            ok = ws_produce(a.Wb[mk], T, sZA, sW, tmem, bar_full, bar_empty, bar_acc, bar_epi, bar_slice);
            if (!ok) atomicExch(a.err, RC_ETIMEOUT);
        }
    } else {
        const int etid = tid, nthr = WS_EPI_WARPS * 32, quarter = warp & 3, part = warp >> 2;
        // dO_{T-1}: stress columns only
        for (int idx = etid; idx < FT_M * K0; idx += nthr) {
            const int r = idx / K0, n = idx - r * K0, b = m0 + r;
            const float v = (n < NOUT && b < a.B) ? wb_stress_grad(a, S, b, T - 1, n) : 0.0f;
            *reinterpret_cast<unsigned short *>(sZA + cm_off(r, n, FT_M)) = bf16_bits(v);
        }
        ws_hand_over(bar_epi, lane);
        // dO rows to global memory once all warps have written them: completion
        // 0 of `epi` (dO_{T-1}), completion i + 1 (after the dZ epilogue of
        // iteration i, dO_{t-1})
        ok = __all_sync(0xffffffffu, ws_wait(bar_epi, 0u));
        if (ok) ws_tape_rows(a.dO + oo + (size_t)(T - 1) * a.B * N4, a.B, sZA, m0, quarter, part, lane);
        __syncwarp();
        float g[NOUT];  // the part-0 warps' stress gradients of dO_{t-1}, loaded while dY2 and dY1 run
#pragma unroll
        for (int n = 0; n < NOUT; n++) g[n] = 0.0f;
        for (int i = 0; i < T && ok; i++)
            for (int l = 0; l < 4 && ok; l++) {
                const int t = T - 1 - i;
                if (part == 0 && l == 1 && t > 0) {
                    const int b = m0 + quarter * 32 + lane;
#pragma unroll
                    for (int n = 0; n < NOUT; n++) g[n] = b < a.B ? wb_stress_grad(a, S, b, t - 1, n) : 0.0f;
                }
                uint4 y[4];
                wb_prefetch(a, yo, zo, l, t, part, m0 + quarter * 32 + lane, y);
                ok = __all_sync(0xffffffffu, ws_wait(bar_acc, (unsigned)((i * 4 + l) & 1)));
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                wb_epilogue(a, zo, yo, oo, l, t, quarter, part, lane, tmem, sZA, S, m0, y, bar_slice, g);
                if (l < 3) continue;  // the hidden epilogues hand their slices over themselves
                ws_hand_over(bar_epi, lane);
                if (t > 0) {
                    ok = __all_sync(0xffffffffu, ws_wait(bar_epi, (unsigned)((i + 1) & 1)));
                    if (ok) ws_tape_rows(a.dO + oo + (size_t)(t - 1) * a.B * N4, a.B, sZA, m0, quarter, part, lane);
                    __syncwarp();
                }
            }
        if (!ok && lane == 0) atomicExch(a.err, RC_ETIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(FT_TMEM_COLS)
                     : "memory");
    }
}

void prepare_ws() {
    cudaFuncSetAttribute(k_forward_ws, cudaFuncAttributeMaxDynamicSharedMemorySize, FT_SMEM);
    cudaFuncSetAttribute(k_backward_ws, cudaFuncAttributeMaxDynamicSharedMemorySize, FT_SMEM);
    cudaFuncSetAttribute(k_wgrad_tc05, cudaFuncAttributeMaxDynamicSharedMemorySize, WG_SMEM);
}

int g_n_sm = 0;

// the weight gradients of nb members: G_i += X_i^T D_i over `rows` rows, about
// one CTA per SM in all
void wgrad_tc05(cudaStream_t st, const __nv_bfloat16 *X, long x_ms, int Kd, const __nv_bfloat16 *D, long d_ms, int Nd,
                long rows, float *G, float *Gb, long g_ms, int nb, int *err) {
    if (g_n_sm <= 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (g_n_sm <= 0) g_n_sm = 1;
    }
    const int per_member = std::max(1, g_n_sm / nb);
    long rpc = (rows + per_member - 1) / per_member;
    rpc = (rpc + WG_ROWS - 1) / WG_ROWS * WG_ROWS;
    const int nx = (int)((rows + rpc - 1) / rpc);
    k_wgrad_tc05<<<dim3(nx, nb), WG_THREADS, WG_SMEM, st>>>(X, x_ms, Kd, D, d_ms, Nd, rows, rpc, G, Gb, g_ms, err);
}


// ---------------------------------------------------------------------------
// elementwise kernels
// ---------------------------------------------------------------------------

// z_t rows: [u_t / u_scale, h_{t-1} (already there, or zero at t = 0), 0]
__global__ void k_build_input(const float *__restrict__ U, int B, int T, int t, const float *__restrict__ u_inv,
                              __nv_bfloat16 *Z, int zero_state) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * K0) return;
    const int b = idx / K0, k = idx % K0;
    if (k < NIN) Z[idx] = __float2bfloat16(U[((size_t)b * T + t) * NIN + k] * u_inv[k]);
    else if (k >= NIN + NH || zero_state) Z[idx] = __float2bfloat16(0.0f);
}

// head gradient do_t = [scale (s - y/s_scale), dh (1 - h^2), 0]; loss partials
// Member blockIdx.y of a member-batched launch: S, Hrow, dZ and dO advance by
// their member strides.
__global__ void k_head_grad(const float *__restrict__ S, long s_ms, const float *__restrict__ Y, int B, int T, int t,
                            const float *__restrict__ s_inv, const __nv_bfloat16 *__restrict__ Hrow, long h_ms,
                            const float *__restrict__ dZ, long dz_ms, int have_dh, float gscale, __nv_bfloat16 *dO,
                            long do_ms) {
    const int z = blockIdx.y;
    S += z * s_ms;
    Hrow += z * h_ms;
    dZ += z * dz_ms;
    dO += z * do_ms;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * N4) return;
    const int b = idx / N4, n = idx % N4;
    float v = 0.0f;
    if (n < NOUT) {
        v = gscale * (S[((size_t)b * T + t) * NOUT + n] - Y[((size_t)b * T + t) * NOUT + n] * s_inv[n]);
    } else if (n < NOUT + NH && have_dh) {
        const float h = __bfloat162float(Hrow[(size_t)b * K0 + NIN + (n - NOUT)]);
        v = dZ[(size_t)b * K0 + NIN + (n - NOUT)] * (1.0f - h * h);
    }
    dO[idx] = __float2bfloat16(v);
}

// loss partial sums sum (s - y / s_scale)^2 over the n stress values of member
// blockIdx.y (S at + y s_ms), one FP64 atomic per block into loss_acc[y]
constexpr int LOSS_THREADS = 256, LOSS_PER_THREAD = 16;
__global__ void __launch_bounds__(LOSS_THREADS) k_loss(const float *__restrict__ S, long s_ms,
                                                       const float *__restrict__ Y, long n,
                                                       const float *__restrict__ s_inv, double *loss_acc) {
    __shared__ double s_part[LOSS_THREADS / 32];
    S += blockIdx.y * s_ms;
    const long i0 = (long)blockIdx.x * LOSS_THREADS * LOSS_PER_THREAD + threadIdx.x;
    double l = 0.0;
#pragma unroll 4
    for (int k = 0; k < LOSS_PER_THREAD; k++) {
        const long i = i0 + (long)k * LOSS_THREADS;
        if (i < n) {
            const float r = S[i] - Y[i] * s_inv[i % NOUT];
            l += (double)(r * r);
        }
    }
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) l += __shfl_xor_sync(0xffffffffu, l, d);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < LOSS_THREADS / 32; w++) t += s_part[w];
        atomicAdd(loss_acc + blockIdx.y, t);
    }
}

// column sums of a [rows x N] bf16 matrix into g (FP32, accumulate); member
// blockIdx.z at X + z x_ms, g + z g_ms
__global__ void k_colsum(const __nv_bfloat16 *__restrict__ X, long rows, int N, float *g, long x_ms, long g_ms) {
    X += blockIdx.z * x_ms;
    g += blockIdx.z * g_ms;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const long r0 = (long)blockIdx.y * 2048, r1 = min(rows, r0 + 2048);
    float s = 0.0f;
    for (long r = r0; r < r1; r++) s += __bfloat162float(X[r * N + n]);
    atomicAdd(&g[n], s);
}

// AdamW on the master weights, then the BF16 copies W (K x N) and W^T (N x K)
__global__ void k_adamw(float *theta, const float *__restrict__ grad, float *m, float *v, int n, float lr, float wd,
                        float b1, float b2, float bc1, float bc2, float eps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = grad[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / bc1, vh = vi / bc2;
    theta[i] -= lr * (mh / (sqrtf(vh) + eps) + wd * theta[i]);
}

__global__ void k_cast_weights(const float *__restrict__ theta, __nv_bfloat16 *W, __nv_bfloat16 *Wt, int off, int K,
                               int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K * N) return;
    const int k = i / N, nn = i % N;
    const __nv_bfloat16 b = __float2bfloat16(theta[off + i]);
    W[i] = b;
    Wt[(size_t)nn * K + k] = b;
}

// ensemble statistics of one increment: mean over members and relative spread
__global__ void k_ensemble(const float *__restrict__ Sm, int n_members, int n, float s_floor, float *mean,
                           float *spread) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float mu[NOUT], var = 0.0f, nrm = 0.0f;
    for (int c = 0; c < NOUT; c++) {
        float s = 0.0f;
        for (int k = 0; k < n_members; k++) s += Sm[((size_t)k * n + i) * NOUT + c];
        mu[c] = s / n_members;
        float q = 0.0f;
        for (int k = 0; k < n_members; k++) {
            const float d = Sm[((size_t)k * n + i) * NOUT + c] - mu[c];
            q += d * d;
        }
        var += n_members > 1 ? q / (n_members - 1) : 0.0f;
        nrm += mu[c] * mu[c];
        mean[(size_t)i * NOUT + c] = mu[c];
    }
    spread[i] = sqrtf(var) / fmaxf(sqrtf(nrm), s_floor);
}

__global__ void k_h_to_input(const float *__restrict__ h, int n, __nv_bfloat16 *Z) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * NH) return;
    const int b = idx / NH, k = idx % NH;
    Z[(size_t)b * K0 + NIN + k] = __float2bfloat16(h[idx]);
}

// surrogate input of one increment: u = (F - F_prev (row-major, 9), E = (F^T F - I)/2 in
// Voigt order xx yy zz xy xz yz (6))
__global__ void k_features(const double *__restrict__ Fp, const double *__restrict__ F, int n, float *u) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *f = F + 9 * i, *fp = Fp + 9 * i;
    float *o = u + (size_t)i * NIN;
    for (int k = 0; k < 9; k++) o[k] = (float)(f[k] - fp[k]);
    double C[9];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) C[3 * a + b] = f[a] * f[b] + f[3 + a] * f[3 + b] + f[6 + a] * f[6 + b];
    o[9] = (float)(0.5 * (C[0] - 1.0));
    o[10] = (float)(0.5 * (C[4] - 1.0));
    o[11] = (float)(0.5 * (C[8] - 1.0));
    o[12] = (float)(0.5 * C[1]);
    o[13] = (float)(0.5 * C[2]);
    o[14] = (float)(0.5 * C[5]);
}

inline int cdiv(long a, int b) { return (int)((a + b - 1) / b); }

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct SurMember {
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *W[4] = {nullptr}, *Wt[4] = {nullptr};
    unsigned char *Wp = nullptr;  // weight chunks in the layout of the fused forward's shared buffers
    unsigned char *Wb = nullptr;  // the same for the fused backward (W4, W3, W2, W1)
    int step = 0;
};

struct sur_ctx {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int K = 0, Bmax = 0, Tmax = 0;
    // 2: whole-forward tcgen05 kernel + tcgen05 data-gradient GEMMs (the default), 1: tcgen05 GEMM
    // per layer and step, 0: mma.sync GEMMs
    int backend = 2;
    int *d_err = nullptr;
    std::vector<SurMember> mem;
    std::vector<void *> allocs;
    float *u_inv = nullptr, *s_inv = nullptr, *s_mul = nullptr;
    float h_u_scale[NIN], h_s_scale[NOUT];
    // activations (T x B rows), one slice per member (member strides zs, ys, os, dzs
    // elements), so that the members train side by side
    __nv_bfloat16 *Z = nullptr, *Y1 = nullptr, *A1 = nullptr, *Y2 = nullptr, *A2 = nullptr, *Y3 = nullptr,
                  *A3 = nullptr, *dO = nullptr, *dY3 = nullptr, *dY2 = nullptr, *dY1 = nullptr;
    long zs = 0, ys = 0, os = 0, dzs = 0;
    float *S = nullptr, *dZ = nullptr, *Sm = nullptr;
    double *loss_acc = nullptr;  // one per member
    // parameters of all members, member after member (the SurMember pointers point into these)
    float *theta_all = nullptr, *grad_all = nullptr, *m_all = nullptr, *v_all = nullptr;
    __nv_bfloat16 *W_all[4] = {nullptr}, *Wt_all[4] = {nullptr};
    unsigned char *Wp_all = nullptr, *Wb_all = nullptr;
};

namespace {
const int KDIM[4] = {K0, WID, WID, WID}, NDIM[4] = {WID, WID, WID, N4};
const int WOFF[4] = {OFF_W1, OFF_W2, OFF_W3, OFF_W4}, BOFF[4] = {OFF_B1, OFF_B2, OFF_B3, OFF_B4};

template <class T>
cudaError_t salloc(sur_ctx *s, T **p, size_t n) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    s->allocs.push_back(q);
    *p = static_cast<T *>(q);
    return cudaMemsetAsync(q, 0, std::max<size_t>(n, 1) * sizeof(T), s->stream);
}

void cast_member(sur_ctx *s, SurMember &M) {
    for (int l = 0; l < 4; l++)
        k_cast_weights<<<cdiv((long)KDIM[l] * NDIM[l], 256), 256, 0, s->stream>>>(M.theta, M.W[l], M.Wt[l], WOFF[l],
                                                                                  KDIM[l], NDIM[l]);
    const int units = WS_WP_BYTES / 16;
    k_pack_weights<<<cdiv(units, 256), 256, 0, s->stream>>>(M.Wt[0], M.Wt[1], M.Wt[2], M.Wt[3], M.Wp);
    // the backward products use W4 [256 x 144], W3, W2 and W1 [144 x 256] as the
    // forward uses W1^T [256 x 144], W2^T, W3^T and W4^T [144 x 256]
    k_pack_weights<<<cdiv(units, 256), 256, 0, s->stream>>>(M.W[3], M.W[2], M.W[1], M.W[0], M.Wb);
}

// forward through T steps for member M; stress predictions into S (B x T x 6)
// Whole-forward kernel for members k0 .. k0 + nk - 1 (see k_forward_ws).
void forward_fused(sur_ctx *s, int k0, int nk, const float *U, int B, int T, float *S, long s_mstride, int s_ld,
                   const float *s_mul, float *h, long h_mstride, bool tape) {
    for (int g = 0; g < nk; g += FT_MAXK) {
        const int ng = std::min(FT_MAXK, nk - g);
        FusedArgs a{};
        a.U = U;
        a.B = B;
        a.T = T;
        a.u_inv = s->u_inv;
        a.s_mul = s_mul;
        a.S = S + (size_t)g * s_mstride;
        a.s_mstride = s_mstride;
        a.s_ld = s_ld;
        a.h = h ? h + (size_t)g * h_mstride : nullptr;
        a.h_mstride = h_mstride;
        if (tape) {  // the members' own tape slices
            const long k = k0 + g;
            a.tZ = s->Z + k * s->zs;
            a.tY[0] = s->Y1 + k * s->ys;
            a.tY[1] = s->Y2 + k * s->ys;
            a.tY[2] = s->Y3 + k * s->ys;
            a.tA[0] = s->A1 + k * s->ys;
            a.tA[1] = s->A2 + k * s->ys;
            a.tA[2] = s->A3 + k * s->ys;
            a.tz_ms = s->zs;
            a.ty_ms = s->ys;
        }
        for (int i = 0; i < ng; i++) {
            a.theta[i] = s->mem[k0 + g + i].theta;
            a.Wp[i] = s->mem[k0 + g + i].Wp;
        }
        a.err = s->d_err;
        dim3 grid(cdiv(B, FT_M), ng);
        k_forward_ws<<<grid, WS_THREADS, FT_SMEM, s->stream>>>(a);
    }
}

// forward through T steps for member k, its tape into the member's slice
void forward(sur_ctx *s, int k, const float *U, int B, int T, float *S, const float *s_mul) {
    if (s->backend == 2) {
        forward_fused(s, k, 1, U, B, T, S, 0, T * NOUT, s_mul, nullptr, 0, true);
        return;
    }
    SurMember &M = s->mem[k];
    const size_t RB = (size_t)B;
    __nv_bfloat16 *Zk = s->Z + k * s->zs;
    __nv_bfloat16 *Ys[3] = {s->Y1 + k * s->ys, s->Y2 + k * s->ys, s->Y3 + k * s->ys};
    __nv_bfloat16 *As_[3] = {s->A1 + k * s->ys, s->A2 + k * s->ys, s->A3 + k * s->ys};
    for (int t = 0; t < T; t++) {
        __nv_bfloat16 *Zt = Zk + (size_t)t * RB * K0;
        k_build_input<<<cdiv(RB * K0, 256), 256, 0, s->stream>>>(U, B, T, t, s->u_inv, Zt, t == 0);
        Epi e{};
        e.ld_out = WID;
        const __nv_bfloat16 *in = Zt;
        int kin = K0;
        for (int l = 0; l < 3; l++) {
            e.bias = M.theta + BOFF[l];
            e.y_out = Ys[l] + (size_t)t * RB * WID;
            e.a_out = As_[l] + (size_t)t * RB * WID;
            if (s->backend) gemm_tc05<EPI_GELU>(s->stream, in, kin, M.Wt[l], kin, B, WID, kin, e, s->d_err);
            else gemm<EPI_GELU, false>(s->stream, in, kin, M.W[l], WID, B, WID, kin, e);
            in = e.a_out;
            kin = WID;
        }
        Epi h{};
        h.bias = M.theta + OFF_B4;
        h.s_out = S + (size_t)t * NOUT;
        h.s_ld = T * NOUT;
        h.s_mul = s_mul;  // null during training: the loss works in network units
        h.h_next = (t + 1 < T) ? Zk + (size_t)(t + 1) * RB * K0 : nullptr;
        h.h_f32 = nullptr;
        if (s->backend) gemm_tc05<EPI_HEAD>(s->stream, in, WID, M.Wt[3], WID, B, N4, WID, h, s->d_err);
        else gemm<EPI_HEAD, false>(s->stream, in, WID, M.W[3], N4, B, N4, WID, h);
    }
}

// BPTT for members k0 .. k0 + nk - 1 at once (their tape slices; predictions S
// of member k0 + i at S + i s_ms): gradients into their grad blocks (zeroed
// here), loss partial sums into loss_acc[k0 + i]
void backward_members(sur_ctx *s, int k0, int nk, const float *Y, int B, int T, const float *S, long s_ms,
                      cudaEvent_t mid = nullptr) {
    const size_t RB = (size_t)B;
    cudaMemsetAsync(s->grad_all + (size_t)k0 * NPAR, 0, sizeof(float) * NPAR * nk, s->stream);
    const float gscale = 2.0f / ((float)B * T * NOUT);
    const long ys = s->ys;
    __nv_bfloat16 *Z = s->Z + k0 * s->zs, *dO = s->dO + k0 * s->os;
    __nv_bfloat16 *Y1 = s->Y1 + k0 * ys, *Y2 = s->Y2 + k0 * ys, *Y3 = s->Y3 + k0 * ys;
    __nv_bfloat16 *A1 = s->A1 + k0 * ys, *A2 = s->A2 + k0 * ys, *A3 = s->A3 + k0 * ys;
    __nv_bfloat16 *dY1 = s->dY1 + k0 * ys, *dY2 = s->dY2 + k0 * ys, *dY3 = s->dY3 + k0 * ys;
    float *dZ = s->dZ + k0 * s->dzs;
    const __nv_bfloat16 *W[4], *Wt[4];
    long wms[4];
    for (int l = 0; l < 4; l++) {
        wms[l] = (long)KDIM[l] * NDIM[l];
        W[l] = s->W_all[l] + k0 * wms[l];
        Wt[l] = s->Wt_all[l] + k0 * wms[l];
    }
    const bool tc = s->backend != 0;
    {
        const long n = (long)B * T * NOUT;
        k_loss<<<dim3(cdiv(n, LOSS_THREADS * LOSS_PER_THREAD), nk), LOSS_THREADS, 0, s->stream>>>(S, s_ms, Y, n, s->s_inv,
                                                                                               s->loss_acc + k0);
    }
    if (s->backend == 2) {  // the whole data-gradient chain in one kernel per FT_MAXK members
        for (int g = 0; g < nk; g += FT_MAXK) {
            const int ng = std::min(FT_MAXK, nk - g);
            BwdArgs ba{};
            ba.B = B;
            ba.T = T;
            ba.S = S + g * s_ms;
            ba.s_mstride = s_ms;
            ba.Y = Y;
            ba.s_inv = s->s_inv;
            ba.gscale = gscale;
            ba.Z = Z + g * s->zs;
            ba.Yt[0] = Y1 + g * ys;
            ba.Yt[1] = Y2 + g * ys;
            ba.Yt[2] = Y3 + g * ys;
            ba.dO = dO + g * s->os;
            ba.dY[0] = dY1 + g * ys;
            ba.dY[1] = dY2 + g * ys;
            ba.dY[2] = dY3 + g * ys;
            ba.z_ms = s->zs;
            ba.y_ms = ys;
            ba.o_ms = s->os;
            for (int i = 0; i < ng; i++) ba.Wb[i] = s->mem[k0 + g + i].Wb;
            ba.err = s->d_err;
            k_backward_ws<<<dim3(cdiv(B, FT_M), ng), WS_THREADS, FT_SMEM, s->stream>>>(ba);
        }
    }
    for (int t = T - 1; t >= 0 && s->backend != 2; t--) {
        __nv_bfloat16 *dOt = dO + (size_t)t * RB * N4;
        const __nv_bfloat16 *Hrow = (t + 1 < T) ? Z + (size_t)(t + 1) * RB * K0 : Z;
        k_head_grad<<<dim3(cdiv(RB * N4, 256), nk), 256, 0, s->stream>>>(S, s_ms, Y, B, T, t, s->s_inv, Hrow, s->zs,
                                                                         dZ, s->dzs, t + 1 < T, gscale, dOt, s->os);
        Epi e{};
        e.ld_out = WID;
        e.ld_in = WID;
        e.ms_in = ys;
        e.ms_out = ys;
        // dY3 = (dO W4^T) * gelu'(Y3)
        e.y_in = Y3 + (size_t)t * RB * WID;
        e.a_out = dY3 + (size_t)t * RB * WID;
        if (tc) gemm_tc05<EPI_DGELU>(s->stream, dOt, N4, W[3], N4, B, WID, N4, e, s->d_err, nk, s->os, wms[3]);
        else gemm<EPI_DGELU, false>(s->stream, dOt, N4, Wt[3], WID, B, WID, N4, e, 1, nk, s->os, wms[3]);
        e.y_in = Y2 + (size_t)t * RB * WID;
        e.a_out = dY2 + (size_t)t * RB * WID;
        const __nv_bfloat16 *g3 = dY3 + (size_t)t * RB * WID;
        if (tc) gemm_tc05<EPI_DGELU>(s->stream, g3, WID, W[2], WID, B, WID, WID, e, s->d_err, nk, ys, wms[2]);
        else gemm<EPI_DGELU, false>(s->stream, g3, WID, Wt[2], WID, B, WID, WID, e, 1, nk, ys, wms[2]);
        e.y_in = Y1 + (size_t)t * RB * WID;
        e.a_out = dY1 + (size_t)t * RB * WID;
        const __nv_bfloat16 *g2 = dY2 + (size_t)t * RB * WID;
        if (tc) gemm_tc05<EPI_DGELU>(s->stream, g2, WID, W[1], WID, B, WID, WID, e, s->d_err, nk, ys, wms[1]);
        else gemm<EPI_DGELU, false>(s->stream, g2, WID, Wt[1], WID, B, WID, WID, e, 1, nk, ys, wms[1]);
        if (t > 0) {  // dZ = dY1 W1^T (only the state part is used by step t-1)
            Epi f{};
            f.s_out = dZ;
            f.s_ld = K0;
            f.ms_out = s->dzs;
            const __nv_bfloat16 *g1 = dY1 + (size_t)t * RB * WID;
            if (tc) gemm_tc05<EPI_F32>(s->stream, g1, WID, W[0], WID, B, K0, WID, f, s->d_err, nk, ys, wms[0]);
            else gemm<EPI_F32, false>(s->stream, g1, WID, Wt[0], K0, B, K0, WID, f, 1, nk, ys, wms[0]);
        }
    }
    if (mid) cudaEventRecord(mid, s->stream);  // data gradients done
    // weight gradients over all steps at once: dW = op(A_all)^T dY_all (split-K)
    const long rows = (long)T * B;
    const int split = (int)std::min<long>(16, std::max<long>(1, rows / 4096));
    const __nv_bfloat16 *Ain[4] = {Z, A1, A2, A3};
    const long ams[4] = {s->zs, ys, ys, ys};
    const __nv_bfloat16 *dOut[4] = {dY1, dY2, dY3, dO};
    const long dms[4] = {ys, ys, ys, s->os};
    float *grad = s->grad_all + (size_t)k0 * NPAR;
    for (int l = 0; l < 4; l++) {
        if (tc) {  // weights and biases in one pass
            wgrad_tc05(s->stream, Ain[l], ams[l], KDIM[l], dOut[l], dms[l], NDIM[l], rows, grad + WOFF[l],
                       grad + BOFF[l], NPAR, nk, s->d_err);
            continue;
        } else {
            Epi w{};
            w.s_out = grad + WOFF[l];
            w.s_ld = NDIM[l];
            w.ms_out = NPAR;
            gemm<EPI_WGRAD, true>(s->stream, Ain[l], KDIM[l], dOut[l], NDIM[l], KDIM[l], NDIM[l], (int)rows, w, split,
                                  nk, ams[l], dms[l]);
        }
        dim3 g(cdiv(NDIM[l], 128), cdiv(rows, 2048), nk);
        k_colsum<<<g, 128, 0, s->stream>>>(dOut[l], rows, NDIM[l], grad + BOFF[l], dms[l], NPAR);
    }
}

int init_member(sur_ctx *s, SurMember &M, uint64_t seed) {
    // seeded uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights from a splitmix64
    // stream, zero biases and zero padding rows / columns
    std::vector<float> th(NPAR, 0.0f);
    uint64_t x = seed * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    auto next = [&]() {
        x += 0x9E3779B97F4A7C15ull;
        uint64_t z = x;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    for (int l = 0; l < 4; l++) {
        const double lim = 1.0 / std::sqrt((double)KDIM[l]);
        for (int k = 0; k < KDIM[l]; k++)
            for (int n = 0; n < NDIM[l]; n++) {
                float w = (float)((2.0 * next() - 1.0) * lim);
                if (l == 0 && k >= NIN + NH) w = 0.0f;
                if (l == 3 && n >= NOUT + NH) w = 0.0f;
                th[WOFF[l] + (size_t)k * NDIM[l] + n] = w;
            }
    }
    if (cudaMemcpyAsync(M.theta, th.data(), sizeof(float) * NPAR, cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
        return RC_ECUDA;
    cudaMemsetAsync(M.m, 0, sizeof(float) * NPAR, s->stream);
    cudaMemsetAsync(M.v, 0, sizeof(float) * NPAR, s->stream);
    M.step = 0;
    cast_member(s, M);
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? RC_OK : RC_ECUDA;
}

}  // namespace

extern "C" {

int sur_create(int n_members, int max_batch, int max_steps, uint64_t seed, void *stream, sur_ctx **out) {
    if (!out || n_members <= 0 || max_batch <= 0 || max_steps <= 0) return RC_EINVAL;
    *out = nullptr;
    sur_ctx *s = new sur_ctx();
    s->K = n_members;
    s->Bmax = max_batch;
    s->Tmax = max_steps;
    if (stream) s->stream = (cudaStream_t)stream;
    else if (cudaStreamCreate(&s->stream) != cudaSuccess) { delete s; return RC_ECUDA; }
    else s->own_stream = true;
    const size_t R = (size_t)max_batch * max_steps, Kn = (size_t)n_members;
    s->zs = (long)(R * K0 + (size_t)max_batch * K0);
    s->ys = (long)(R * WID);
    s->os = (long)(R * N4);
    s->dzs = (long)max_batch * K0;
    bool ok = true;
    ok &= salloc(s, &s->u_inv, NIN) == cudaSuccess;
    ok &= salloc(s, &s->s_inv, NOUT) == cudaSuccess;
    ok &= salloc(s, &s->s_mul, NOUT) == cudaSuccess;
    ok &= salloc(s, &s->Z, Kn * s->zs) == cudaSuccess;
    for (__nv_bfloat16 **p : {&s->Y1, &s->A1, &s->Y2, &s->A2, &s->Y3, &s->A3, &s->dY3, &s->dY2, &s->dY1})
        ok &= salloc(s, p, Kn * s->ys) == cudaSuccess;
    ok &= salloc(s, &s->dO, Kn * s->os) == cudaSuccess;
    ok &= salloc(s, &s->S, R * NOUT * Kn) == cudaSuccess;
    ok &= salloc(s, &s->Sm, (size_t)max_batch * NOUT * Kn) == cudaSuccess;
    ok &= salloc(s, &s->dZ, Kn * s->dzs) == cudaSuccess;
    ok &= salloc(s, &s->loss_acc, Kn) == cudaSuccess;
    ok &= salloc(s, &s->d_err, 1) == cudaSuccess;
    ok &= salloc(s, &s->theta_all, Kn * NPAR) == cudaSuccess;
    ok &= salloc(s, &s->grad_all, Kn * NPAR) == cudaSuccess;
    ok &= salloc(s, &s->m_all, Kn * NPAR) == cudaSuccess;
    ok &= salloc(s, &s->v_all, Kn * NPAR) == cudaSuccess;
    for (int l = 0; l < 4; l++) {
        ok &= salloc(s, &s->W_all[l], Kn * KDIM[l] * NDIM[l]) == cudaSuccess;
        ok &= salloc(s, &s->Wt_all[l], Kn * KDIM[l] * NDIM[l]) == cudaSuccess;
    }
    ok &= salloc(s, &s->Wp_all, Kn * WS_WP_BYTES) == cudaSuccess;
    ok &= salloc(s, &s->Wb_all, Kn * WS_WP_BYTES) == cudaSuccess;
    if (!ok) { sur_destroy(s); return RC_ENOMEM; }
    prepare_tc05();
    prepare_ws();
    s->mem.resize(n_members);
    for (size_t k = 0; k < Kn; k++) {
        SurMember &M = s->mem[k];
        M.theta = s->theta_all + k * NPAR;
        M.grad = s->grad_all + k * NPAR;
        M.m = s->m_all + k * NPAR;
        M.v = s->v_all + k * NPAR;
        for (int l = 0; l < 4; l++) {
            M.W[l] = s->W_all[l] + k * KDIM[l] * NDIM[l];
            M.Wt[l] = s->Wt_all[l] + k * KDIM[l] * NDIM[l];
        }
        M.Wp = s->Wp_all + k * WS_WP_BYTES;
        M.Wb = s->Wb_all + k * WS_WP_BYTES;
    }
    float one[NIN];
    for (int k = 0; k < NIN; k++) one[k] = 1.0f;
    if (sur_set_scaling(s, one, one) != RC_OK) { sur_destroy(s); return RC_ECUDA; }
    for (int k = 0; k < n_members; k++)
        if (init_member(s, s->mem[k], seed + (uint64_t)k) != RC_OK) { sur_destroy(s); return RC_ECUDA; }
    *out = s;
    return RC_OK;
}

int sur_set_scaling(sur_ctx *s, const float *u_scale, const float *s_scale) {
    if (!s || !u_scale || !s_scale) return RC_EINVAL;
    float ui[NIN], si[NOUT], sm[NOUT];
    for (int k = 0; k < NIN; k++) {
        if (!(u_scale[k] > 0)) return RC_EINVAL;
        ui[k] = 1.0f / u_scale[k];
        s->h_u_scale[k] = u_scale[k];
    }
    for (int k = 0; k < NOUT; k++) {
        if (!(s_scale[k] > 0)) return RC_EINVAL;
        si[k] = 1.0f / s_scale[k];
        sm[k] = s_scale[k];
        s->h_s_scale[k] = s_scale[k];
    }
    cudaMemcpyAsync(s->u_inv, ui, sizeof ui, cudaMemcpyHostToDevice, s->stream);
    cudaMemcpyAsync(s->s_inv, si, sizeof si, cudaMemcpyHostToDevice, s->stream);
    cudaMemcpyAsync(s->s_mul, sm, sizeof sm, cudaMemcpyHostToDevice, s->stream);
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? RC_OK : RC_ECUDA;
}

int sur_get_params(sur_ctx *s, int member, float *theta) {
    if (!s || !theta || member < 0 || member >= s->K) return RC_EINVAL;
    if (cudaMemcpyAsync(theta, s->mem[member].theta, sizeof(float) * NPAR, cudaMemcpyDeviceToHost, s->stream) !=
        cudaSuccess)
        return RC_ECUDA;
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? RC_OK : RC_ECUDA;
}

int sur_set_params(sur_ctx *s, int member, const float *theta) {
    if (!s || !theta || member < 0 || member >= s->K) return RC_EINVAL;
    SurMember &M = s->mem[member];
    if (cudaMemcpyAsync(M.theta, theta, sizeof(float) * NPAR, cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
        return RC_ECUDA;
    cudaMemsetAsync(M.m, 0, sizeof(float) * NPAR, s->stream);
    cudaMemsetAsync(M.v, 0, sizeof(float) * NPAR, s->stream);
    M.step = 0;
    cast_member(s, M);
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? RC_OK : RC_ECUDA;
}

static int check_batch(sur_ctx *s, int B, int T) {
    if (B <= 0 || T <= 0 || B > s->Bmax || T > s->Tmax) return RC_EINVAL;
    return RC_OK;
}

int sur_loss_grad(sur_ctx *s, int member, const float *U, const float *Y, int B, int T, double *loss, float *grad) {
    if (!s || !U || !Y || member < 0 || member >= s->K) return RC_EINVAL;
    if (check_batch(s, B, T) != RC_OK) return RC_EINVAL;
    SurMember &M = s->mem[member];
    float *Sk = s->S + (size_t)member * B * T * NOUT;
    cudaMemsetAsync(s->loss_acc + member, 0, sizeof(double), s->stream);
    forward(s, member, U, B, T, Sk, nullptr);
    backward_members(s, member, 1, Y, B, T, Sk, 0);
    double l = 0.0;
    cudaMemcpyAsync(&l, s->loss_acc + member, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (grad) cudaMemcpyAsync(grad, M.grad, sizeof(float) * NPAR, cudaMemcpyDeviceToHost, s->stream);
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return RC_ECUDA;
    if (loss) *loss = l / ((double)B * T * NOUT);
    return cudaGetLastError() == cudaSuccess ? RC_OK : RC_ECUDA;
}

int sur_train_step(sur_ctx *s, const float *U, const float *Y, int B, int T, float lr, float wd, double *loss) {
    if (!s || !U || !Y) return RC_EINVAL;
    if (check_batch(s, B, T) != RC_OK) return RC_EINVAL;
    const long s_ms = (long)B * T * NOUT;
    cudaMemsetAsync(s->loss_acc, 0, sizeof(double) * s->K, s->stream);
    if (s->backend == 2) {  // every member at once: one fused forward, member-batched backward launches
        forward_fused(s, 0, s->K, U, B, T, s->S, s_ms, T * NOUT, nullptr, nullptr, 0, true);
        backward_members(s, 0, s->K, Y, B, T, s->S, s_ms);
    } else {
        for (int k = 0; k < s->K; k++) {
            forward(s, k, U, B, T, s->S + k * s_ms, nullptr);
            backward_members(s, k, 1, Y, B, T, s->S + k * s_ms, 0);
        }
    }
    for (int k = 0; k < s->K; k++) {
        SurMember &M = s->mem[k];
        M.step++;
        const float b1 = 0.9f, b2 = 0.999f;
        const float bc1 = 1.0f - std::pow(b1, (float)M.step), bc2 = 1.0f - std::pow(b2, (float)M.step);
        k_adamw<<<cdiv(NPAR, 256), 256, 0, s->stream>>>(M.theta, M.grad, M.m, M.v, NPAR, lr, wd, b1, b2, bc1, bc2,
                                                        1e-8f);
        cast_member(s, M);
    }
    if (loss) {
        std::vector<double> l(s->K, 0.0);
        cudaMemcpyAsync(l.data(), s->loss_acc, sizeof(double) * s->K, cudaMemcpyDeviceToHost, s->stream);
        if (cudaStreamSynchronize(s->stream) != cudaSuccess) return RC_ECUDA;
        for (int k = 0; k < s->K; k++) loss[k] = l[k] / ((double)B * T * NOUT);
    }
    return cudaGetLastError() == cudaSuccess ? RC_OK : RC_ECUDA;
}

int sur_profile_step(sur_ctx *s, const float *U, const float *Y, int B, int T, double *ms_out) {
    if (!s || !U || !Y || !ms_out) return RC_EINVAL;
    if (check_batch(s, B, T) != RC_OK) return RC_EINVAL;
    const long s_ms = (long)B * T * NOUT;
    cudaEvent_t ev[4];
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) return RC_ECUDA;
    cudaMemsetAsync(s->loss_acc, 0, sizeof(double) * s->K, s->stream);
    cudaEventRecord(ev[0], s->stream);
    if (s->backend == 2) {
        forward_fused(s, 0, s->K, U, B, T, s->S, s_ms, T * NOUT, nullptr, nullptr, 0, true);
        cudaEventRecord(ev[1], s->stream);
        backward_members(s, 0, s->K, Y, B, T, s->S, s_ms, ev[2]);
    } else {  // per member: the phases summed over the members
        for (int k = 0; k < s->K; k++) forward(s, k, U, B, T, s->S + k * s_ms, nullptr);
        cudaEventRecord(ev[1], s->stream);
        for (int k = 0; k < s->K; k++) backward_members(s, k, 1, Y, B, T, s->S + k * s_ms, 0);
        cudaEventRecord(ev[2], s->stream);
    }
    cudaEventRecord(ev[3], s->stream);
    int rc = cudaEventSynchronize(ev[3]) == cudaSuccess ? RC_OK : RC_ECUDA;
    float t[3] = {0.f, 0.f, 0.f};
    for (int i = 0; i < 3 && rc == RC_OK; i++)
        if (cudaEventElapsedTime(&t[i], ev[i], ev[i + 1]) != cudaSuccess) rc = RC_ECUDA;
    for (int i = 0; i < 3; i++) ms_out[i] = t[i];
    for (auto &e : ev) cudaEventDestroy(e);
    return rc == RC_OK && cudaGetLastError() == cudaSuccess ? RC_OK : RC_ECUDA;
}

int sur_predict(sur_ctx *s, const float *U, int B, int T, float *Sout) {
    if (!s || !U || !Sout) return RC_EINVAL;
    if (check_batch(s, B, T) != RC_OK) return RC_EINVAL;
    if (s->backend == 2) {
        forward_fused(s, 0, s->K, U, B, T, Sout, (long)B * T * NOUT, T * NOUT, s->s_mul, nullptr, 0, false);
        return cudaGetLastError() == cudaSuccess ? RC_OK : RC_ECUDA;
    }
    for (int k = 0; k < s->K; k++) forward(s, k, U, B, T, Sout + (size_t)k * B * T * NOUT, s->s_mul);
    return cudaGetLastError() == cudaSuccess ? RC_OK : RC_ECUDA;
}

int sur_step(sur_ctx *s, const float *u, int n, float *h, float s_floor, float *s_mean, float *spread) {
    if (!s || !u || !h || !s_mean || !spread || n <= 0 || n > s->Bmax) return RC_EINVAL;
    if (s->backend == 2) {
        forward_fused(s, 0, s->K, u, n, 1, s->Sm, (long)n * NOUT, NOUT, s->s_mul, h, (long)n * NH, false);
        k_ensemble<<<cdiv(n, 128), 128, 0, s->stream>>>(s->Sm, s->K, n, s_floor, s_mean, spread);
        return cudaGetLastError() == cudaSuccess ? RC_OK : RC_ECUDA;
    }
    __nv_bfloat16 *Z = s->Z;  // n rows of [u, h, 0]
    __nv_bfloat16 *Ys[3] = {s->Y1, s->Y2, s->Y3}, *As_[3] = {s->A1, s->A2, s->A3};
    for (int k = 0; k < s->K; k++) {
        SurMember &M = s->mem[k];
        float *hk = h + (size_t)k * n * NH;
        k_build_input<<<cdiv((long)n * K0, 256), 256, 0, s->stream>>>(u, n, 1, 0, s->u_inv, Z, 0);
        k_h_to_input<<<cdiv((long)n * NH, 256), 256, 0, s->stream>>>(hk, n, Z);
        const __nv_bfloat16 *in = Z;
        int kin = K0;
        for (int l = 0; l < 3; l++) {
            Epi e{};
            e.ld_out = WID;
            e.bias = M.theta + BOFF[l];
            e.y_out = Ys[l];
            e.a_out = As_[l];
            if (s->backend) gemm_tc05<EPI_GELU>(s->stream, in, kin, M.Wt[l], kin, n, WID, kin, e, s->d_err);
            else gemm<EPI_GELU, false>(s->stream, in, kin, M.W[l], WID, n, WID, kin, e);
            in = As_[l];
            kin = WID;
        }
        Epi hd{};
        hd.bias = M.theta + OFF_B4;
        hd.s_out = s->Sm + (size_t)k * n * NOUT;
        hd.s_ld = NOUT;
        hd.s_mul = s->s_mul;
        hd.h_next = nullptr;
        hd.h_f32 = hk;  // the new state replaces the old one (the input row holds a BF16 copy)
        if (s->backend) gemm_tc05<EPI_HEAD>(s->stream, in, WID, M.Wt[3], WID, n, N4, WID, hd, s->d_err);
        else gemm<EPI_HEAD, false>(s->stream, in, WID, M.W[3], N4, n, N4, WID, hd);
    }
    k_ensemble<<<cdiv(n, 128), 128, 0, s->stream>>>(s->Sm, s->K, n, s_floor, s_mean, spread);
    return cudaGetLastError() == cudaSuccess ? RC_OK : RC_ECUDA;
}

int sur_set_backend(sur_ctx *s, int backend) {
    if (!s || backend < 0 || backend > 2) return RC_EINVAL;
    s->backend = backend;
    return RC_OK;
}

int sur_sync(sur_ctx *s) {
    if (!s) return RC_EINVAL;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return RC_ECUDA;
    int e = 0;
    if (cudaMemcpy(&e, s->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return RC_ECUDA;
    return e;
}

int sur_features(const double *F_prev, const double *F, int n, float *u, void *stream) {
    if (!F_prev || !F || !u || n <= 0) return RC_EINVAL;
    k_features<<<cdiv(n, 128), 128, 0, (cudaStream_t)stream>>>(F_prev, F, n, u);
    return cudaGetLastError() == cudaSuccess ? RC_OK : RC_ECUDA;
}

int sur_info(const sur_ctx *s, int *n_members, void **stream) {
    if (!s) return RC_EINVAL;
    if (n_members) *n_members = s->K;
    if (stream) *stream = (void *)s->stream;
    return RC_OK;
}

void sur_destroy(sur_ctx *s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (void *p : s->allocs) cudaFree(p);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
