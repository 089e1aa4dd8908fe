// FP64 coupling kernels (Sec. 2.1): QR split of F, the MD box R H(0), the
// incremental stretch Delta R = R(t) R(t-1)^{-1} (Eq. LAMMPS2) and the affine
// remap of the atoms; the time-averaged stress, its rotation back to the FE
// frame (sigma_FEM = Q sigma_MD Q^T) and the first Piola-Kirchhoff stress
// P = J sigma_FEM F^{-T} (Eq. Pmd).  All tiny: one thread (or one warp) per cell.
#include "rc_internal.cuh"

namespace {

__device__ __forceinline__ double det3(const double *A) {
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) + A[2] * (A[3] * A[7] - A[4] * A[6]);
}

// one thread per cell
__global__ void k_deform(const double *__restrict__ Fin, double *H, double *Rprev, double *Qo, double *Ro,
                         double *Fst, double *dR, const double *__restrict__ H0, float *Hf, float *Hif, int *status,
                         int *need_rebuild, int *nbins, const int *bin_cap, const int *active, double rlist,
                         int n_cells) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    double *dRc = dR + 9 * c;
    for (int k = 0; k < 9; k++) dRc[k] = (k % 4 == 0) ? 1.0 : 0.0;  // identity unless the cell is updated
    if (status[c] != 0 || !active[c]) return;  // inactive cells keep box, R(t-1) and atoms
    double F[9];
    for (int k = 0; k < 9; k++) F[k] = Fin[9 * c + k];
    if (!(det3(F) > 0.0)) {
        atomicCAS(&status[c], 0, RC_EDEGEN);
        return;
    }
    // modified Gram-Schmidt on the columns a_0, a_1, a_2 of F (Sec. 2.1); the
    // norms make the diagonal of R positive.
    double q[3][3], R[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int j = 0; j < 3; j++) {
        double v0 = F[j], v1 = F[3 + j], v2 = F[6 + j];
        for (int i = 0; i < j; i++) {
            const double r = q[i][0] * v0 + q[i][1] * v1 + q[i][2] * v2;
            R[3 * i + j] = r;
            v0 -= r * q[i][0];
            v1 -= r * q[i][1];
            v2 -= r * q[i][2];
        }
        const double nrm = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
        if (!(nrm > 0.0)) {
            atomicCAS(&status[c], 0, RC_EDEGEN);
            return;
        }
        R[3 * j + j] = nrm;
        q[j][0] = v0 / nrm;
        q[j][1] = v1 / nrm;
        q[j][2] = v2 / nrm;
    }
    // new box H = R H0 (both upper triangular)
    const double *h0 = H0 + 9 * c;
    double Hn[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < 3; i++)
        for (int j = i; j < 3; j++) {
            double s = 0.0;
            for (int k = i; k <= j; k++) s += R[3 * i + k] * h0[3 * k + j];
            Hn[3 * i + j] = s;
        }
    // the MD box is held FP32-exact (positions are FP32): round it once here and
    // use the rounded box everywhere (shifts, bins, volume)
    for (int k = 0; k < 9; k++) Hn[k] = (double)(float)Hn[k];
    // perpendicular widths of an upper-triangular box [[a b c][0 d e][0 0 f]]:
    // w_d = 1 / |row d of H^{-1}|
    const double a = Hn[0], b = Hn[1], cc = Hn[2], d = Hn[4], e = Hn[5], f = Hn[8];
    const double i00 = 1.0 / a, i01 = -b / (a * d), i02 = (b * e - cc * d) / (a * d * f);
    const double i11 = 1.0 / d, i12 = -e / (d * f), i22 = 1.0 / f;
    const double w[3] = {1.0 / sqrt(i00 * i00 + i01 * i01 + i02 * i02), 1.0 / sqrt(i11 * i11 + i12 * i12),
                         1.0 / fabs(i22)};
    for (int k = 0; k < 3; k++)
        if (!(w[k] >= 2.0 * rlist)) {
            atomicCAS(&status[c], 0, RC_EBOX);
            return;
        }
    int nb[3];
    for (int k = 0; k < 3; k++) nb[k] = (int)floor(2.0 * w[k] / rlist);  // bins at least r_list / 2 wide
    while (nb[0] * nb[1] * nb[2] > bin_cap[c]) {
        int m = nb[0] >= nb[1] ? (nb[0] >= nb[2] ? 0 : 2) : (nb[1] >= nb[2] ? 1 : 2);
        nb[m]--;
    }
    // Delta R = R_new R_prev^{-1}; R_prev upper triangular: back substitution per column
    double *Rp = Rprev + 9 * c;
    double Rpi[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int j = 0; j < 3; j++) {
        for (int i = j; i >= 0; i--) {
            double s = (i == j) ? 1.0 : 0.0;
            for (int k = i + 1; k <= j; k++) s -= Rp[3 * i + k] * Rpi[3 * k + j];
            Rpi[3 * i + j] = s / Rp[3 * i + i];
        }
    }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += R[3 * i + k] * Rpi[3 * k + j];
            dRc[3 * i + j] = s;
        }
    for (int k = 0; k < 9; k++) {
        Rp[k] = R[k];
        Ro[9 * c + k] = R[k];
        Fst[9 * c + k] = F[k];
        H[9 * c + k] = Hn[k];
    }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) Qo[9 * c + 3 * i + j] = q[j][i];  // Q columns are q_j
    float *hf = Hf + 8 * c, *hif = Hif + 8 * c;
    hf[0] = (float)a; hf[1] = (float)b; hf[2] = (float)cc; hf[3] = (float)d; hf[4] = (float)e; hf[5] = (float)f;
    hif[0] = (float)i00; hif[1] = (float)i01; hif[2] = (float)i02;
    hif[3] = (float)i11; hif[4] = (float)i12; hif[5] = (float)i22;
    nbins[4 * c] = nb[0];
    nbins[4 * c + 1] = nb[1];
    nbins[4 * c + 2] = nb[2];
    need_rebuild[c] = 1;
}

// x <- Delta R x (FP64 arithmetic on the FP32 positions); one thread per atom slot
__global__ void k_remap(KArrays a, const double *__restrict__ dR, int cur) {
    const int t = blockIdx.x;
    const int c = a.tile_cell[t];
    if (a.status[c] != 0 || !a.active[c]) return;
    const int li = (t - a.cell_tile0[c]) * RC_TILE + threadIdx.x;
    if (li >= a.cell_n[c]) return;
    const int g = a.cell_off[c] + li;
    const double *m = dR + 9 * c;
    float4 *X = cur ? a.x1 : a.x0;
    const float4 x = X[g];
    const double x0 = x.x, x1 = x.y, x2 = x.z;
    X[g] = make_float4((float)(m[0] * x0 + m[1] * x1 + m[2] * x2), (float)(m[3] * x0 + m[4] * x1 + m[5] * x2),
                       (float)(m[6] * x0 + m[7] * x1 + m[8] * x2), 0.0f);
}

// sigma_MD(t) = -(K + W) * pconv / det H from one sample record (K[6], W[6], pe, ke)
__device__ __forceinline__ void sample_md(const double *rec, double scale, double *S /* 9 */) {
    const int vi[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    for (int k = 0; k < 6; k++) {
        const double s = -(rec[k] + rec[6 + k]) * scale;
        S[3 * vi[k][0] + vi[k][1]] = s;
        S[3 * vi[k][1] + vi[k][0]] = s;
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

// One CTA per cell.  Phase 1: every sample rotated to the FE frame
// (Q sigma_MD Q^T) into `rot` (n_avg x 6).  Phase 2: warp k < 6 takes component
// k: mean and the blocking standard error (level l: floor(n/2^l) block means;
// largest SE over levels with >= 16 blocks, level 0 always).  Phase 3: P.
constexpr int STRESS_THREADS = 256;
__global__ void __launch_bounds__(STRESS_THREADS) k_stress(const double *__restrict__ series, int n_avg, int cap,
                         const double *__restrict__ H, const double *__restrict__ Qall,
                         const double *__restrict__ Fall, double pconv, double *rot_all, double *sig_fem,
                         double *sig_se, double *sig_md, double *P) {
    const int c = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ double s_md[STRESS_THREADS / 32][6];
    __shared__ double s_mean[6];
    const double *Hc = H + 9 * c, *Q = Qall + 9 * c;
    const double scale = pconv / (Hc[0] * Hc[4] * Hc[8]);
    const double *rec0 = series + (size_t)c * cap * RC_SAMPLE_W;
    double *rot = rot_all + (size_t)c * cap * 6;
    const int vi[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    double md[6] = {0, 0, 0, 0, 0, 0};
    for (int t = tid; t < n_avg; t += STRESS_THREADS) {
        double S[9];
        sample_md(rec0 + (size_t)t * RC_SAMPLE_W, scale, S);
        for (int k = 0; k < 6; k++) {
            const int a = vi[k][0], b = vi[k][1];
            double r = 0.0;
            for (int u = 0; u < 3; u++)
                for (int v = 0; v < 3; v++) r += Q[3 * a + u] * S[3 * u + v] * Q[3 * b + v];
            rot[(size_t)t * 6 + k] = r;
            md[k] += S[3 * a + b];
        }
    }
    for (int k = 0; k < 6; k++) {
        const double w = warp_sum(md[k]);
        if (lane == 0) s_md[warp][k] = w;
    }
    __syncthreads();
    if (warp < 6) {
        const int k = warp;
        double sum = 0.0;
        for (int t = lane; t < n_avg; t += 32) sum += rot[(size_t)t * 6 + k];
        sum = warp_sum(sum);
        const double mean = n_avg > 0 ? sum / n_avg : 0.0;
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
            mb = warp_sum(mb) / nk;
            double v = 0.0;
            for (int b = lane; b < nk; b += 32) {
                double m = 0.0;
                for (int t = 0; t < bs; t++) m += rot[(size_t)(b * bs + t) * 6 + k];
                m /= bs;
                v += (m - mb) * (m - mb);
            }
            v = warp_sum(v);
            const double se = sqrt(v / ((double)nk * (nk - 1)));
            if (se > best) best = se;
        }
        if (lane == 0) {
            double mdsum = 0.0;
            for (int w = 0; w < STRESS_THREADS / 32; w++) mdsum += s_md[w][k];
            sig_fem[6 * c + k] = mean;
            sig_se[6 * c + k] = best;
            sig_md[6 * c + k] = n_avg > 0 ? mdsum / n_avg : 0.0;
            s_mean[k] = mean;
        }
    }
    __syncthreads();
    if (tid == 0) {
        // P = J sigma F^{-T}
        const double *F = Fall + 9 * c;
        const double J = det3(F);
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
                for (int l = 0; l < 3; l++) s += S[3 * i + l] * Fi[3 * j + l];  // (F^{-T})_{lj} = Fi[j][l]
                P[9 * c + 3 * i + j] = J * s;
            }
    }
}

// Cells skipped by a run (activity mask 0) keep their positions in the buffer
// that was current when the run began; after an odd number of steps the other
// buffer is current, so their positions are copied into it.
__global__ void __launch_bounds__(RC_TILE) k_keep_frozen(KArrays a, int cur_new) {
    const int t = blockIdx.x;
    const int c = a.tile_cell[t];
    if (a.active[c]) return;
    const int li = (t - a.cell_tile0[c]) * RC_TILE + threadIdx.x;
    if (li >= a.cell_n[c]) return;
    const int g = a.cell_off[c] + li;
    (cur_new ? a.x1 : a.x0)[g] = (cur_new ? a.x0 : a.x1)[g];
}

__global__ void k_advance(unsigned long long *evals, const int *active, int n_cells, int n) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n_cells && active[c]) evals[c] += (unsigned long long)n;
}

}  // namespace

void rc_launch_deform_impl(const double *F, double *H, double *Rprev, double *Q, double *R, double *Fst, double *dR,
                           const double *H0, float *Hf, float *Hif, int *status, int *need_rebuild, int *nbins,
                           const int *bin_cap, const int *active, double rlist, int n_cells, cudaStream_t s) {
    k_deform<<<(n_cells + 127) / 128, 128, 0, s>>>(F, H, Rprev, Q, R, Fst, dR, H0, Hf, Hif, status, need_rebuild,
                                                   nbins, bin_cap, active, rlist, n_cells);
}

void rc_launch_remap(const KArrays &a, const double *dR, int cur, int n_tiles, cudaStream_t s) {
    k_remap<<<n_tiles, RC_TILE, 0, s>>>(a, dR, cur);
}

void rc_launch_stress(const double *series, int n_avg, int series_cap, const double *H, const double *Q,
                      const double *F, double pconv, double *rot_scratch, double *sig_fem, double *sig_se,
                      double *sig_md, double *P, int n_cells, cudaStream_t s) {
    k_stress<<<n_cells, STRESS_THREADS, 0, s>>>(series, n_avg, series_cap, H, Q, F, pconv, rot_scratch, sig_fem,
                                                sig_se, sig_md, P);
}

void rc_launch_keep_frozen(const KArrays &a, int cur_new, int n_tiles, cudaStream_t s) {
    k_keep_frozen<<<n_tiles, RC_TILE, 0, s>>>(a, cur_new);
}

void rc_launch_advance(unsigned long long *evals, const int *active, int n_cells, int n, cudaStream_t s) {
    k_advance<<<(n_cells + 127) / 128, 128, 0, s>>>(evals, active, n_cells, n);
}
