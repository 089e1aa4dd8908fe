// Molecular statics of the r-cells (Sec. 2.2, Eqs. CGPR1-CGPR3, PK1): energy
// minimisation at fixed box by FIRE (Bitzek, Koskinen, Gaehler, Moseler and
// Gumbsch, Phys. Rev. Lett. 97, 170201, 2006), cell by cell in one batch, and
// the reduction of the pair-sum first Piola-Kirchhoff stress.
//
// One FIRE iteration per cell, with f the forces of the current positions and
// norms over the cell's 3N-vectors: converged when max_i |f_i| < f_tol;
// p = f . v; p > 0: n_pos += 1, v = (1 - alpha) v + alpha |v| f / |f|, and
// after more than 5 such steps dt = min(1.1 dt, dt_max), alpha = 0.99 alpha;
// p <= 0: n_pos = 0, v = 0, dt = dt / 2, alpha = 0.1; then v += dt f / m,
// x += dt v, an atom whose move would exceed dmax (> 0) having its velocity
// scaled to move dmax.  Kernels: k_fire_power (per-cell p, |v|^2, |f|^2, max |f|^2),
// k_fire_control (per cell), k_fire_move (per atom).
#include "rc_internal.cuh"

namespace {

constexpr int FIRE_NMIN = 5;
constexpr float FIRE_FINC = 1.1f, FIRE_FDEC = 0.5f, FIRE_ALPHA0 = 0.1f, FIRE_FALPHA = 0.99f;

__global__ void k_fire_init(FireState s, const int *status, const int *active, int n_cells, float dt0) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    s.dt[c] = dt0;
    s.alpha[c] = FIRE_ALPHA0;
    s.npos[c] = 0;
    s.done[c] = (status[c] != 0 || !active[c]) ? 1 : 0;
    s.moving[c] = 1 - s.done[c];
    s.iters[c] = -1;
    s.it[c] = 0;
    s.mixa[c] = 1.0f;
    s.mixb[c] = 0.0f;
    s.zero[c] = 1;
    s.fmax2[c] = 0u;
    for (int k = 0; k < 4; k++) s.acc[4 * c + k] = 0.0;
}

// velocities to zero: cells still minimising, or (all_cells) every active cell
// without an error
__global__ void __launch_bounds__(RC_TILE) k_fire_zero_v(KArrays a, FireState s, int all_cells) {
    const int t = blockIdx.x, c = a.tile_cell[t];
    const int li = (t - a.cell_tile0[c]) * RC_TILE + threadIdx.x;
    const bool go = all_cells ? (a.active[c] && a.status[c] == 0) : !s.done[c];
    if (li < a.cell_n[c] && go) a.v[a.cell_off[c] + li] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void __launch_bounds__(RC_TILE) k_fire_power(KArrays a, FireState s) {
    const int t = blockIdx.x, c = a.tile_cell[t];
    if (s.done[c]) return;
    const int li = (t - a.cell_tile0[c]) * RC_TILE + threadIdx.x;
    float p = 0.f, vv = 0.f, ff = 0.f, f2max = 0.f;
    if (li < a.cell_n[c]) {
        const int g = a.cell_off[c] + li;
        const float4 f = a.f[g], v = a.v[g];
        p = f.x * v.x + f.y * v.y + f.z * v.z;
        vv = v.x * v.x + v.y * v.y + v.z * v.z;
        ff = f.x * f.x + f.y * f.y + f.z * f.z;
        f2max = ff;
    }
    __shared__ double s_part[RC_TILE / 32][3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
        p += __shfl_xor_sync(0xffffffffu, p, d);
        vv += __shfl_xor_sync(0xffffffffu, vv, d);
        ff += __shfl_xor_sync(0xffffffffu, ff, d);
        f2max = fmaxf(f2max, __shfl_xor_sync(0xffffffffu, f2max, d));
    }
    if (lane == 0) {
        s_part[warp][0] = p;
        s_part[warp][1] = vv;
        s_part[warp][2] = ff;
        atomicMax(&s.fmax2[c], __float_as_uint(f2max));  // non-negative floats order like their bits
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double sum = 0.0;
        for (int w = 0; w < RC_TILE / 32; w++) sum += s_part[w][threadIdx.x];
        atomicAdd(&s.acc[4 * c + threadIdx.x], sum);
    }
}

__global__ void k_fire_control(FireState s, int n_cells, float f_tol2, float dt_max, int *n_left) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells || s.done[c]) return;
    const float f2max = __uint_as_float(s.fmax2[c]);
    const double p = s.acc[4 * c], vv = s.acc[4 * c + 1], ff = s.acc[4 * c + 2];
    s.fmax2[c] = 0u;
    s.acc[4 * c] = s.acc[4 * c + 1] = s.acc[4 * c + 2] = 0.0;
    if (f2max < f_tol2) {
        s.done[c] = 1;
        s.moving[c] = 0;  // the force kernels skip the cell from now on
        s.iters[c] = s.it[c];
        return;
    }
    s.it[c] += 1;
    float alpha = s.alpha[c], dt = s.dt[c];
    if (p > 0.0) {
        const int np = s.npos[c] + 1;
        s.npos[c] = np;
        s.zero[c] = 0;
        s.mixa[c] = 1.0f - alpha;
        s.mixb[c] = ff > 0.0 ? (float)(alpha * sqrt(vv) / sqrt(ff)) : 0.0f;
        if (np > FIRE_NMIN) {
            dt = fminf(FIRE_FINC * dt, dt_max);
            alpha *= FIRE_FALPHA;
        }
    } else {
        s.npos[c] = 0;
        s.zero[c] = 1;
        dt *= FIRE_FDEC;
        alpha = FIRE_ALPHA0;
    }
    s.dt[c] = dt;
    s.alpha[c] = alpha;
    if (n_left) atomicAdd(n_left, 1);
}

__global__ void __launch_bounds__(RC_TILE) k_fire_move(KParams p, KArrays a, int cur, FireState s, float dmax) {
    const int t = blockIdx.x, c = a.tile_cell[t];
    if (s.done[c]) return;
    const int li = (t - a.cell_tile0[c]) * RC_TILE + threadIdx.x;
    if (li >= a.cell_n[c]) return;
    const int g = a.cell_off[c] + li;
    const float4 f = a.f[g];
    float4 v = a.v[g];
    const float mixa = s.mixa[c], mixb = s.mixb[c], dt = s.dt[c];
    if (s.zero[c]) {
        v = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        v.x = fmaf(mixa, v.x, mixb * f.x);
        v.y = fmaf(mixa, v.y, mixb * f.y);
        v.z = fmaf(mixa, v.z, mixb * f.z);
    }
    const float h = dt * p.fm;
    v.x = fmaf(h, f.x, v.x);
    v.y = fmaf(h, f.y, v.y);
    v.z = fmaf(h, f.z, v.z);
    const float s2 = dt * dt * (v.x * v.x + v.y * v.y + v.z * v.z);
    if (dmax > 0.0f && s2 > dmax * dmax) {  // per-atom move cap
        const float sc = dmax * rsqrtf(s2);
        v.x *= sc;
        v.y *= sc;
        v.z *= sc;
    }
    a.v[g] = v;
    float4 *X = cur ? a.x1 : a.x0;
    float4 x = X[g];
    x.x = fmaf(dt, v.x, x.x);
    x.y = fmaf(dt, v.y, x.y);
    x.z = fmaf(dt, v.z, x.z);
    X[g] = x;
    const float4 xr0 = a.xref[g];
    const float ddx = x.x - xr0.x, ddy = x.y - xr0.y, ddz = x.z - xr0.z;
    if (ddx * ddx + ddy * ddy + ddz * ddz > p.skin_half2) a.need_rebuild[c] = 1;
}

// M = H(0) H^{-1} per cell (both upper triangular; FP64, stored as FP32 m00 m01
// m02 m11 m12 m22) and a zeroed accumulator
__global__ void k_static_prep(const double *H, const double *H0, float *mcell, double *acc, int n_cells) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    const double *h = H + 9 * c, *h0 = H0 + 9 * c;
    const double a = h[0], b = h[1], cc = h[2], d = h[4], e = h[5], f = h[8];
    const double i00 = 1.0 / a, i01 = -b / (a * d), i02 = (b * e - cc * d) / (a * d * f);
    const double i11 = 1.0 / d, i12 = -e / (d * f), i22 = 1.0 / f;
    // H0 is diagonal (orthogonal reference box)
    float *m = mcell + 6 * c;
    m[0] = (float)(h0[0] * i00);
    m[1] = (float)(h0[0] * i01);
    m[2] = (float)(h0[0] * i02);
    m[3] = (float)(h0[4] * i11);
    m[4] = (float)(h0[4] * i12);
    m[5] = (float)(h0[8] * i22);
    for (int k = 0; k < 9; k++) acc[9 * c + k] = 0.0;
}

// P_MD = acc pconv / (2 Omega_0); P_FEM = Q P_MD; sigma_FEM = P_FEM F^T / J
// (Voigt xx yy zz xy xz yz, off-diagonals symmetrised)
__global__ void k_static_finish(const double *acc, const double *H0, const double *Q, const double *F, double pconv,
                                double *P, double *sig, const int *status, int n_cells) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    const double *h0 = H0 + 9 * c, *q = Q + 9 * c, *Fc = F + 9 * c;
    const double om0 = h0[0] * h0[4] * h0[8];
    double Pm[9], Pf[9], S[9];
    for (int k = 0; k < 9; k++) Pm[k] = status[c] == 0 ? acc[9 * c + k] * pconv / (2.0 * om0) : 0.0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += q[3 * i + k] * Pm[3 * k + j];
            Pf[3 * i + j] = s;
        }
    const double J = Fc[0] * (Fc[4] * Fc[8] - Fc[5] * Fc[7]) - Fc[1] * (Fc[3] * Fc[8] - Fc[5] * Fc[6]) +
                     Fc[2] * (Fc[3] * Fc[7] - Fc[4] * Fc[6]);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += Pf[3 * i + k] * Fc[3 * j + k];
            S[3 * i + j] = s / J;
        }
    if (P)
        for (int k = 0; k < 9; k++) P[9 * c + k] = Pf[k];
    if (sig) {
        double *o = sig + 6 * c;
        o[0] = S[0];
        o[1] = S[4];
        o[2] = S[8];
        o[3] = 0.5 * (S[1] + S[3]);
        o[4] = 0.5 * (S[2] + S[6]);
        o[5] = 0.5 * (S[5] + S[7]);
    }
}

}  // namespace

void rc_launch_fire_init(const FireState &s, const int *status, const int *active, int n_cells, float dt0,
                         cudaStream_t st) {
    k_fire_init<<<(n_cells + 127) / 128, 128, 0, st>>>(s, status, active, n_cells, dt0);
}

void rc_launch_fire_zero_v(const KArrays &a, const FireState &s, int n_tiles, int all_cells, cudaStream_t st) {
    k_fire_zero_v<<<n_tiles, RC_TILE, 0, st>>>(a, s, all_cells);
}

void rc_launch_fire_iteration(const KParams &p, const KArrays &a, int cur, const FireState &s, int n_tiles, int n_cells,
                              float f_tol, float dt_max, float dmax, int *n_left, cudaStream_t st) {
    k_fire_power<<<n_tiles, RC_TILE, 0, st>>>(a, s);
    k_fire_control<<<(n_cells + 127) / 128, 128, 0, st>>>(s, n_cells, f_tol * f_tol, dt_max, n_left);
    k_fire_move<<<n_tiles, RC_TILE, 0, st>>>(p, a, cur, s, dmax);
}

void rc_launch_static_prep(const double *H, const double *H0, float *mcell, double *acc, int n_cells,
                           cudaStream_t st) {
    k_static_prep<<<(n_cells + 127) / 128, 128, 0, st>>>(H, H0, mcell, acc, n_cells);
}

void rc_launch_static_finish(const double *acc, const double *H0, const double *Q, const double *F, double pconv,
                             double *P, double *sig, const int *status, int n_cells, cudaStream_t st) {
    k_static_finish<<<(n_cells + 127) / 128, 128, 0, st>>>(acc, H0, Q, F, pconv, P, sig, status, n_cells);
}
