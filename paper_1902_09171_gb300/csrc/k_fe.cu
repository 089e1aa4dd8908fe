// Explicit finite elements in FP64 (Sec. 2.2, Eq. f): 8-node hexahedra (one
// centroid quadrature point, Flanagan-Belytschko stiffness hourglass control)
// or 4-node tetrahedra (the paper's C3D4: linear, constant gradients, no
// hourglass modes); one quadrature point and one r-cell per element, lumped
// mass, damped central-difference update.  One thread per element / per DOF;
// nodal sums by FP64 atomics.  NPE = nodes per element (8 or 4).
#include "rc_internal.cuh"

namespace {

// natural coordinates of the 8 nodes: (-,-,-) (+,-,-) (+,+,-) (-,+,-) (-,-,+) (+,-,+) (+,+,+) (-,+,+)
__constant__ signed char c_nat[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                                        {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};

// tetrahedron: N = (1 - xi - eta - zeta, xi, eta, zeta), dN_a/dxi_alpha
__constant__ signed char c_tet[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};

// dN_a/dxi_alpha at the quadrature point
template <int NPE>
__device__ __forceinline__ double dshape(int a, int al) {
    return NPE == 8 ? 0.125 * c_nat[a][al] : (double)c_tet[a][al];
}

template <int NPE>
__global__ void k_geometry(const double *__restrict__ X, const int *__restrict__ conn, int ne, double rho0,
                           double *gradN, double *V0, double *mass, int *err) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    // J_{i alpha} = sum_a X_{a i} dN_a/dxi_alpha
    double J[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int a = 0; a < NPE; a++) {
        const double *Xa = X + 3 * conn[NPE * e + a];
        for (int i = 0; i < 3; i++)
            for (int al = 0; al < 3; al++) J[3 * i + al] += Xa[i] * dshape<NPE>(a, al);
    }
    const double det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
                       J[2] * (J[3] * J[7] - J[4] * J[6]);
    if (!(det > 0.0)) {
        atomicExch(err, 1);
        return;
    }
    double Ji[9];
    Ji[0] = (J[4] * J[8] - J[5] * J[7]) / det;
    Ji[1] = (J[2] * J[7] - J[1] * J[8]) / det;
    Ji[2] = (J[1] * J[5] - J[2] * J[4]) / det;
    Ji[3] = (J[5] * J[6] - J[3] * J[8]) / det;
    Ji[4] = (J[0] * J[8] - J[2] * J[6]) / det;
    Ji[5] = (J[2] * J[3] - J[0] * J[5]) / det;
    Ji[6] = (J[3] * J[7] - J[4] * J[6]) / det;
    Ji[7] = (J[1] * J[6] - J[0] * J[7]) / det;
    Ji[8] = (J[0] * J[4] - J[1] * J[3]) / det;
    // grad_X N_a = J^{-T} dN_a/dxi
    for (int a = 0; a < NPE; a++)
        for (int k = 0; k < 3; k++) {
            double s = 0.0;
            for (int al = 0; al < 3; al++) s += Ji[3 * al + k] * dshape<NPE>(a, al);
            gradN[3 * NPE * e + 3 * a + k] = s;
        }
    const double V = NPE == 8 ? 8.0 * det : det / 6.0;  // reference volumes 8 and 1/6
    V0[e] = V;
    for (int a = 0; a < NPE; a++) atomicAdd(&mass[conn[NPE * e + a]], rho0 * V / NPE);
}

// prescribed DOFs take lambda val; with an affine predictor g of the load
// increment, every free DOF first moves by (lambda - lambda_prev) g
__global__ void k_apply_bc(const int *__restrict__ mask, const double *__restrict__ val,
                           const double *__restrict__ g, double lambda, double dlambda, double *d, int n3) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n3) return;
    if (mask[q]) d[q] = lambda * val[q];
    else if (g) d[q] += dlambda * g[q];
}

template <int NPE>
__global__ void k_F(const int *__restrict__ conn, const double *__restrict__ gradN, const double *__restrict__ d,
                    double *F, int ne) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    double G[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    for (int a = 0; a < NPE; a++) {
        const double *da = d + 3 * conn[NPE * e + a];
        const double *ga = gradN + 3 * NPE * e + 3 * a;
        for (int i = 0; i < 3; i++)
            for (int J = 0; J < 3; J++) G[3 * i + J] += da[i] * ga[J];
    }
    for (int k = 0; k < 9; k++) F[9 * e + k] = G[k];
}

// f_int,a = V0 P grad N_a + kappa sum_alpha gamma_{alpha a} q_alpha, kappa = hg V0^{1/3},
// gamma_{alpha a} = (h_{alpha a} - (sum_b h_{alpha b} X_b) . grad N_a) / 8,
// h = (eta zeta, zeta xi, xi eta, xi eta zeta) at the nodes, q_alpha = sum_b gamma_{alpha b} d_b.
template <int NPE>
__global__ void k_fint(const double *__restrict__ X, const int *__restrict__ conn, const double *__restrict__ gradN,
                       const double *__restrict__ V0, const double *__restrict__ P, const double *__restrict__ d,
                       double hg, double *fint, int ne) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const double *g = gradN + 3 * NPE * e, *Pe = P + 9 * e;
    const double V = V0[e];
    double fe[3 * NPE];
    for (int a = 0; a < NPE; a++)
        for (int i = 0; i < 3; i++)
            fe[3 * a + i] = V * (Pe[3 * i] * g[3 * a] + Pe[3 * i + 1] * g[3 * a + 1] + Pe[3 * i + 2] * g[3 * a + 2]);
    if (NPE == 8 && hg != 0.0) {
        const double kappa = hg * cbrt(V);
        for (int al = 0; al < 4; al++) {
            double h[8], hX[3] = {0, 0, 0};
            for (int a = 0; a < 8; a++) {
                const int x = c_nat[a][0], y = c_nat[a][1], z = c_nat[a][2];
                h[a] = al == 0 ? y * z : al == 1 ? z * x : al == 2 ? x * y : x * y * z;
                const double *Xa = X + 3 * conn[8 * e + a];
                hX[0] += h[a] * Xa[0];
                hX[1] += h[a] * Xa[1];
                hX[2] += h[a] * Xa[2];
            }
            double gam[8], q[3] = {0, 0, 0};
            for (int a = 0; a < 8; a++) {
                gam[a] = 0.125 * (h[a] - (hX[0] * g[3 * a] + hX[1] * g[3 * a + 1] + hX[2] * g[3 * a + 2]));
                const double *da = d + 3 * conn[8 * e + a];
                q[0] += gam[a] * da[0];
                q[1] += gam[a] * da[1];
                q[2] += gam[a] * da[2];
            }
            for (int a = 0; a < 8; a++)
                for (int i = 0; i < 3; i++) fe[3 * a + i] += kappa * gam[a] * q[i];
        }
    }
    for (int a = 0; a < NPE; a++)
        for (int i = 0; i < 3; i++) atomicAdd(&fint[3 * conn[NPE * e + a] + i], fe[3 * a + i]);
}

__global__ void k_update(const int *__restrict__ mask, const double *__restrict__ mass, const double *__restrict__ fint,
                         double dt, double damping, double *d, double *v, int n3) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n3) return;
    if (mask[q]) {
        v[q] = 0.0;
        return;
    }
    const double c0 = 1.0 - 0.5 * damping * dt, c1 = 1.0 + 0.5 * damping * dt;
    const double acc = -fint[q] / mass[q / 3];
    const double vn = (c0 * v[q] + dt * acc) / c1;
    v[q] = vn;
    d[q] += dt * vn;
}

// MD-fallback decision per quadrature point with hysteresis: a point trips to MD
// when the ensemble spread exceeds `on` and, once tripped, stays on MD while the
// spread exceeds `off`.  Flags: 0 surrogate, 1 tripped (MD), 2 forced MD
// (start-up increments; a forced point is not tripped).
__global__ void k_decide(const float *__restrict__ spread, float on, float off, int force_md, int *md_flag, int *n_md,
                         int ne) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const float sp = spread[e];
    const int tripped = !(sp <= on) || (md_flag[e] == 1 && !(sp <= off));
    const int flag = tripped ? 1 : (force_md ? 2 : 0);
    md_flag[e] = flag;
    if (flag) atomicAdd(n_md, 1);
}

// Replay of missed increments: mask of the points that run MD at this increment
// and still have a recorded deformation at replay position j.
__global__ void k_replay_mask(const int *__restrict__ md_flag, const int *__restrict__ n_frozen, int j, int *mask,
                              int ne) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    mask[e] = (md_flag[e] != 0 && n_frozen[e] > j) ? 1 : 0;
}

// After the step: a point on MD has no missed increment left; a point on the
// surrogate records this increment's F at the next free position of its history
// (when all kmax positions are taken, the last one is overwritten, so the
// history keeps the first kmax - 1 missed increments and the latest).
__global__ void k_track_frozen(const int *__restrict__ md_flag, const double *__restrict__ F, double *F_hist,
                               int *n_frozen, int ne, int kmax) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    if (md_flag[e] != 0) {
        n_frozen[e] = 0;
        return;
    }
    const int n = n_frozen[e];
    const int slot = n < kmax ? n : kmax - 1;
    for (int k = 0; k < 9; k++) F_hist[((size_t)slot * ne + e) * 9 + k] = F[9 * e + k];
    n_frozen[e] = n < kmax ? n + 1 : kmax;
}

// P = J sigma F^{-T} from the surrogate stress (FE frame) where the point is not on MD
__global__ void k_merge_P(const int *__restrict__ md_flag, const float *__restrict__ s_sur, const double *__restrict__ F,
                          const double *__restrict__ P_md, double *P, int ne) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    if (md_flag[e]) {
        for (int k = 0; k < 9; k++) P[9 * e + k] = P_md[9 * e + k];
        return;
    }
    const double *Fe = F + 9 * e;
    const double J = Fe[0] * (Fe[4] * Fe[8] - Fe[5] * Fe[7]) - Fe[1] * (Fe[3] * Fe[8] - Fe[5] * Fe[6]) +
                     Fe[2] * (Fe[3] * Fe[7] - Fe[4] * Fe[6]);
    double Fi[9];
    Fi[0] = (Fe[4] * Fe[8] - Fe[5] * Fe[7]) / J;
    Fi[1] = (Fe[2] * Fe[7] - Fe[1] * Fe[8]) / J;
    Fi[2] = (Fe[1] * Fe[5] - Fe[2] * Fe[4]) / J;
    Fi[3] = (Fe[5] * Fe[6] - Fe[3] * Fe[8]) / J;
    Fi[4] = (Fe[0] * Fe[8] - Fe[2] * Fe[6]) / J;
    Fi[5] = (Fe[2] * Fe[3] - Fe[0] * Fe[5]) / J;
    Fi[6] = (Fe[3] * Fe[7] - Fe[4] * Fe[6]) / J;
    Fi[7] = (Fe[1] * Fe[6] - Fe[0] * Fe[7]) / J;
    Fi[8] = (Fe[0] * Fe[4] - Fe[1] * Fe[3]) / J;
    const float *sv = s_sur + 6 * e;
    const double S[9] = {sv[0], sv[3], sv[4], sv[3], sv[1], sv[5], sv[4], sv[5], sv[2]};
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double acc = 0.0;
            for (int l = 0; l < 3; l++) acc += S[3 * i + l] * Fi[3 * j + l];
            P[9 * e + 3 * i + j] = J * acc;
        }
}

__global__ void k_copy_F(const double *__restrict__ F, double *F_prev, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) F_prev[i] = F[i];
}

}  // namespace

void fe_launch_surrogate_merge(const int *md_flag, const float *s_sur, const double *F, const double *P_md, double *P,
                               int ne, cudaStream_t s) {
    k_merge_P<<<(ne + 127) / 128, 128, 0, s>>>(md_flag, s_sur, F, P_md, P, ne);
}
void fe_launch_decide(const float *spread, float on, float off, int force_md, int *md_flag, int *n_md, int ne,
                      cudaStream_t s) {
    k_decide<<<(ne + 127) / 128, 128, 0, s>>>(spread, on, off, force_md, md_flag, n_md, ne);
}
void fe_launch_replay_mask(const int *md_flag, const int *n_frozen, int j, int *mask, int ne, cudaStream_t s) {
    k_replay_mask<<<(ne + 127) / 128, 128, 0, s>>>(md_flag, n_frozen, j, mask, ne);
}
void fe_launch_track_frozen(const int *md_flag, const double *F, double *F_hist, int *n_frozen, int ne, int kmax,
                            cudaStream_t s) {
    k_track_frozen<<<(ne + 127) / 128, 128, 0, s>>>(md_flag, F, F_hist, n_frozen, ne, kmax);
}
void fe_launch_copy_F(const double *F, double *F_prev, int ne, cudaStream_t s) {
    k_copy_F<<<(9 * ne + 255) / 256, 256, 0, s>>>(F, F_prev, 9 * ne);
}

void fe_launch_geometry(int npe, const double *X, const int *conn, int ne, double rho0, double *gradN, double *V0,
                        double *mass, int *err, cudaStream_t s) {
    if (npe == 4) k_geometry<4><<<(ne + 127) / 128, 128, 0, s>>>(X, conn, ne, rho0, gradN, V0, mass, err);
    else k_geometry<8><<<(ne + 127) / 128, 128, 0, s>>>(X, conn, ne, rho0, gradN, V0, mass, err);
}
void fe_launch_apply_bc(const int *mask, const double *val, const double *g, double lambda, double dlambda, double *d,
                        int n3, cudaStream_t s) {
    k_apply_bc<<<(n3 + 255) / 256, 256, 0, s>>>(mask, val, g, lambda, dlambda, d, n3);
}
void fe_launch_F(int npe, const int *conn, const double *gradN, const double *d, double *F, int ne, cudaStream_t s) {
    if (npe == 4) k_F<4><<<(ne + 127) / 128, 128, 0, s>>>(conn, gradN, d, F, ne);
    else k_F<8><<<(ne + 127) / 128, 128, 0, s>>>(conn, gradN, d, F, ne);
}
void fe_launch_fint(int npe, const double *X, const int *conn, const double *gradN, const double *V0, const double *P,
                    const double *d, double hg, double *fint, int ne, cudaStream_t s) {
    if (npe == 4) k_fint<4><<<(ne + 127) / 128, 128, 0, s>>>(X, conn, gradN, V0, P, d, hg, fint, ne);
    else k_fint<8><<<(ne + 127) / 128, 128, 0, s>>>(X, conn, gradN, V0, P, d, hg, fint, ne);
}
void fe_launch_update(const int *mask, const double *mass, const double *fint, double dt, double damping, double *d,
                      double *v, int n3, cudaStream_t s) {
    k_update<<<(n3 + 255) / 256, 256, 0, s>>>(mask, mass, fint, dt, damping, d, v, n3);
}
