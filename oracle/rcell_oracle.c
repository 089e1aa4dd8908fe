/*
 * FP64 CPU oracle for the r-cell hot path of the FEM <-> MD hierarchical coupling
 * (Murashima, Urata & Li, arXiv:1902.09171).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark load it.  It shares
 * no code, header, table or constant generator with the CUDA library.
 *
 * Every routine follows a passage of the paper (Sec. 2.1, Eqs. LAMMPS1..LAMMPS2,
 * Eq. Pmd, Eq. f) or the potential / integrator definitions that the paper
 * delegates to its MD engine; each function names its source.
 *
 * Conventions
 *   - 3x3 matrices are row-major double[9]; a box matrix H holds the three box
 *     vectors as COLUMNS, so r = H s for fractional s (Eq. LAMMPS1).
 *   - Positions / velocities / forces are double[3n], atom-major.
 *   - Virial W = sum over unordered pairs of r_ij (x) f_ij, with r_ij = x_i - x_j
 *     and f_ij the force on i due to j (compression-positive, like a pressure).
 *   - Stress returned to callers is the tension-positive Cauchy stress
 *     sigma = -(K + W)/V, in Voigt order xx, yy, zz, xy, xz, yz.
 *
 * Parity pins: every function here is pinned by a CPU test (tests/test_oracle_*.py)
 * against a closed form, a worked example printed in the paper (Table 1), a
 * brute-force evaluation, or an invariant; none is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* status codes (oracle-local)                                               */
/* ------------------------------------------------------------------------ */
enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2, OR_EDEGEN = 4, OR_EBOX = 5, OR_EBOND = 6 };

/* ------------------------------------------------------------------------ */
/* small 3x3 helpers                                                         */
/* ------------------------------------------------------------------------ */
static void m3_mul(const double *A, const double *B, double *C) {
    double T[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += A[3 * i + k] * B[3 * k + j];
            T[3 * i + j] = s;
        }
    memcpy(C, T, sizeof T);
}

static double m3_det(const double *A) {
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}

/* inverse by the adjugate; returns the determinant */
static double m3_inv(const double *A, double *B) {
    double d = m3_det(A);
    double T[9];
    T[0] = (A[4] * A[8] - A[5] * A[7]) / d;
    T[1] = (A[2] * A[7] - A[1] * A[8]) / d;
    T[2] = (A[1] * A[5] - A[2] * A[4]) / d;
    T[3] = (A[5] * A[6] - A[3] * A[8]) / d;
    T[4] = (A[0] * A[8] - A[2] * A[6]) / d;
    T[5] = (A[2] * A[3] - A[0] * A[5]) / d;
    T[6] = (A[3] * A[7] - A[4] * A[6]) / d;
    T[7] = (A[1] * A[6] - A[0] * A[7]) / d;
    T[8] = (A[0] * A[4] - A[1] * A[3]) / d;
    memcpy(B, T, sizeof T);
    return d;
}

static void m3_mv(const double *A, const double *x, double *y) {
    double t0 = A[0] * x[0] + A[1] * x[1] + A[2] * x[2];
    double t1 = A[3] * x[0] + A[4] * x[1] + A[5] * x[2];
    double t2 = A[6] * x[0] + A[7] * x[1] + A[8] * x[2];
    y[0] = t0; y[1] = t1; y[2] = t2;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.1: F = Q R with Q orthogonal and R upper triangular with a positive  */
/* diagonal ("R should be positive definite").  The paper computes it by      */
/* Gram-Schmidt; the oracle deliberately uses Householder reflections, which  */
/* reach the same unique factor once the diagonal signs are fixed.            */
/* Returns OR_EDEGEN when det F <= 0 (no rotation + positive stretch exists). */
/* ------------------------------------------------------------------------ */
int or_qr(const double *F, double *Q, double *R) {
    double A[9], Qm[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    memcpy(A, F, sizeof A);
    double detF = m3_det(F);
    if (!(detF > 0.0)) return OR_EDEGEN;
    for (int k = 0; k < 2; k++) {
        double nrm = 0.0;
        for (int i = k; i < 3; i++) nrm += A[3 * i + k] * A[3 * i + k];
        nrm = sqrt(nrm);
        if (nrm == 0.0) continue;
        double alpha = A[3 * k + k] > 0.0 ? -nrm : nrm;
        double u[3] = {0, 0, 0};
        for (int i = k; i < 3; i++) u[i] = A[3 * i + k];
        u[k] -= alpha;
        double un2 = 0.0;
        for (int i = k; i < 3; i++) un2 += u[i] * u[i];
        if (un2 == 0.0) continue;
        /* A <- (I - 2 u u^T / |u|^2) A */
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int i = k; i < 3; i++) s += u[i] * A[3 * i + j];
            s *= 2.0 / un2;
            for (int i = k; i < 3; i++) A[3 * i + j] -= s * u[i];
        }
        /* Qm <- Qm (I - 2 u u^T / |u|^2) */
        for (int i = 0; i < 3; i++) {
            double s = 0.0;
            for (int j = k; j < 3; j++) s += Qm[3 * i + j] * u[j];
            s *= 2.0 / un2;
            for (int j = k; j < 3; j++) Qm[3 * i + j] -= s * u[j];
        }
    }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < i; j++) A[3 * i + j] = 0.0;
    /* fix signs so that diag(R) > 0: R <- D R, Q <- Q D */
    for (int i = 0; i < 3; i++) {
        if (A[3 * i + i] < 0.0) {
            for (int j = 0; j < 3; j++) A[3 * i + j] = -A[3 * i + j];
            for (int j = 0; j < 3; j++) Qm[3 * j + i] = -Qm[3 * j + i];
        }
        if (!(A[3 * i + i] > 0.0)) return OR_EDEGEN;
    }
    memcpy(Q, Qm, sizeof Qm);
    memcpy(R, A, sizeof A);
    return OR_OK;
}

/* Eq. LAMMPS2: Delta R = R(t) R(t-1)^{-1} */
void or_delta_R(const double *R_new, const double *R_prev, double *dR) {
    double Ri[9];
    m3_inv(R_prev, Ri);
    m3_mul(R_new, Ri, dR);
}

/* The remap that Delta R implies for atoms held by the MD engine: x <- Delta R x.
 * (Velocities are left as they are.) */
void or_remap(int n, double *x, const double *dR) {
    for (int i = 0; i < n; i++) m3_mv(dR, x + 3 * i, x + 3 * i);
}

/* Perpendicular width of the box along each fractional axis d: V / |a_e x a_f|,
 * i.e. 1 / |row d of H^{-1}|. */
void or_box_widths(const double *H, double *w) {
    double Hi[9];
    m3_inv(H, Hi);
    for (int d = 0; d < 3; d++) {
        double s = Hi[3 * d] * Hi[3 * d] + Hi[3 * d + 1] * Hi[3 * d + 1] + Hi[3 * d + 2] * Hi[3 * d + 2];
        w[d] = 1.0 / sqrt(s);
    }
}

/* Sec. 2.1 (after Eq. LAMMPS2): sigma_FEM = Q sigma_MD Q^T and Eq. Pmd:
 * P = J sigma_FEM F^{-T}.  sigma in Voigt (xx,yy,zz,xy,xz,yz); P row-major. */
void or_rotate_pk1(const double *Q, const double *F, const double *s_md, double *s_fem, double *P) {
    double S[9] = {s_md[0], s_md[3], s_md[4], s_md[3], s_md[1], s_md[5], s_md[4], s_md[5], s_md[2]};
    double QT[9], T[9], SF[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) QT[3 * i + j] = Q[3 * j + i];
    m3_mul(Q, S, T);
    m3_mul(T, QT, SF);
    if (s_fem) {
        s_fem[0] = SF[0]; s_fem[1] = SF[4]; s_fem[2] = SF[8];
        s_fem[3] = 0.5 * (SF[1] + SF[3]);
        s_fem[4] = 0.5 * (SF[2] + SF[6]);
        s_fem[5] = 0.5 * (SF[5] + SF[7]);
    }
    if (P) {
        double Fi[9], FiT[9];
        double J = m3_inv(F, Fi);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) FiT[3 * i + j] = Fi[3 * j + i];
        m3_mul(SF, FiT, P);
        for (int k = 0; k < 9; k++) P[k] *= J;
    }
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw,        */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11), written from the    */
/* published round function: two 32x32->64 multiplies, a word permutation and */
/* a Weyl-sequence key schedule, ten rounds.                                  */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Three standard normals for (atom tag, cell, force evaluation, seed): one
 * Philox block -> four uniforms u = (k + 1/2) 2^-32 in (0,1) -> two Box-Muller
 * pairs; the first three normals are used. */
void or_normals3(uint32_t tag, uint32_t cell, uint64_t eval, uint64_t seed, double *z) {
    uint32_t ctr[4] = {tag, cell, (uint32_t)eval, (uint32_t)(eval >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    or_philox4x32_10(ctr, key, o);
    const double two32 = 4294967296.0, twopi = 6.283185307179586476925287;
    double u0 = ((double)o[0] + 0.5) / two32, u1 = ((double)o[1] + 0.5) / two32;
    double u2 = ((double)o[2] + 0.5) / two32, u3 = ((double)o[3] + 0.5) / two32;
    double r0 = sqrt(-2.0 * log(u0)), r1 = sqrt(-2.0 * log(u2));
    z[0] = r0 * cos(twopi * u1);
    z[1] = r0 * sin(twopi * u1);
    z[2] = r1 * cos(twopi * u3);
}

/* ------------------------------------------------------------------------ */
/* Potentials                                                                */
/* ------------------------------------------------------------------------ */
enum { OR_LJ = 0, OR_SC = 1, OR_KG = 2 };

typedef struct {
    int kind;        /* OR_LJ, OR_SC, OR_KG                                   */
    double eps;      /* LJ epsilon, or Sutton-Chen epsilon                     */
    double sigma;    /* LJ sigma, or Sutton-Chen lattice parameter a            */
    double rc;       /* cutoff: strict r < rc, plain truncation (no shift)      */
    double n, m, c;  /* Sutton-Chen exponents and c                            */
    double k_fene, R0; /* FENE bond (Kremer-Grest)                             */
} or_pot;

/* ordered neighbour pair (i, j) with d = x_j(image) - x_i */
typedef struct {
    int i, j;
    double d[3];
    double r2;
} or_pair;

typedef struct {
    or_pair *p;
    long n, cap;
} or_plist;

static int pl_push(or_plist *L, int i, int j, const double *d, double r2) {
    if (L->n == L->cap) {
        long nc = L->cap ? 2 * L->cap : 4096;
        or_pair *np = (or_pair *)realloc(L->p, (size_t)nc * sizeof(or_pair));
        if (!np) return OR_ENOMEM;
        L->p = np;
        L->cap = nc;
    }
    or_pair *q = &L->p[L->n++];
    q->i = i; q->j = j; q->d[0] = d[0]; q->d[1] = d[1]; q->d[2] = d[2]; q->r2 = r2;
    return OR_OK;
}

/* All ordered pairs (i, j, image) with |x_j + H t - x_i| < rc, by brute force
 * over every pair and the 27 images around the nearest fractional image.
 * Exact whenever every perpendicular box width is >= 2 rc. */
static int pairs_brute(int n, const double *x, const double *H, double rc, or_plist *L) {
    double Hi[9];
    m3_inv(H, Hi);
    double *s = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (!s) return OR_ENOMEM;
    for (int i = 0; i < n; i++) m3_mv(Hi, x + 3 * i, s + 3 * i);
    double rc2 = rc * rc;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            double k0[3];
            for (int d = 0; d < 3; d++) k0[d] = -rint(s[3 * j + d] - s[3 * i + d]);
            for (int a = -1; a <= 1; a++)
                for (int b = -1; b <= 1; b++)
                    for (int c = -1; c <= 1; c++) {
                        double t[3] = {k0[0] + a, k0[1] + b, k0[2] + c};
                        if (i == j && t[0] == 0 && t[1] == 0 && t[2] == 0) continue;
                        double Ht[3];
                        m3_mv(H, t, Ht);
                        double dd[3];
                        for (int d = 0; d < 3; d++) dd[d] = x[3 * j + d] - x[3 * i + d] + Ht[d];
                        double r2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
                        if (r2 < rc2) {
                            int e = pl_push(L, i, j, dd, r2);
                            if (e) { free(s); return e; }
                        }
                    }
        }
    free(s);
    return OR_OK;
}

static long floordiv_l(long a, long b) {
    long q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q--;
    return q;
}

/* Same pair set through a cell list over fractional coordinates: n_d =
 * floor(w_d / rc) bins per axis and the 27-stencil with explicit image
 * shifts.  Each (atom, image) within rc lies within one bin of the home bin in
 * the unwrapped bin lattice, and distinct stencil offsets are distinct
 * unwrapped bins, so every pair is found exactly once whenever w_d >= rc. */
static int pairs_cells(int n, const double *x, const double *H, double rc, or_plist *L) {
    double Hi[9], w[3];
    m3_inv(H, Hi);
    or_box_widths(H, w);
    long nb[3];
    for (int d = 0; d < 3; d++) {
        nb[d] = (long)floor(w[d] / rc);
        if (nb[d] < 1) return OR_EBOX;
        if (nb[d] > 64) nb[d] = 64;
    }
    long ncell = nb[0] * nb[1] * nb[2];
    long *head = (long *)malloc(sizeof(long) * (size_t)ncell);
    long *next = (long *)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
    long *img = (long *)malloc(sizeof(long) * 3 * (size_t)(n > 0 ? n : 1));
    long *bin = (long *)malloc(sizeof(long) * 3 * (size_t)(n > 0 ? n : 1));
    if (!head || !next || !img || !bin) { free(head); free(next); free(img); free(bin); return OR_ENOMEM; }
    for (long c = 0; c < ncell; c++) head[c] = -1;
    for (int i = n - 1; i >= 0; i--) {
        double s[3];
        m3_mv(Hi, x + 3 * i, s);
        for (int d = 0; d < 3; d++) {
            double fl = floor(s[d]);
            double sw = s[d] - fl;
            long b = (long)floor(sw * (double)nb[d]);
            if (b >= nb[d]) b = nb[d] - 1;
            if (b < 0) b = 0;
            img[3 * i + d] = (long)fl;
            bin[3 * i + d] = b;
        }
        long c = (bin[3 * i] * nb[1] + bin[3 * i + 1]) * nb[2] + bin[3 * i + 2];
        next[i] = head[c];
        head[c] = i;
    }
    double rc2 = rc * rc;
    int err = OR_OK;
    for (int i = 0; i < n && !err; i++) {
        for (int a = -1; a <= 1; a++)
            for (int b = -1; b <= 1; b++)
                for (int cc = -1; cc <= 1; cc++) {
                    long u[3] = {bin[3 * i] + a, bin[3 * i + 1] + b, bin[3 * i + 2] + cc};
                    long sh[3], wb[3];
                    for (int d = 0; d < 3; d++) {
                        sh[d] = floordiv_l(u[d], nb[d]);
                        wb[d] = u[d] - sh[d] * nb[d];
                    }
                    long c = (wb[0] * nb[1] + wb[1]) * nb[2] + wb[2];
                    for (long j = head[c]; j >= 0; j = next[j]) {
                        double t[3];
                        for (int d = 0; d < 3; d++) t[d] = (double)(sh[d] + img[3 * i + d] - img[3 * j + d]);
                        if (j == i && t[0] == 0 && t[1] == 0 && t[2] == 0) continue;
                        double Ht[3];
                        m3_mv(H, t, Ht);
                        double dd[3];
                        for (int d = 0; d < 3; d++) dd[d] = x[3 * j + d] - x[3 * i + d] + Ht[d];
                        double r2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
                        if (r2 < rc2) {
                            err = pl_push(L, i, (int)j, dd, r2);
                            if (err) break;
                        }
                    }
                }
    }
    free(head); free(next); free(img); free(bin);
    return err;
}

/* Ordered neighbour pairs within rlist, written as (i, j) int pairs.
 * Returns the pair count, or -1 on error / overflow of max_pairs. */
long or_neighbor_pairs(int n, const double *x, const double *H, double rlist, int use_cells, int *out,
                       long max_pairs) {
    or_plist L = {0, 0, 0};
    int e = use_cells ? pairs_cells(n, x, H, rlist, &L) : pairs_brute(n, x, H, rlist, &L);
    if (e) { free(L.p); return -1; }
    if (L.n > max_pairs) { free(L.p); return -1; }
    for (long k = 0; k < L.n; k++) { out[2 * k] = L.p[k].i; out[2 * k + 1] = L.p[k].j; }
    long cnt = L.n;
    free(L.p);
    return cnt;
}

/* bonded partner lookup: is (i, j) one of the bonds? (bonds sorted per atom) */
typedef struct {
    int *start, *nbr;
} or_bondmap;

static int bondmap_build(int n, int nb, const int *bonds, or_bondmap *B) {
    B->start = (int *)calloc((size_t)n + 1, sizeof(int));
    B->nbr = (int *)malloc(sizeof(int) * (size_t)(2 * nb > 0 ? 2 * nb : 1));
    if (!B->start || !B->nbr) return OR_ENOMEM;
    for (int b = 0; b < nb; b++) { B->start[bonds[2 * b] + 1]++; B->start[bonds[2 * b + 1] + 1]++; }
    for (int i = 0; i < n; i++) B->start[i + 1] += B->start[i];
    int *fill = (int *)calloc((size_t)n, sizeof(int));
    if (!fill) return OR_ENOMEM;
    for (int b = 0; b < nb; b++) {
        int i = bonds[2 * b], j = bonds[2 * b + 1];
        B->nbr[B->start[i] + fill[i]++] = j;
        B->nbr[B->start[j] + fill[j]++] = i;
    }
    free(fill);
    return OR_OK;
}

static int bonded(const or_bondmap *B, int i, int j) {
    for (int k = B->start[i]; k < B->start[i + 1]; k++)
        if (B->nbr[k] == j) return 1;
    return 0;
}

/*
 * Conservative forces, potential energy and pair virial of one periodic cell.
 *   LJ  : U(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6], r < rc, unshifted.
 *   SC  : Sutton-Chen EAM, E = eps [ 1/2 sum_i sum_j!=i (a/r)^n - c sum_i sqrt(rho_i) ],
 *         rho_i = sum_j!=i (a/r)^m, r < rc.
 *   KG  : Kremer-Grest bead-spring: LJ between non-bonded pairs (r < rc) plus,
 *         for each bond, FENE -1/2 k R0^2 ln(1 - (r/R0)^2) and the purely
 *         repulsive WCA LJ (cut and shifted at 2^{1/6} sigma).
 * f: 3n out, W: 9 out (pair virial, compression-positive), returns energy via *pe.
 * pe_atom (optional): per-atom share of the energy.
 */
int or_forces(const or_pot *P, int n, const double *x, const double *H, int n_bonds, const int *bonds,
              int use_cells, double *f, double *W, double *pe, double *pe_atom) {
    or_plist L = {0, 0, 0};
    int e = use_cells ? pairs_cells(n, x, H, P->rc, &L) : pairs_brute(n, x, H, P->rc, &L);
    if (e) { free(L.p); return e; }
    for (int k = 0; k < 3 * n; k++) f[k] = 0.0;
    for (int k = 0; k < 9; k++) W[k] = 0.0;
    if (pe_atom)
        for (int k = 0; k < n; k++) pe_atom[k] = 0.0;
    double E = 0.0;
    int err = OR_OK;
    or_bondmap B = {0, 0};
    if (P->kind == OR_KG) {
        err = bondmap_build(n, n_bonds, bonds, &B);
        if (err) goto done;
    }
    if (P->kind == OR_LJ || P->kind == OR_KG) {
        double s2 = P->sigma * P->sigma;
        for (long k = 0; k < L.n; k++) {
            const or_pair *q = &L.p[k];
            if (P->kind == OR_KG && bonded(&B, q->i, q->j)) continue;
            double sr2 = s2 / q->r2, sr6 = sr2 * sr2 * sr2, sr12 = sr6 * sr6;
            double U = 4.0 * P->eps * (sr12 - sr6);
            /* dU/dr / r */
            double g_over_r = -24.0 * P->eps * (2.0 * sr12 - sr6) / q->r2;
            E += 0.5 * U;
            if (pe_atom) pe_atom[q->i] += 0.5 * U;
            for (int a = 0; a < 3; a++) f[3 * q->i + a] += g_over_r * q->d[a];
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) W[3 * a + b] -= 0.5 * g_over_r * q->d[a] * q->d[b];
        }
    } else if (P->kind == OR_SC) {
        double *rho = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
        if (!rho) { err = OR_ENOMEM; goto done; }
        for (long k = 0; k < L.n; k++) {
            const or_pair *q = &L.p[k];
            double ar = P->sigma / sqrt(q->r2);
            rho[q->i] += pow(ar, P->m);
        }
        for (int i = 0; i < n; i++) {
            double emb = -P->eps * P->c * sqrt(rho[i]);
            E += emb;
            if (pe_atom) pe_atom[i] += emb;
        }
        for (long k = 0; k < L.n; k++) {
            const or_pair *q = &L.p[k];
            double r = sqrt(q->r2), ar = P->sigma / r;
            double arn = pow(ar, P->n), arm = pow(ar, P->m);
            double Upair = P->eps * arn;
            E += 0.5 * Upair;
            if (pe_atom) pe_atom[q->i] += 0.5 * Upair;
            double dEdr = (P->eps / r) *
                          (-P->n * arn + 0.5 * P->c * P->m * (1.0 / sqrt(rho[q->i]) + 1.0 / sqrt(rho[q->j])) * arm);
            double g_over_r = dEdr / r;
            for (int a = 0; a < 3; a++) f[3 * q->i + a] += g_over_r * q->d[a];
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) W[3 * a + b] -= 0.5 * g_over_r * q->d[a] * q->d[b];
        }
        free(rho);
    } else {
        err = OR_EINVAL;
        goto done;
    }
    if (P->kind == OR_KG) {
        double Hi[9];
        m3_inv(H, Hi);
        double rwca2 = pow(2.0, 1.0 / 3.0) * P->sigma * P->sigma;
        for (int b = 0; b < n_bonds; b++) {
            int i = bonds[2 * b], j = bonds[2 * b + 1];
            /* minimum image of the bond vector */
            double dx[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1], x[3 * j + 2] - x[3 * i + 2]};
            double ds[3];
            m3_mv(Hi, dx, ds);
            double best = 1e300, bd[3] = {0, 0, 0};
            for (int a0 = -1; a0 <= 1; a0++)
                for (int a1 = -1; a1 <= 1; a1++)
                    for (int a2 = -1; a2 <= 1; a2++) {
                        double t[3] = {a0 - rint(ds[0]), a1 - rint(ds[1]), a2 - rint(ds[2])}, Ht[3];
                        m3_mv(H, t, Ht);
                        double dd[3] = {dx[0] + Ht[0], dx[1] + Ht[1], dx[2] + Ht[2]};
                        double r2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
                        if (r2 < best) { best = r2; bd[0] = dd[0]; bd[1] = dd[1]; bd[2] = dd[2]; }
                    }
            double r2 = best, R02 = P->R0 * P->R0;
            if (!(r2 < R02)) { err = OR_EBOND; goto done; }
            double U = -0.5 * P->k_fene * R02 * log(1.0 - r2 / R02);
            double g_over_r = P->k_fene / (1.0 - r2 / R02);
            if (r2 < rwca2) {
                double sr2 = P->sigma * P->sigma / r2, sr6 = sr2 * sr2 * sr2, sr12 = sr6 * sr6;
                U += 4.0 * P->eps * (sr12 - sr6) + P->eps;
                g_over_r += -24.0 * P->eps * (2.0 * sr12 - sr6) / r2;
            }
            E += U;
            if (pe_atom) { pe_atom[i] += 0.5 * U; pe_atom[j] += 0.5 * U; }
            for (int a = 0; a < 3; a++) { f[3 * i + a] += g_over_r * bd[a]; f[3 * j + a] -= g_over_r * bd[a]; }
            for (int a = 0; a < 3; a++)
                for (int c = 0; c < 3; c++) W[3 * a + c] -= g_over_r * bd[a] * bd[c];
        }
    }
done:
    free(L.p);
    free(B.start);
    free(B.nbr);
    *pe = E;
    return err;
}

/* ------------------------------------------------------------------------ */
/* Fixed-box MD of one r-cell: velocity Verlet with a force-form Langevin     */
/* thermostat, sampling the virial stress over the last n_avg steps.          */
/* ------------------------------------------------------------------------ */
typedef struct {
    int units;      /* 0: metal (eV, A, ps, amu, stress in GPa); 1: reduced LJ units */
    double mass;    /* particle mass                                           */
    double kT;      /* thermostat temperature (energy units)                    */
    double tau;     /* Langevin damping time; <= 0 switches the thermostat off  */
    double dt;      /* time step                                                */
    uint64_t seed;  /* Philox key                                               */
} or_md;

/* unit factors from CODATA constants (metal) or 1 (lj) */
static double md_ftm2v(int units) {
    /* (eV / (Angstrom amu)) expressed in Angstrom / ps^2 */
    const double eV = 1.602176634e-19, amu = 1.66053906660e-27;
    return units == 0 ? eV / (1e-10 * amu) / 1e14 : 1.0;
}
static double md_pconv(int units) { return units == 0 ? 1.602176634e-19 / 1e-30 / 1e9 : 1.0; }

double or_ftm2v(int units) { return md_ftm2v(units); }
double or_pconv(int units) { return md_pconv(units); }

/* instantaneous tension-positive stress of a configuration (Voigt, units of
 * the unit system): sigma = -(sum m v (x) v + W) / det H */
void or_stress_inst(int units, double mass, int n, const double *v, const double *W, const double *H, double *s6) {
    double K[9] = {0};
    double mvv2e = 1.0 / md_ftm2v(units);
    for (int i = 0; i < n; i++)
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) K[3 * a + b] += mass * v[3 * i + a] * v[3 * i + b] * mvv2e;
    double V = m3_det(H), c = -md_pconv(units) / V;
    s6[0] = c * (K[0] + W[0]);
    s6[1] = c * (K[4] + W[4]);
    s6[2] = c * (K[8] + W[8]);
    s6[3] = c * 0.5 * (K[1] + W[1] + K[3] + W[3]);
    s6[4] = c * 0.5 * (K[2] + W[2] + K[6] + W[6]);
    s6[5] = c * 0.5 * (K[5] + W[5] + K[7] + W[7]);
}

/* acceleration including the Langevin friction (on the velocity held at force
 * time) and random force drawn for force evaluation number `eval` */
static void md_accel(const or_md *M, int n, const double *f, const double *v, uint32_t cell, uint64_t eval,
                     double *acc) {
    double fm = md_ftm2v(M->units) / M->mass;
    int thermo = M->tau > 0.0;
    double sig = thermo ? sqrt(2.0 * M->kT * md_ftm2v(M->units) / (M->mass * M->tau * M->dt)) : 0.0;
    for (int i = 0; i < n; i++) {
        double z[3] = {0, 0, 0};
        if (thermo) or_normals3((uint32_t)i, cell, eval, M->seed, z);
        for (int a = 0; a < 3; a++) {
            double ai = f[3 * i + a] * fm;
            if (thermo) ai += -v[3 * i + a] / M->tau + sig * z[a];
            acc[3 * i + a] = ai;
        }
    }
}

/*
 * Run n_steps of MD on one cell at fixed box H (upper triangular or general).
 * State semantics, shared with the CUDA library by specification (not code):
 *   setup:   f = F(x_0); a_0 = f/m + Langevin(v_0, eval e); e += 1
 *   step s:  v += dt/2 a;  x += dt v;  f = F(x_s); a = f/m + Langevin(v, eval e); e += 1;
 *            v += dt/2 a;  sample when s > n_steps - n_avg
 * Samples (stress Voigt, potential energy, kinetic energy) go to the series
 * arrays (n_avg entries each, may be NULL).  *eval is advanced.
 */
int or_md_run(const or_pot *P, const or_md *M, int n, double *x, double *v, const double *H, int n_bonds,
              const int *bonds, uint32_t cell, uint64_t *eval, int n_steps, int n_avg, double *stress_series,
              double *pe_series, double *ke_series) {
    if (n_steps <= 0) return OR_OK;
    if (n_avg > n_steps) n_avg = n_steps;
    double *f = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *acc = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    if (!f || !acc) { free(f); free(acc); return OR_ENOMEM; }
    double W[9], pe;
    int err = or_forces(P, n, x, H, n_bonds, bonds, 1, f, W, &pe, NULL);
    if (err) goto out;
    md_accel(M, n, f, v, cell, *eval, acc);
    (*eval)++;
    double hdt = 0.5 * M->dt;
    for (int s = 1; s <= n_steps; s++) {
        for (int k = 0; k < 3 * n; k++) { v[k] += hdt * acc[k]; x[k] += M->dt * v[k]; }
        err = or_forces(P, n, x, H, n_bonds, bonds, 1, f, W, &pe, NULL);
        if (err) goto out;
        md_accel(M, n, f, v, cell, *eval, acc);
        (*eval)++;
        for (int k = 0; k < 3 * n; k++) v[k] += hdt * acc[k];
        if (s > n_steps - n_avg) {
            int slot = s - (n_steps - n_avg) - 1;
            if (stress_series) or_stress_inst(M->units, M->mass, n, v, W, H, stress_series + 6 * slot);
            if (pe_series) pe_series[slot] = pe;
            if (ke_series) {
                double ke = 0.0;
                for (int k = 0; k < 3 * n; k++) ke += v[k] * v[k];
                ke_series[slot] = 0.5 * M->mass * ke / md_ftm2v(M->units);
            }
        }
    }
out:
    free(f);
    free(acc);
    return err;
}

/* ------------------------------------------------------------------------ */
/* Sampling statistics: mean and a blocking (Flyvbjerg-Petersen) standard     */
/* error.  Level k uses n_k = floor(n / 2^k) consecutive block means of 2^k   */
/* samples; SE_k = sqrt(sum (m - mbar)^2 / (n_k (n_k - 1))).  The reported    */
/* error is the largest SE_k over levels that keep at least 16 blocks (level  */
/* 0 always counts).                                                          */
/* ------------------------------------------------------------------------ */
void or_block_stats(int n, const double *y, int stride, double *mean, double *se) {
    double s = 0.0;
    for (int t = 0; t < n; t++) s += y[(size_t)t * stride];
    *mean = n > 0 ? s / n : 0.0;
    double best = 0.0;
    for (int k = 0;; k++) {
        int bs = 1 << k, nk = n / bs;
        if (nk < 2) break;
        if (k > 0 && nk < 16) break;
        double mb = 0.0;
        for (int b = 0; b < nk; b++) {
            double m = 0.0;
            for (int t = 0; t < bs; t++) m += y[(size_t)(b * bs + t) * stride];
            mb += m / bs;
        }
        mb /= nk;
        double v = 0.0;
        for (int b = 0; b < nk; b++) {
            double m = 0.0;
            for (int t = 0; t < bs; t++) m += y[(size_t)(b * bs + t) * stride];
            m /= bs;
            v += (m - mb) * (m - mb);
        }
        double sek = sqrt(v / ((double)nk * (nk - 1)));
        if (sek > best) best = sek;
    }
    *se = best;
}

/* ------------------------------------------------------------------------ */
/* Finite elements (Sec. 2.2, Eq. f): 8-node hexahedron, one quadrature point */
/* at the centroid, lumped mass, central-difference explicit update with      */
/* mass-proportional damping, Flanagan-Belytschko stiffness hourglass control.*/
/* Local node a sits at natural coordinates (xi_a, eta_a, zeta_a) in {-1,1}^3  */
/* in the order (-,-,-) (+,-,-) (+,+,-) (-,+,-) (-,-,+) (+,-,+) (+,+,+) (-,+,+).*/
/* ------------------------------------------------------------------------ */
static const int HEX_NAT[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                                  {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};

/* grad_X N_a at the centroid (8x3) and the element volume 8 det J(0) */
int or_hex8_geometry(const double *X, double *gradN, double *V0) {
    double J[9] = {0};
    for (int a = 0; a < 8; a++)
        for (int i = 0; i < 3; i++)
            for (int al = 0; al < 3; al++) J[3 * i + al] += X[3 * a + i] * 0.125 * HEX_NAT[a][al];
    double Ji[9];
    double det = m3_inv(J, Ji);
    if (!(det > 0.0)) return OR_EDEGEN;
    /* grad_X N_a = J^{-T} dN_a/dxi */
    for (int a = 0; a < 8; a++)
        for (int k = 0; k < 3; k++) {
            double s = 0.0;
            for (int al = 0; al < 3; al++) s += Ji[3 * al + k] * 0.125 * HEX_NAT[a][al];
            gradN[3 * a + k] = s;
        }
    *V0 = 8.0 * det;
    return OR_OK;
}

/* F = I + sum_a d_a (x) grad_X N_a */
void or_hex8_F(const double *gradN, const double *d, double *F) {
    for (int i = 0; i < 3; i++)
        for (int J = 0; J < 3; J++) {
            double s = (i == J) ? 1.0 : 0.0;
            for (int a = 0; a < 8; a++) s += d[3 * a + i] * gradN[3 * a + J];
            F[3 * i + J] = s;
        }
}

/* f_int,a = V0 P grad_X N_a  plus the hourglass force
 *   gamma_{alpha,a} = (h_{alpha,a} - (sum_b h_{alpha,b} X_b) . grad_X N_a) / 8,
 *   h = (eta zeta, zeta xi, xi eta, xi eta zeta) at the nodes,
 *   f_hg,a = +kappa sum_alpha gamma_{alpha,a} q_alpha,  q_alpha = sum_b gamma_{alpha,b} d_b,
 *   kappa = hg_coef * V0^{1/3}.  As part of f_int (M a = f_ext - f_int) the term
 *   resists the mode: f_hg . d = kappa sum_alpha |q_alpha|^2 >= 0. */
void or_hex8_fint(const double *X, const double *gradN, double V0, const double *P, const double *d, double hg_coef,
                  double *fint) {
    for (int a = 0; a < 8; a++)
        for (int i = 0; i < 3; i++) {
            double s = 0.0;
            for (int J = 0; J < 3; J++) s += P[3 * i + J] * gradN[3 * a + J];
            fint[3 * a + i] = V0 * s;
        }
    if (hg_coef == 0.0) return;
    double kappa = hg_coef * cbrt(V0);
    for (int al = 0; al < 4; al++) {
        double h[8];
        for (int a = 0; a < 8; a++) {
            const int *z = HEX_NAT[a];
            h[a] = al == 0 ? z[1] * z[2] : al == 1 ? z[2] * z[0] : al == 2 ? z[0] * z[1] : z[0] * z[1] * z[2];
        }
        double hX[3] = {0, 0, 0};
        for (int b = 0; b < 8; b++)
            for (int k = 0; k < 3; k++) hX[k] += h[b] * X[3 * b + k];
        double g[8];
        for (int a = 0; a < 8; a++)
            g[a] = 0.125 * (h[a] - (hX[0] * gradN[3 * a] + hX[1] * gradN[3 * a + 1] + hX[2] * gradN[3 * a + 2]));
        double q[3] = {0, 0, 0};
        for (int b = 0; b < 8; b++)
            for (int i = 0; i < 3; i++) q[i] += g[b] * d[3 * b + i];
        for (int a = 0; a < 8; a++)
            for (int i = 0; i < 3; i++) fint[3 * a + i] += kappa * g[a] * q[i];
    }
}

/*
 * Mesh level.  X: nn x 3 reference coordinates; conn: ne x 8 node ids.
 * or_fe_geometry: per-element grad N (ne x 24), volumes, lumped nodal masses.
 */
int or_fe_geometry(int nn, const double *X, int ne, const int *conn, double rho0, double *gradN, double *V0,
                   double *mass) {
    for (int a = 0; a < nn; a++) mass[a] = 0.0;
    for (int e = 0; e < ne; e++) {
        double Xe[24];
        for (int a = 0; a < 8; a++)
            for (int k = 0; k < 3; k++) Xe[3 * a + k] = X[3 * conn[8 * e + a] + k];
        int err = or_hex8_geometry(Xe, gradN + 24 * e, V0 + e);
        if (err) return err;
        for (int a = 0; a < 8; a++) mass[conn[8 * e + a]] += rho0 * V0[e] / 8.0;
    }
    return OR_OK;
}

/* prescribed DOFs: d = lambda * bc_val where bc_mask != 0 (nn x 3 each) */
void or_fe_apply_bc(int nn, const int *bc_mask, const double *bc_val, double lambda, double *d) {
    for (int k = 0; k < 3 * nn; k++)
        if (bc_mask[k]) d[k] = lambda * bc_val[k];
}

/* The same with an affine predictor of the load increment: every free DOF moves
 * by (lambda - lambda_prev) g before the explicit update, the prescribed ones
 * take lambda bc_val (g NULL: no predictor). */
void or_fe_apply_bc_pred(int nn, const int *bc_mask, const double *bc_val, const double *g, double lambda,
                         double dlambda, double *d) {
    for (int k = 0; k < 3 * nn; k++) {
        if (bc_mask[k]) d[k] = lambda * bc_val[k];
        else if (g) d[k] += dlambda * g[k];
    }
}

/* per-element deformation gradients (ne x 9) */
void or_fe_F(int ne, const int *conn, const double *gradN, const double *d, double *F) {
    for (int e = 0; e < ne; e++) {
        double de[24];
        for (int a = 0; a < 8; a++)
            for (int k = 0; k < 3; k++) de[3 * a + k] = d[3 * conn[8 * e + a] + k];
        or_hex8_F(gradN + 24 * e, de, F + 9 * e);
    }
}

/*
 * One explicit step given the element first Piola-Kirchhoff stresses P (ne x 9):
 *   f_int assembled (Eq. f, plus hourglass), a = -f_int / m on free DOFs,
 *   v <- ((1 - c dt/2) v + dt a) / (1 + c dt/2),  d <- d + dt v.
 * Prescribed DOFs keep their displacement; their velocity is set to zero.
 * fint_out (nn x 3, optional) receives the assembled internal force.
 */
void or_fe_update(int nn, const double *X, int ne, const int *conn, const double *gradN, const double *V0,
                  const double *mass, const int *bc_mask, const double *P, double hg_coef, double dt, double damping,
                  double *d, double *vel, double *fint_out) {
    double *fint = (double *)calloc((size_t)3 * nn, sizeof(double));
    for (int e = 0; e < ne; e++) {
        double Xe[24], de[24], fe[24];
        for (int a = 0; a < 8; a++)
            for (int k = 0; k < 3; k++) {
                Xe[3 * a + k] = X[3 * conn[8 * e + a] + k];
                de[3 * a + k] = d[3 * conn[8 * e + a] + k];
            }
        or_hex8_fint(Xe, gradN + 24 * e, V0[e], P + 9 * e, de, hg_coef, fe);
        for (int a = 0; a < 8; a++)
            for (int k = 0; k < 3; k++) fint[3 * conn[8 * e + a] + k] += fe[3 * a + k];
    }
    double c0 = 1.0 - 0.5 * damping * dt, c1 = 1.0 + 0.5 * damping * dt;
    for (int a = 0; a < nn; a++)
        for (int k = 0; k < 3; k++) {
            int q = 3 * a + k;
            if (bc_mask[q]) { vel[q] = 0.0; continue; }
            double acc = -fint[q] / mass[a];
            vel[q] = (c0 * vel[q] + dt * acc) / c1;
            d[q] += dt * vel[q];
        }
    if (fint_out) memcpy(fint_out, fint, sizeof(double) * 3 * (size_t)nn);
    free(fint);
}

/* ------------------------------------------------------------------------ */
/* 4-node tetrahedra, the paper's element (C3D4, Sec. 3.2): linear shape     */
/* functions N = (1 - xi - eta - zeta, xi, eta, zeta), so grad N and F are    */
/* constant in the element; one quadrature point (one r-cell), no hourglass  */
/* modes.  Lumped mass rho0 V / 4 per node; the same explicit update.        */
/* ------------------------------------------------------------------------ */
static const int TET_DN[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};

/* grad_X N_a (4x3) and the volume det J / 6, J_{i alpha} = sum_a X_{a i} dN_a/dxi_alpha */
int or_tet4_geometry(const double *X, double *gradN, double *V0) {
    double J[9] = {0};
    for (int a = 0; a < 4; a++)
        for (int i = 0; i < 3; i++)
            for (int al = 0; al < 3; al++) J[3 * i + al] += X[3 * a + i] * TET_DN[a][al];
    double Ji[9];
    double det = m3_inv(J, Ji);
    if (!(det > 0.0)) return OR_EDEGEN;
    for (int a = 0; a < 4; a++)
        for (int k = 0; k < 3; k++) {
            double s = 0.0;
            for (int al = 0; al < 3; al++) s += Ji[3 * al + k] * TET_DN[a][al];
            gradN[3 * a + k] = s;
        }
    *V0 = det / 6.0;
    return OR_OK;
}

int or_fe_tet_geometry(int nn, const double *X, int ne, const int *conn, double rho0, double *gradN, double *V0,
                       double *mass) {
    for (int a = 0; a < nn; a++) mass[a] = 0.0;
    for (int e = 0; e < ne; e++) {
        double Xe[12];
        for (int a = 0; a < 4; a++)
            for (int k = 0; k < 3; k++) Xe[3 * a + k] = X[3 * conn[4 * e + a] + k];
        int err = or_tet4_geometry(Xe, gradN + 12 * e, V0 + e);
        if (err) return err;
        for (int a = 0; a < 4; a++) mass[conn[4 * e + a]] += rho0 * V0[e] / 4.0;
    }
    return OR_OK;
}

/* F = I + sum_a d_a (x) grad_X N_a per element (ne x 9) */
void or_fe_tet_F(int ne, const int *conn, const double *gradN, const double *d, double *F) {
    for (int e = 0; e < ne; e++)
        for (int i = 0; i < 3; i++)
            for (int J = 0; J < 3; J++) {
                double s = (i == J) ? 1.0 : 0.0;
                for (int a = 0; a < 4; a++) s += d[3 * conn[4 * e + a] + i] * gradN[12 * e + 3 * a + J];
                F[9 * e + 3 * i + J] = s;
            }
}

/* One explicit step (as or_fe_update) with f_int,a = V0 P grad_X N_a (Eq. f) */
void or_fe_tet_update(int nn, int ne, const int *conn, const double *gradN, const double *V0, const double *mass,
                      const int *bc_mask, const double *P, double dt, double damping, double *d, double *vel,
                      double *fint_out) {
    double *fint = (double *)calloc((size_t)3 * nn, sizeof(double));
    for (int e = 0; e < ne; e++)
        for (int a = 0; a < 4; a++)
            for (int i = 0; i < 3; i++) {
                double s = 0.0;
                for (int J = 0; J < 3; J++) s += P[9 * e + 3 * i + J] * gradN[12 * e + 3 * a + J];
                fint[3 * conn[4 * e + a] + i] += V0[e] * s;
            }
    double c0 = 1.0 - 0.5 * damping * dt, c1 = 1.0 + 0.5 * damping * dt;
    for (int a = 0; a < nn; a++)
        for (int k = 0; k < 3; k++) {
            int q = 3 * a + k;
            if (bc_mask[q]) { vel[q] = 0.0; continue; }
            double acc = -fint[q] / mass[a];
            vel[q] = (c0 * vel[q] + dt * acc) / c1;
            d[q] += dt * vel[q];
        }
    if (fint_out) memcpy(fint_out, fint, sizeof(double) * 3 * (size_t)nn);
    free(fint);
}

/* ------------------------------------------------------------------------ */
/* Molecular statics of an r-cell (Sec. 2.2, Eqs. CGPR1-CGPR3 and PK1).      */
/* ------------------------------------------------------------------------ */

/*
 * First Piola-Kirchhoff stress from the pair sum (Eq. PK1 / Eq. CGPR2):
 *   P = 1/(2 Omega_0) sum_{i != j} dE/dr_ij  r_ij (x) R_ij / r_ij,
 * r_ij = x_j - x_i (current, nearest image within rc), R_ij = H0 H^{-1} r_ij
 * the same separation in the reference box H0 (= H(0) S_ij), Omega_0 = det H0.
 * dE/dr_ij is the derivative of the total energy with respect to the pair
 * distance: the pair potential's for LJ / KG, and for Sutton-Chen the pair
 * term plus both embedding contributions.  Kremer-Grest bonds (FENE + WCA)
 * enter once per bond with their bond derivative.  Potential part only (no
 * kinetic term); in the units of the unit system (GPa for metal).  Row-major
 * P[3a+b] = P_ab.
 */
int or_pk1_pairs(const or_pot *P, int units, int n, const double *x, const double *H, const double *H0, int n_bonds,
                 const int *bonds, double *Pk) {
    or_plist L = {0, 0, 0};
    int e = pairs_brute(n, x, H, P->rc, &L);
    if (e) { free(L.p); return e; }
    double Hi[9], M[9];
    m3_inv(H, Hi);
    m3_mul(H0, Hi, M);  /* R_ij = M r_ij */
    double T[9] = {0};  /* sum over ordered pairs of dE/dr r (x) R / r */
    int err = OR_OK;
    or_bondmap B = {0, 0};
    double *rho = NULL;
    if (P->kind == OR_KG) {
        err = bondmap_build(n, n_bonds, bonds, &B);
        if (err) goto done;
    }
    if (P->kind == OR_SC) {
        rho = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
        if (!rho) { err = OR_ENOMEM; goto done; }
        for (long k = 0; k < L.n; k++) rho[L.p[k].i] += pow(P->sigma / sqrt(L.p[k].r2), P->m);
    }
    for (long k = 0; k < L.n; k++) {
        const or_pair *q = &L.p[k];
        if (P->kind == OR_KG && bonded(&B, q->i, q->j)) continue;
        double r = sqrt(q->r2), dEdr;
        if (P->kind == OR_SC) {
            double ar = P->sigma / r;
            dEdr = (P->eps / r) * (-P->n * pow(ar, P->n) +
                                   0.5 * P->c * P->m * (1.0 / sqrt(rho[q->i]) + 1.0 / sqrt(rho[q->j])) * pow(ar, P->m));
        } else {
            double sr6 = pow(P->sigma * P->sigma / q->r2, 3);
            dEdr = -24.0 * P->eps * (2.0 * sr6 * sr6 - sr6) / r;
        }
        double Rv[3];
        m3_mv(M, q->d, Rv);
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) T[3 * a + b] += dEdr * q->d[a] * Rv[b] / r;
    }
    if (P->kind == OR_KG) {
        /* each bond once, with weight 2 against the ordered-pair half */
        double rwca2 = pow(2.0, 1.0 / 3.0) * P->sigma * P->sigma, R02 = P->R0 * P->R0;
        for (int b = 0; b < n_bonds; b++) {
            int i = bonds[2 * b], j = bonds[2 * b + 1];
            double dx[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1], x[3 * j + 2] - x[3 * i + 2]}, ds[3];
            m3_mv(Hi, dx, ds);
            double best = 1e300, bd[3] = {0, 0, 0};
            for (int a0 = -1; a0 <= 1; a0++)
                for (int a1 = -1; a1 <= 1; a1++)
                    for (int a2 = -1; a2 <= 1; a2++) {
                        double t[3] = {a0 - rint(ds[0]), a1 - rint(ds[1]), a2 - rint(ds[2])}, Ht[3];
                        m3_mv(H, t, Ht);
                        double dd[3] = {dx[0] + Ht[0], dx[1] + Ht[1], dx[2] + Ht[2]};
                        double r2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
                        if (r2 < best) { best = r2; bd[0] = dd[0]; bd[1] = dd[1]; bd[2] = dd[2]; }
                    }
            if (!(best < R02)) { err = OR_EBOND; goto done; }
            double r = sqrt(best);
            double dEdr = P->k_fene * r / (1.0 - best / R02);
            if (best < rwca2) {
                double sr6 = pow(P->sigma * P->sigma / best, 3);
                dEdr += -24.0 * P->eps * (2.0 * sr6 * sr6 - sr6) / r;
            }
            double Rv[3];
            m3_mv(M, bd, Rv);
            for (int a = 0; a < 3; a++)
                for (int c = 0; c < 3; c++) T[3 * a + c] += 2.0 * dEdr * bd[a] * Rv[c] / r;
        }
    }
    {
        double s = md_pconv(units) / (2.0 * m3_det(H0));
        for (int k = 0; k < 9; k++) Pk[k] = s * T[k];
    }
done:
    free(L.p);
    free(B.start);
    free(B.nbr);
    free(rho);
    return err;
}

/*
 * Energy minimisation at fixed box (Eq. CGPR1: r_opt = argmin V from the
 * guess r_ge) by FIRE, the fast inertial relaxation engine of Bitzek,
 * Koskinen, Gaehler, Moseler and Gumbsch (Phys. Rev. Lett. 97, 170201, 2006).
 * One iteration, with f = F(x) the forces, |.| norms over the whole cell:
 *   stop if max_i |f_i| < f_tol (converged);
 *   power p = f . v;
 *   p > 0: n_pos += 1; v = (1 - alpha) v + alpha |v| f / |f|;
 *          if n_pos > n_min: dt = min(f_inc dt, dt_max), alpha = f_alpha alpha;
 *   p <= 0: n_pos = 0; v = 0; dt = f_dec dt; alpha = alpha_start;
 *   v += dt f / m;  x += dt v   (semi-implicit Euler step), where an atom whose
 *   move dt |v| would exceed dmax (> 0) has its velocity scaled to move dmax
 *   (a per-atom displacement cap, dmax <= 0: none).
 * Starts from v = 0, dt = dt0, alpha = alpha_start.  Returns the number of
 * force evaluations before convergence in *iters (-1: not converged within
 * max_iter).  x is updated in place; the minimiser's constants are those of
 * the cited paper (n_min 5, f_inc 1.1, f_dec 0.5, alpha_start 0.1, f_alpha 0.99).
 */
int or_fire_minimize(const or_pot *P, int units, double mass, int n, double *x, const double *H, int n_bonds,
                     const int *bonds, double f_tol, double dt0, double dt_max, double dmax, int max_iter, int *iters) {
    const int n_min = 5;
    const double f_inc = 1.1, f_dec = 0.5, alpha_start = 0.1, f_alpha = 0.99;
    double *f = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *v = (double *)calloc(3 * (size_t)(n > 0 ? n : 1), sizeof(double));
    if (!f || !v) { free(f); free(v); return OR_ENOMEM; }
    double fm = md_ftm2v(units) / mass, dt = dt0, alpha = alpha_start;
    int n_pos = 0, err = OR_OK;
    *iters = -1;
    for (int it = 0; it < max_iter; it++) {
        double W[9], pe;
        err = or_forces(P, n, x, H, n_bonds, bonds, 1, f, W, &pe, NULL);
        if (err) break;
        double fmax2 = 0.0, p = 0.0, vv = 0.0, ff = 0.0;
        for (int i = 0; i < n; i++) {
            double f2 = f[3 * i] * f[3 * i] + f[3 * i + 1] * f[3 * i + 1] + f[3 * i + 2] * f[3 * i + 2];
            if (f2 > fmax2) fmax2 = f2;
        }
        if (fmax2 < f_tol * f_tol) { *iters = it; break; }
        for (int k = 0; k < 3 * n; k++) { p += f[k] * v[k]; vv += v[k] * v[k]; ff += f[k] * f[k]; }
        if (p > 0.0) {
            n_pos++;
            double c = alpha * sqrt(vv) / sqrt(ff);
            for (int k = 0; k < 3 * n; k++) v[k] = (1.0 - alpha) * v[k] + c * f[k];
            if (n_pos > n_min) {
                dt = fmin(f_inc * dt, dt_max);
                alpha *= f_alpha;
            }
        } else {
            n_pos = 0;
            for (int k = 0; k < 3 * n; k++) v[k] = 0.0;
            dt *= f_dec;
            alpha = alpha_start;
        }
        for (int i = 0; i < n; i++) {
            for (int a = 0; a < 3; a++) v[3 * i + a] += dt * f[3 * i + a] * fm;
            double s2 = dt * dt * (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2]);
            if (dmax > 0.0 && s2 > dmax * dmax) {
                double sc = dmax / sqrt(s2);
                for (int a = 0; a < 3; a++) v[3 * i + a] *= sc;
            }
            for (int a = 0; a < 3; a++) x[3 * i + a] += dt * v[3 * i + a];
        }
    }
    free(f);
    free(v);
    return err;
}
