// Internal definitions of the GB300 r-cell engine (not part of the C ABI).
//
// Data layout in HBM (one context = a batch of r-cells):
//   * Atoms of all cells live in one padded array; cell c owns the slots
//     [atom_off[c], atom_off[c] + ntile[c]*TILE), of which the first n[c] are
//     real atoms.  A tile of TILE = 128 consecutive slots never spans two
//     cells, so every CTA works for exactly one r-cell.
//   * Positions: float4 {x, y, z, 0}, Cartesian in the cell's triangular MD box
//     (ping-pong pair so one kernel can read x(t) of all neighbours while it
//     writes x(t+dt) of its own atoms).  Velocities: float4 {vx, vy, vz, 0}.
//   * Inside a cell, atoms are kept sorted by neighbour bin (counting sort at
//     every list rebuild); `tag` maps a slot back to the caller's atom index.
//     Bins are at least r_list / 2 wide (in perpendicular width), so the
//     candidates of an atom lie in the 5 x 5 x 5 bins around its own.
//   * Verlet list: per tile, [max_nb/4][TILE] groups of four int32 entries
//     j_global | (image << 27) (one 16-byte load per lane per group, coalesced
//     across the tile); the image code 0..26 selects one of the 27 periodic
//     shift vectors of the cell.
//   * Per-cell FP64 state: box H, stretch R(t-1), Q, R, F of the last
//     deformation, Philox force-evaluation counter, status word.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rcell.h"

#define RC_TILE 128
#define RC_IDX_BITS 27
#define RC_IDX_MASK ((1u << RC_IDX_BITS) - 1u)
#define RC_MAX_BONDS 4
#define RC_MAX_BINS_PER_CELL 8192
#define RC_SAMPLE_W 14  // per-step sample record: K[6], W[6], pe, ke

// per-step force-kernel modes
enum { MODE_EVAL = 0, MODE_SETUP = 1, MODE_STEP = 2, MODE_LAST = 3 };

// Everything a kernel needs, passed by value.
struct KParams {
    int pot;
    int units;
    float eps, sigma, rc2, rlist2, skin_half2, skin2;
    float sc_n, sc_m, sc_c;
    float k_fene, R02, wca2;
    float dt, fm;         // fm = (force -> acceleration) / mass
    float inv_tau;        // 0 when the thermostat is off
    float noise;          // sqrt(2 kT fm_units / (m tau dt))
    float mvv2e;          // m v^2 -> energy units, times mass (per atom)
    uint64_t seed;
    int max_nb;
    float max_step;       // > 0: displacement limit per step
    int n_tiles;          // tiles of RC_TILE atoms in the batch
    int n_sm;             // SMs of the device (tile order of the pair kernels)
    int wait_polls;       // polls of a bounded device-side wait before it gives up
};

struct KArrays {
    // per cell
    const int *cell_n, *cell_off, *tile_cell, *cell_tile0;
    const float *Hf;     // 8 floats per cell: h00 h01 h02 h11 h12 h22 . .
    const float *Hif;    // inverse, same layout
    const int *nbins;    // 4 ints per cell
    const int *bin_off;  // first bin slot per cell
    int *bin_start;      // bin_off[c] .. + nbins+1
    int *status;
    int *need_rebuild, *built;
    unsigned long long *rebuilds;  // per cell: neighbour-list builds so far
    const int *active;   // per cell: 0 = skipped by every MD kernel (state frozen)
    const unsigned long long *evals;
    double *series;      // [cell][slot][RC_SAMPLE_W]
    int series_cap;
    double *eval_acc;    // [cell][8]: pe, W xx yy zz xy xz yz, pad
    // per atom
    float4 *x0, *x1;     // ping-pong
    float4 *v, *xref, *xr, *f;
    int *tag;
    int4 *partner;       // cell-local indices, -1 = none
    int *nbr, *nnb, *bin_of;
    // sort scratch
    float4 *x_tmp, *v_tmp;
    int *tag_tmp, *newpos, *oldidx, *binid;
    int4 *partner_tmp;
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11), from the published round
// definition: words (c0..c3), key (k0,k1); per round
//   (hi0,lo0) = M0*c0, (hi1,lo1) = M1*c2,
//   c <- (hi1^c1^k0, lo1, hi0^c3^k1, lo0), then key += (W0, W1).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 rc_philox(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        unsigned int hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        unsigned int hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// Three standard normals for (tag, cell, force evaluation, seed): uniforms
// u = (k + 1/2) 2^-32 and two Box-Muller pairs, of which three values are used.
__device__ __forceinline__ float3 rc_normals3(unsigned int tag, unsigned int cell, unsigned long long ev,
                                              unsigned long long seed) {
    uint4 o = rc_philox(make_uint4(tag, cell, (unsigned int)ev, (unsigned int)(ev >> 32)),
                        make_uint2((unsigned int)seed, (unsigned int)(seed >> 32)));
    const float s = 2.3283064365386963e-10f, h = 1.1641532182693481e-10f;
    float u0 = fmaf((float)o.x, s, h), u1 = fmaf((float)o.y, s, h);
    float u2 = fmaf((float)o.z, s, h), u3 = fmaf((float)o.w, s, h);
    float r0 = sqrtf(-2.0f * logf(u0)), r1 = sqrtf(-2.0f * logf(u2));
    float s0, c0, s1, c1;
    sincospif(2.0f * u1, &s0, &c0);
    sincospif(2.0f * u3, &s1, &c1);
    return make_float3(r0 * c0, r0 * s0, r1 * c1);
}

__device__ __forceinline__ void rc_set_status(int *status, int cell, int code) { atomicCAS(&status[cell], 0, code); }

// Periodic image shift tables.  The MD box H is stored FP32-exact (the FP64
// box of the deformation is rounded once), so the Cartesian shift
// sh = H (sx, sy, sz) of image (sx, sy, sz), s in {-1, 0, 1}, is exact in FP64
// and split into an FP32 value plus an FP32 remainder `lo` (nonzero only for
// combinations of tilted box vectors).  The displacement x_j + sh - x_i is then
// formed as ((x_j + sn) - (x_i - sp)) + lo with sn = min(sh, 0), sp = max(sh, 0):
// x_j + sn and x_i - sp subtract numbers of similar size (exact), so only the
// final subtraction rounds -- the result is the correctly rounded displacement
// instead of one carrying an error of half an ulp of the box length.
// Per image slot: a = {min(sh,0) (3), lo.x}, b = {max(sh,0) (3), lo.y}; the z
// shift n2 * H_zz is exact in FP32, so lo.z = 0.  Two 16-byte shared loads per pair.
//
// Images are numbered by slot k = (code + 14) mod 27 of the image code
// code = (sx+1) + 3(sy+1) + 9(sz+1): the central image (code 13) is slot 0, so
// a list entry j | k << RC_IDX_BITS of the central image is the bare index j.
struct ShiftTab {
    float4 a[27], b[27];
};

constexpr int RC_SLOT_CENTRAL = 0;
__host__ __device__ __forceinline__ int rc_image_slot(int sx, int sy, int sz) {
    return ((sx + 1) + 3 * (sy + 1) + 9 * (sz + 1) + 14) % 27;
}

__device__ __forceinline__ void rc_build_shift(ShiftTab &T, const float *H, int slot) {
    const int code = (slot + 13) % 27;
    const double sx = (double)(code % 3 - 1), sy = (double)((code / 3) % 3 - 1), sz = (double)(code / 9 - 1);
    const double hx = (double)H[0] * sx + (double)H[1] * sy + (double)H[2] * sz;
    const double hy = (double)H[3] * sy + (double)H[4] * sz;
    const double hz = (double)H[5] * sz;
    const float fx = (float)hx, fy = (float)hy, fz = (float)hz;
    T.a[slot] = make_float4(fminf(fx, 0.f), fminf(fy, 0.f), fminf(fz, 0.f), (float)(hx - fx));
    T.b[slot] = make_float4(fmaxf(fx, 0.f), fmaxf(fy, 0.f), fmaxf(fz, 0.f), (float)(hy - fy));
}

// fill the table from cell c's box (call with all threads; syncs)
__device__ __forceinline__ void rc_load_shifts(ShiftTab &T, float *s_H, const float *Hf, int c) {
    if (threadIdx.x < 6) s_H[threadIdx.x] = Hf[8 * c + threadIdx.x];
    __syncthreads();
    if (threadIdx.x < 27) rc_build_shift(T, s_H, threadIdx.x);
    __syncthreads();
}

// The central image has all-zero table entries, so its displacement is
// x_j - x_i bit for bit (rc_disp_central).  Lists hold their central entries
// first, so the lanes of a warp walk long runs of central entries together.
__device__ __forceinline__ float3 rc_disp(const float4 &xi, const float4 &xj, const ShiftTab &T, int slot) {
    const float4 sa = T.a[slot], sb = T.b[slot];
    return make_float3(((xj.x + sa.x) - (xi.x - sb.x)) + sa.w, ((xj.y + sa.y) - (xi.y - sb.y)) + sb.w,
                       (xj.z + sa.z) - (xi.z - sb.z));
}

// rc_disp with the slot's entries sa = T.a[slot] and xs = {x_i - T.b[slot] (3),
// T.b[slot].w} formed once for several neighbours of the same image slot
__device__ __forceinline__ float3 rc_disp_pre(const float4 &xj, const float4 &sa, const float4 &xs) {
    return make_float3(((xj.x + sa.x) - xs.x) + sa.w, ((xj.y + sa.y) - xs.y) + xs.w, (xj.z + sa.z) - xs.z);
}

__device__ __forceinline__ float3 rc_disp_central(const float4 &xi, const float4 &xj) {
    return make_float3(xj.x - xi.x, xj.y - xi.y, xj.z - xi.z);
}

// Programmatic dependent launch of the MD-step kernels (sort, list, density,
// force): each is launched with programmatic stream serialisation, so that its
// CTAs can be scheduled while the previous kernel of the stream drains, and
// begins with rc_pdl_wait(), which returns once that kernel has completed and
// its memory operations are visible -- before any access to shared state.  It
// then allows its own dependent to be scheduled (rc_pdl_trigger).  Launched
// without the attribute, the wait returns at once.
__device__ __forceinline__ void rc_pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void rc_pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <class... KArgs, class... Args>
void rc_launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                   Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

// per-cell state of the FIRE minimiser (k_fire.cu)
struct FireState {
    double *acc;      // [cell][4]: f.v, |v|^2, |f|^2, pad
    unsigned *fmax2;  // max |f_i|^2 as float bits
    float *dt, *alpha, *mixa, *mixb;
    int *npos, *done, *iters, *it, *zero;
    int *moving;  // per cell: 1 while the cell minimises (stands in for the activity mask meanwhile)
};

// host-side launchers (defined in the kernel translation units)
void rc_launch_sort(const KParams &p, const KArrays &a, int cur, int n_cells, cudaStream_t s);
void rc_launch_nlist(const KParams &p, const KArrays &a, int cur, int n_tiles, cudaStream_t s);
// stage_atoms > 0: every CTA first copies its whole r-cell (stage_atoms = the
// largest cell of the batch) into shared memory and gathers neighbours there
void rc_launch_density(const KParams &p, const KArrays &a, int cur, int n_tiles, int tpa, int stage_atoms,
                       cudaStream_t s);
void rc_launch_force(const KParams &p, const KArrays &a, int cur, int n_tiles, int tpa, int mode, int slot,
                     int step_index, int stage_atoms, cudaStream_t s);
int rc_stage_max_atoms();
void rc_prepare_staged(int max_cell_atoms);
void rc_launch_deform_impl(const double *F, double *H, double *Rprev, double *Q, double *R, double *Fst, double *dR,
                           const double *H0, float *Hf, float *Hif, int *status, int *need_rebuild, int *nbins,
                           const int *bin_cap, const int *active, double rlist, int n_cells, cudaStream_t s);
void rc_launch_remap(const KArrays &a, const double *dR, int cur, int n_tiles, cudaStream_t s);
void rc_launch_stress(const double *series, int n_avg, int series_cap, const double *H, const double *Q,
                      const double *F, double pconv, double *rot_scratch, double *sig_fem, double *sig_se,
                      double *sig_md, double *P, int n_cells, cudaStream_t s);
void rc_launch_static_pk1(const KParams &p, const KArrays &a, int cur, int n_tiles, const float *mcell, double *acc,
                          cudaStream_t s);
void rc_launch_fire_init(const FireState &s, const int *status, const int *active, int n_cells, float dt0,
                         cudaStream_t st);
void rc_launch_fire_zero_v(const KArrays &a, const FireState &s, int n_tiles, int all_cells, cudaStream_t st);
void rc_launch_fire_iteration(const KParams &p, const KArrays &a, int cur, const FireState &s, int n_tiles, int n_cells,
                              float f_tol, float dt_max, float dmax, int *n_left, cudaStream_t st);
void rc_launch_static_prep(const double *H, const double *H0, float *mcell, double *acc, int n_cells,
                           cudaStream_t st);
void rc_launch_static_finish(const double *acc, const double *H0, const double *Q, const double *F, double pconv,
                             double *P, double *sig, const int *status, int n_cells, cudaStream_t st);
void rc_launch_advance(unsigned long long *evals, const int *active, int n_cells, int n, cudaStream_t s);
void rc_launch_keep_frozen(const KArrays &a, int cur_new, int n_tiles, cudaStream_t s);

// finite elements (k_fe.cu)
void fe_launch_geometry(int npe, const double *X, const int *conn, int ne, double rho0, double *gradN, double *V0,
                        double *mass, int *err, cudaStream_t s);
void fe_launch_apply_bc(const int *mask, const double *val, const double *g, double lambda, double dlambda, double *d,
                        int n3, cudaStream_t s);
void fe_launch_F(int npe, const int *conn, const double *gradN, const double *d, double *F, int ne, cudaStream_t s);
void fe_launch_fint(int npe, const double *X, const int *conn, const double *gradN, const double *V0, const double *P,
                    const double *d, double hg, double *fint, int ne, cudaStream_t s);
void fe_launch_update(const int *mask, const double *mass, const double *fint, double dt, double damping,
                      double *d, double *v, int n3, cudaStream_t s);
void fe_launch_surrogate_merge(const int *md_flag, const float *s_sur, const double *F, const double *P_md, double *P,
                               int ne, cudaStream_t s);
void fe_launch_decide(const float *spread, float on, float off, int force_md, int *md_flag, int *n_md, int ne,
                      cudaStream_t s);
void fe_launch_copy_F(const double *F, double *F_prev, int ne, cudaStream_t s);
void fe_launch_replay_mask(const int *md_flag, const int *n_frozen, int j, int *mask, int ne, cudaStream_t s);
void fe_launch_track_frozen(const int *md_flag, const double *F, double *F_hist, int *n_frozen, int ne, int kmax,
                            cudaStream_t s);
