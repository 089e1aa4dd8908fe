// Force evaluation fused with the velocity-Verlet / Langevin update and the
// per-cell virial reduction -- one launch per MD step (two for Sutton-Chen,
// whose embedding term needs every rho_i before any force).
//
// Thread mapping: a CTA owns one tile of RC_TILE atoms of one r-cell; TPA
// consecutive lanes share one atom and split its Verlet list (TPA in 1,2,4,8),
// combining their partial sums with xor-shuffles.  Neighbour positions are
// gathered as float4 (16-byte, read-only path); atoms of a cell are stored
// bin-sorted, so the gathers of a warp hit a few L1/L2 lines.
//
// Arithmetic: pair math in FP32 (fused multiply-adds); per-atom virial and
// energy partials in FP32; per-warp sums promoted to FP64 before the per-cell
// atomic accumulation.
//
// Per step (mode STEP): f(t) from x(t); v(t) = v(t-dt/2) + dt/2 a(t) with
// a = f/m - v/tau + noise (Langevin friction on the velocity held at force
// time); sample K = sum m v(t) (x) v(t), W(t), PE(t); then v(t+dt/2) = v(t) +
// dt/2 a(t), x(t+dt) = x(t) + dt v(t+dt/2) written to the other position
// buffer, and the skin test that schedules the next neighbour rebuild.
#include "rc_internal.cuh"

namespace {

// lanes that share one atom: TPA, or 1 for the lean walk (TPA == 0)
__host__ __device__ constexpr int lanes_of(int tpa) { return tpa > 0 ? tpa : 1; }

template <int TPA>
__device__ __forceinline__ float sub_sum(float v) {
#pragma unroll
    for (int d = 1; d < TPA; d <<= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

// Where neighbour records come from: the global array through the read-only
// path, or the whole r-cell staged in shared memory (index minus cell offset).
struct GlobalSrc {
    const float4 *__restrict__ p;
    __device__ __forceinline__ float4 operator()(unsigned j) const { return __ldg(p + j); }
};
struct SharedSrc {
    const float4 *p;
    int off;
    __device__ __forceinline__ float4 operator()(unsigned j) const { return p[(int)j - off]; }
};

// Largest cell (in atoms) whose records are staged in shared memory.
constexpr int RC_STAGE_MAX_ATOMS = 12800;  // 200 KB of float4
constexpr unsigned RC_STAGE_CHUNK = 32768;  // bytes per bulk copy
constexpr int RC_SPIN_LIMIT = 1 << 22;

// Copy n float4 records (16-byte aligned) from global memory into shared memory
// with TMA bulk copies that complete on one mbarrier; every thread waits with a
// bounded spin of `polls` polls.  On a timeout the cell is flagged RC_ETIMEOUT
// and false returned, after a second wait (RC_SPIN_LIMIT polls, independent of
// `polls`) for the copies already issued, so that none is in flight when the
// CTA leaves.
__device__ __forceinline__ bool stage_records(float4 *dst, const float4 *src, int n, int *status, int c, int polls) {
    __shared__ __align__(8) unsigned long long s_bar;
    const unsigned bar = (unsigned)__cvta_generic_to_shared(&s_bar);
    const unsigned bytes = (unsigned)n * 16u;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        const unsigned d0 = (unsigned)__cvta_generic_to_shared(dst);
        for (unsigned o = 0; o < bytes; o += RC_STAGE_CHUNK) {
            const unsigned sz = min(RC_STAGE_CHUNK, bytes - o);
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d0 + o),
                "l"(reinterpret_cast<const char *>(src) + o), "r"(sz), "r"(bar)
                : "memory");
        }
    }
    unsigned done = 0;
    for (int it = 0; it < polls && !done; it++)
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar)
            : "memory");
    // the whole block agrees, so that either every thread goes on or every thread leaves
    if (__syncthreads_and(done)) return true;
    if (threadIdx.x == 0) rc_set_status(status, c, RC_ETIMEOUT);
    for (int it = 0; it < RC_SPIN_LIMIT && !done; it++)  // let a late copy land before leaving
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar)
            : "memory");
    __syncthreads();
    return false;
}

// Slots of a list group past the end of the list hold stale data: point them at
// the group's first entry, which is always valid, so that they can be gathered.
// List groups are read once per pass: loaded without allocating in L1, which
// then keeps the neighbour records that the atoms of a tile share.
__device__ __forceinline__ int4 ld_list(const int4 *p) {
    int4 v;
    asm("ld.global.nc.L1::no_allocate.v4.s32 {%0, %1, %2, %3}, [%4];"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p));
    return v;
}

// Tile order of the pair kernels.  The grid is padded to a multiple R of the
// SM count S, and block b takes tile (b mod S) R + b / S: blocks b, b + S,
// b + 2S, ... -- those that the first wave deals to one SM -- get consecutive
// tiles, the spatial neighbours of one r-cell, whose shared neighbour records
// then stay in that SM's L1.  Blocks past the last tile return at once.
__device__ __forceinline__ int tile_of_block(int n_sm) {
    const int R = (int)gridDim.x / n_sm;
    return (int)(blockIdx.x % n_sm) * R + (int)(blockIdx.x / n_sm);
}
inline unsigned pair_grid(const KParams &p) {
    return (unsigned)(((p.n_tiles + p.n_sm - 1) / p.n_sm) * p.n_sm);
}

__device__ __forceinline__ int4 clamp_group(int4 e, int left) {
    if (left < 4) {
        if (left < 2) e.y = e.x;
        if (left < 3) e.z = e.x;
        e.w = e.x;
    }
    return e;
}

// Displacements and pair evaluations of one list group (entries e, records
// c0..c3, `left` entries of the list from this group on).  Warp-uniform fast
// paths for full groups: all four entries of the image slot 0 (the central
// image: x_j - x_i, the bits rc_disp gives for it) in every converged lane, or
// one image slot per lane's group (the runs of a stencil bin): one shift-table
// read and one x_i - sp per group instead of one per entry, the same arithmetic
// as rc_disp.
template <class Fn>
__device__ __forceinline__ void eval_group(const int4 &e, int left, const float4 &c0, const float4 &c1,
                                           const float4 &c2, const float4 &c3, const float4 &xi, const ShiftTab &T,
                                           Fn &&fn) {
    const unsigned s0 = (unsigned)e.x >> RC_IDX_BITS;
    const bool one_slot =
        left >= 4 && (((unsigned)(e.x ^ e.y) | (unsigned)(e.x ^ e.z) | (unsigned)(e.x ^ e.w)) >> RC_IDX_BITS) == 0;
    const unsigned am = __activemask();
    float3 d0, d1, d2, d3;
    if (__all_sync(am, one_slot && s0 == RC_SLOT_CENTRAL)) {
        d0 = rc_disp_central(xi, c0);
        d1 = rc_disp_central(xi, c1);
        d2 = rc_disp_central(xi, c2);
        d3 = rc_disp_central(xi, c3);
    } else if (__all_sync(am, one_slot)) {
        const float4 sa = T.a[s0], sb = T.b[s0];
        const float4 xs = make_float4(xi.x - sb.x, xi.y - sb.y, xi.z - sb.z, sb.w);
        d0 = rc_disp_pre(c0, sa, xs);
        d1 = rc_disp_pre(c1, sa, xs);
        d2 = rc_disp_pre(c2, sa, xs);
        d3 = rc_disp_pre(c3, sa, xs);
    } else {  // mixed image slots, or the list's last, partial group (whose missing
              // entries repeat its first one: valid indices, results unused)
        d0 = rc_disp(xi, c0, T, s0);
        d1 = rc_disp(xi, c1, T, (unsigned)e.y >> RC_IDX_BITS);
        d2 = rc_disp(xi, c2, T, (unsigned)e.z >> RC_IDX_BITS);
        d3 = rc_disp(xi, c3, T, (unsigned)e.w >> RC_IDX_BITS);
    }
    if (left >= 4) {
        fn(c0, d0);
        fn(c1, d1);
        fn(c2, d2);
        fn(c3, d3);
    } else {
        fn(c0, d0);
        if (left > 1) fn(c1, d1);
        if (left > 2) fn(c2, d2);
    }
}

// Walk one atom's Verlet list (this lane's share: groups sub, sub+TPA, ... of
// four entries).  Each group is one 16-byte load.  The loop is software
// pipelined: while the pairs of group g are evaluated, the four neighbour
// records of the next group are already being gathered and the list entries of
// the group after that are being loaded, so the gather latency overlaps the
// pair arithmetic.  fn(xj, d) receives the neighbour's record and the exact
// periodic displacement d = x_j(image) - x_i.
// TPA == 0 is the lean walk: one lane per atom, one group at a time with no
// pipelining -- fewer registers, so that more warps per SM hide the latency
// instead (the force kernel is compiled for 10 resident CTAs then, the density
// kernel for 12), which pays when the batch has enough tiles to fill them.
template <int TPA, class Src, class Fn>
__device__ __forceinline__ void for_each_neighbor(const int4 *__restrict__ nb4, int nn, int sub, const Src &src,
                                                  const float4 &xi, const ShiftTab &T, Fn &&fn) {
    const int ng = (nn + 3) >> 2;
    if constexpr (TPA == 0) {
        for (int g = 0; g < ng; g++) {
            // the list streams from DRAM: ask L2 for the group after next now, so
            // that its load finds it there (no register holds it meanwhile)
            if (g + 2 < ng) asm volatile("prefetch.global.L2 [%0];" ::"l"(nb4 + (size_t)(g + 2) * RC_TILE));
            const int left = nn - 4 * g;
            const int4 e = clamp_group(ld_list(nb4 + (size_t)g * RC_TILE), left);
            const float4 c0 = src((unsigned)e.x & RC_IDX_MASK), c1 = src((unsigned)e.y & RC_IDX_MASK);
            const float4 c2 = src((unsigned)e.z & RC_IDX_MASK), c3 = src((unsigned)e.w & RC_IDX_MASK);
            eval_group(e, left, c0, c1, c2, c3, xi, T, fn);
        }
        return;
    }
    int g = sub;
    if (g >= ng) return;
    int4 e = clamp_group(ld_list(nb4 + (size_t)g * RC_TILE), nn - 4 * g);
    float4 c0 = src((unsigned)e.x & RC_IDX_MASK), c1 = src((unsigned)e.y & RC_IDX_MASK);
    float4 c2 = src((unsigned)e.z & RC_IDX_MASK), c3 = src((unsigned)e.w & RC_IDX_MASK);
    int gn = g + TPA;
    int4 en = e;
    if (gn < ng) en = ld_list(nb4 + (size_t)gn * RC_TILE);
    while (true) {
        const int gnn = gn + TPA;
        float4 n0 = c0, n1 = c1, n2 = c2, n3 = c3;
        int4 enn = en;
        if (gn < ng) {  // next stage: gather group gn, load the entries of group gnn
            en = clamp_group(en, nn - 4 * gn);
            n0 = src((unsigned)en.x & RC_IDX_MASK);
            n1 = src((unsigned)en.y & RC_IDX_MASK);
            n2 = src((unsigned)en.z & RC_IDX_MASK);
            n3 = src((unsigned)en.w & RC_IDX_MASK);
            if (gnn < ng) enn = ld_list(nb4 + (size_t)gnn * RC_TILE);
        }
        const int left = nn - 4 * g;
        // Warp-uniform fast paths for full groups: all four entries of the image
        // slot 0 (the central image: x_j - x_i, the bits rc_disp gives for it) in
        // every converged lane, or one image slot per lane's group (the runs of a
        // stencil bin): one shift-table read and one x_i - sp per group instead of
        // one per entry, the same arithmetic as rc_disp.
        const unsigned s0 = (unsigned)e.x >> RC_IDX_BITS;
        const bool one_slot =
            left >= 4 && (((unsigned)(e.x ^ e.y) | (unsigned)(e.x ^ e.z) | (unsigned)(e.x ^ e.w)) >> RC_IDX_BITS) == 0;
        const unsigned am = __activemask();
        float3 d0, d1, d2, d3;
        if (__all_sync(am, one_slot && s0 == RC_SLOT_CENTRAL)) {
            d0 = rc_disp_central(xi, c0);
            d1 = rc_disp_central(xi, c1);
            d2 = rc_disp_central(xi, c2);
            d3 = rc_disp_central(xi, c3);
        } else if (__all_sync(am, one_slot)) {
            const float4 sa = T.a[s0], sb = T.b[s0];
            const float4 xs = make_float4(xi.x - sb.x, xi.y - sb.y, xi.z - sb.z, sb.w);
            d0 = rc_disp_pre(c0, sa, xs);
            d1 = rc_disp_pre(c1, sa, xs);
            d2 = rc_disp_pre(c2, sa, xs);
            d3 = rc_disp_pre(c3, sa, xs);
        } else {  // mixed image slots, or the list's last, partial group (whose missing
                  // entries repeat its first one: valid indices, results unused)
            d0 = rc_disp(xi, c0, T, s0);
            d1 = rc_disp(xi, c1, T, (unsigned)e.y >> RC_IDX_BITS);
            d2 = rc_disp(xi, c2, T, (unsigned)e.z >> RC_IDX_BITS);
            d3 = rc_disp(xi, c3, T, (unsigned)e.w >> RC_IDX_BITS);
        }
        if (left >= 4) {
            fn(c0, d0);
            fn(c1, d1);
            fn(c2, d2);
            fn(c3, d3);
        } else {
            fn(c0, d0);
            if (left > 1) fn(c1, d1);
            if (left > 2) fn(c2, d2);
        }
        if (gn >= ng) break;
        g = gn;
        gn = gnn;
        e = en;
        en = enn;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
}

// Sutton-Chen density pass: rho_i = sum_j (a/r_ij)^m over r < rc; writes
// xr_i = {x_i, rho_i^{-1/2}} for the force pass.
// resident CTAs per SM the density pass is compiled for (a register cap of
// 65536 / (128 x this) at one lane per atom): 12 for the lean walk, else 7 --
// a 128 000-atom batch (1000 tiles) in one wave on 152 SMs
constexpr int density_min_ctas(int tpa) { return tpa == 0 ? 12 : (7 / tpa > 0 ? 7 / tpa : 1); }

template <int TPA, bool M6, bool STG>
__global__ void __launch_bounds__(RC_TILE *lanes_of(TPA), density_min_ctas(TPA)) k_density(KParams p, KArrays a, int cur) {
    extern __shared__ __align__(16) float4 s_cell[];
    rc_pdl_wait();
    rc_pdl_trigger();
    const int t = tile_of_block(p.n_sm);
    if (t >= p.n_tiles) return;
    const int c = a.tile_cell[t];
    if (a.status[c] != 0 || !a.active[c]) return;
    __shared__ ShiftTab s_tab;
    __shared__ float s_H[8];
    rc_load_shifts(s_tab, s_H, a.Hf, c);

    const int at = threadIdx.x / lanes_of(TPA), sub = threadIdx.x % lanes_of(TPA);
    const int n = a.cell_n[c], off = a.cell_off[c];
    const int li = (t - a.cell_tile0[c]) * RC_TILE + at;
    const float4 *__restrict__ X = cur ? a.x1 : a.x0;
    if (STG && !stage_records(s_cell, X + off, n, a.status, c, p.wait_polls)) return;
    const bool live = li < n;
    const int g = off + li;
    float rho = 0.0f;
    float4 xi = make_float4(0.f, 0.f, 0.f, 0.f);
    if (live) {
        xi = X[g];
        const int nn = a.nnb[g];
        const int4 *__restrict__ nb = reinterpret_cast<const int4 *>(a.nbr) + (size_t)t * (p.max_nb / 4) * RC_TILE + at;
        const float a2 = p.sigma * p.sigma, hm = 0.5f * p.sc_m;
        const float rc2 = p.rc2;
        auto body = [&](const float4 &, const float3 &d) {
            const float r2 = fmaf(d.x, d.x, fmaf(d.y, d.y, d.z * d.z));
            if (r2 < rc2) {
                const float ar2 = a2 * __fdividef(1.0f, r2);
                rho += M6 ? ar2 * ar2 * ar2 : powf(ar2, hm);
            }
        };
        if (STG) for_each_neighbor<TPA>(nb, nn, sub, SharedSrc{s_cell, off}, xi, s_tab, body);
        else for_each_neighbor<TPA>(nb, nn, sub, GlobalSrc{X}, xi, s_tab, body);
    }
    rho = sub_sum<TPA>(rho);
    if (live && sub == 0) a.xr[g] = make_float4(xi.x, xi.y, xi.z, rho > 0.0f ? rsqrtf(rho) : 0.0f);
}

// Block reduction of NV per-atom float values into FP64, then one atomicAdd per
// value into dst[0..NV).
template <int NV, int NT>
__device__ __forceinline__ void block_reduce_add(float (&v)[NV], double *dst) {
    __shared__ double s_part[NT / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        float x = v[k];
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
        if (lane == 0) s_part[warp][k] = (double)x;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < NT / 32; w++) s += s_part[w][threadIdx.x];
        atomicAdd(dst + threadIdx.x, s);
    }
}

// Resident CTAs per SM the force kernel is compiled for at one lane per atom
// (caps its registers at 65536 / (128 * RC_FORCE_MIN_CTAS)).  7 keeps a
// 128 000-atom batch (1000 tiles) in one wave on 152 SMs; 1 leaves the
// register count to the compiler.  The lean walk takes 10 (48 registers): on
// the 80 000 tiles of a 10.24 M-bead batch, 12 (40 registers, with spills) ran
// the force step 3 % and the sampling step 7 % slower, 8 and 9 (no spills)
// 4-6 % and 1-3 % slower.
#ifndef RC_FORCE_MIN_CTAS
#define RC_FORCE_MIN_CTAS 7
#endif
constexpr int force_min_ctas(int tpa) {
    return tpa == 0 ? 10 : (RC_FORCE_MIN_CTAS / tpa > 0 ? RC_FORCE_MIN_CTAS / tpa : 1);
}

// SAMPLE: this launch records a stress sample (slot >= 0) or evaluates the
// energy and virial (MODE_EVAL); without it the pair loop skips the virial and
// energy terms, which only feed those records.
template <int POT, int TPA, bool M6, bool STG, bool SAMPLE>
__global__ void __launch_bounds__(RC_TILE *lanes_of(TPA), force_min_ctas(TPA)) k_force(KParams p, KArrays a, int cur, int mode, int slot,
                                                       int step_index) {
    extern __shared__ __align__(16) float4 s_cell[];
    rc_pdl_wait();
    rc_pdl_trigger();
    const int t = tile_of_block(p.n_sm);
    if (t >= p.n_tiles) return;
    const int c = a.tile_cell[t];
    if (a.status[c] != 0 || !a.active[c]) return;
    __shared__ ShiftTab s_tab;
    __shared__ float s_H[8];
    rc_load_shifts(s_tab, s_H, a.Hf, c);

    const int at = threadIdx.x / lanes_of(TPA), sub = threadIdx.x % lanes_of(TPA);
    const int n = a.cell_n[c], off = a.cell_off[c];
    const int li = (t - a.cell_tile0[c]) * RC_TILE + at;
    const bool live = li < n;
    const int g = off + li;
    const float4 *__restrict__ X = cur ? a.x1 : a.x0;
    const float4 *__restrict__ XG = (POT == RC_POT_SC) ? a.xr : X;  // gathered array
    if (STG && !stage_records(s_cell, XG + off, n, a.status, c, p.wait_polls)) return;

    float fx = 0.f, fy = 0.f, fz = 0.f;
    float w0 = 0.f, w1 = 0.f, w2 = 0.f, w3 = 0.f, w4 = 0.f, w5 = 0.f;  // xx yy zz xy xz yz
    float pe = 0.f;
    float4 xi = make_float4(0.f, 0.f, 0.f, 0.f);
    if (live) {
        xi = XG[g];
        const int nn = a.nnb[g];
        const int4 *__restrict__ nb = reinterpret_cast<const int4 *>(a.nbr) + (size_t)t * (p.max_nb / 4) * RC_TILE + at;
        if (POT == RC_POT_SC) {
            const float a2 = p.sigma * p.sigma, hm = 0.5f * p.sc_m, hn = 0.5f * p.sc_n;
            const float cm2 = 0.5f * p.sc_c * p.sc_m;
            const float rc2 = p.rc2, eps = p.eps, sc_n = p.sc_n, sig = p.sigma;
            auto body = [&](const float4 &xj, const float3 &d) {
                const float dx = d.x, dy = d.y, dz = d.z;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                if (r2 < rc2) {
                    const float ir2 = __fdividef(1.0f, r2);
                    const float ar2 = a2 * ir2;
                    float arm, arn;
                    if (M6) {
                        arm = ar2 * ar2 * ar2;               // (a/r)^6
                        arn = arm * ar2 * (sig * rsqrtf(r2));  // (a/r)^9
                    } else {
                        arm = powf(ar2, hm);
                        arn = powf(ar2, hn);
                    }
                    // dE/dr / r = eps / r^2 [ -n (a/r)^n + c m/2 (rho_i^-1/2 + rho_j^-1/2) (a/r)^m ]
                    const float gr = eps * ir2 * fmaf(cm2 * (xi.w + xj.w), arm, -sc_n * arn);
                    const float gx = gr * dx, gy = gr * dy, gz = gr * dz;
                    fx += gx;
                    fy += gy;
                    fz += gz;
                    if (SAMPLE) {  // scaled once per atom after the walk: W by -1/2, pe by eps/2
                        w0 = fmaf(gx, dx, w0);
                        w1 = fmaf(gy, dy, w1);
                        w2 = fmaf(gz, dz, w2);
                        w3 = fmaf(gx, dy, w3);
                        w4 = fmaf(gx, dz, w4);
                        w5 = fmaf(gy, dz, w5);
                        pe += arn;
                    }
                }
            };
            if (STG) for_each_neighbor<TPA>(nb, nn, sub, SharedSrc{s_cell, off}, xi, s_tab, body);
            else for_each_neighbor<TPA>(nb, nn, sub, GlobalSrc{XG}, xi, s_tab, body);
            if (SAMPLE) pe *= 0.5f * eps;
        } else {
            const float s2 = p.sigma * p.sigma;
            const float c24 = 24.0f * p.eps, c2 = 2.0f * p.eps;
            const float rc2 = p.rc2;
            auto body = [&](const float4 &, const float3 &d) {
                const float dx = d.x, dy = d.y, dz = d.z;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                if (r2 < rc2) {
                    const float ir2 = __fdividef(1.0f, r2);
                    const float sr2 = s2 * ir2;
                    const float sr6 = sr2 * sr2 * sr2;
                    // dU/dr / r = -24 eps (2 (s/r)^12 - (s/r)^6) / r^2
                    const float gr = -c24 * ir2 * sr6 * (2.0f * sr6 - 1.0f);
                    const float gx = gr * dx, gy = gr * dy, gz = gr * dz;
                    fx += gx;
                    fy += gy;
                    fz += gz;
                    if (SAMPLE) {  // scaled once per atom after the walk: W by -1/2, pe by 2 eps
                        w0 = fmaf(gx, dx, w0);
                        w1 = fmaf(gy, dy, w1);
                        w2 = fmaf(gz, dz, w2);
                        w3 = fmaf(gx, dy, w3);
                        w4 = fmaf(gx, dz, w4);
                        w5 = fmaf(gy, dz, w5);
                        pe = fmaf(sr6, sr6 - 1.0f, pe);  // 1/2 * 4 eps (sr12 - sr6) / (2 eps)
                    }
                }
            };
            if (STG) for_each_neighbor<TPA>(nb, nn, sub, SharedSrc{s_cell, off}, xi, s_tab, body);
            else for_each_neighbor<TPA>(nb, nn, sub, GlobalSrc{XG}, xi, s_tab, body);
            if (SAMPLE) pe *= c2;
        }
        if (SAMPLE) {
            w0 *= -0.5f;
            w1 *= -0.5f;
            w2 *= -0.5f;
            w3 *= -0.5f;
            w4 *= -0.5f;
            w5 *= -0.5f;
        }
    }
    fx = sub_sum<TPA>(fx);
    fy = sub_sum<TPA>(fy);
    fz = sub_sum<TPA>(fz);
    if (SAMPLE) {
        w0 = sub_sum<TPA>(w0);
        w1 = sub_sum<TPA>(w1);
        w2 = sub_sum<TPA>(w2);
        w3 = sub_sum<TPA>(w3);
        w4 = sub_sum<TPA>(w4);
        w5 = sub_sum<TPA>(w5);
        pe = sub_sum<TPA>(pe);
    }
    const bool own = live && sub == 0;

    if (own && POT == RC_POT_SC && xi.w > 0.0f) pe -= p.eps * p.sc_c / xi.w;  // embedding -eps c sqrt(rho_i)

    if (own && POT == RC_POT_KG) {
        // FENE + WCA on the (at most four) bond partners; each bond is seen from
        // both ends, so each end takes half of the virial and energy.
        const int4 pr = a.partner[g];
        const int q[4] = {pr.x, pr.y, pr.z, pr.w};
        const float *Hi = a.Hif + 8 * c;
#pragma unroll
        for (int b = 0; b < RC_MAX_BONDS; b++) {
            if (q[b] < 0) continue;
            const float4 xj = STG ? s_cell[q[b]] : X[off + q[b]];
            // minimum image: pick the integer shift from fractional coordinates, then
            // form the displacement through the exact shift table
            const float ex = xj.x - xi.x, ey = xj.y - xi.y, ez = xj.z - xi.z;
            const float f2 = Hi[5] * ez, f1 = Hi[3] * ey + Hi[4] * ez, f0 = Hi[0] * ex + Hi[1] * ey + Hi[2] * ez;
            const int n0 = -(int)rintf(f0), n1 = -(int)rintf(f1), n2 = -(int)rintf(f2);
            if (n0 < -1 || n0 > 1 || n1 < -1 || n1 > 1 || n2 < -1 || n2 > 1) {
                rc_set_status(a.status, c, RC_EBOND);
                continue;
            }
            const float3 dd = rc_disp(xi, xj, s_tab, rc_image_slot(n0, n1, n2));
            const float dx = dd.x, dy = dd.y, dz = dd.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (!(r2 < p.R02)) {
                rc_set_status(a.status, c, RC_EBOND);
                continue;
            }
            const float ratio = r2 / p.R02;
            float gr = p.k_fene / (1.0f - ratio);
            float U = -0.5f * p.k_fene * p.R02 * log1pf(-ratio);
            if (r2 < p.wca2) {
                const float sr2 = p.sigma * p.sigma / r2, sr6 = sr2 * sr2 * sr2;
                gr -= 24.0f * p.eps * sr6 * (2.0f * sr6 - 1.0f) / r2;
                U += 4.0f * p.eps * sr6 * (sr6 - 1.0f) + p.eps;
            }
            fx = fmaf(gr, dx, fx);
            fy = fmaf(gr, dy, fy);
            fz = fmaf(gr, dz, fz);
            const float hx = -0.5f * gr * dx, hy = -0.5f * gr * dy;
            w0 = fmaf(hx, dx, w0);
            w1 = fmaf(hy, dy, w1);
            w2 = fmaf(-0.5f * gr * dz, dz, w2);
            w3 = fmaf(hx, dy, w3);
            w4 = fmaf(hx, dz, w4);
            w5 = fmaf(hy, dz, w5);
            pe += 0.5f * U;
        }
    }

    if (mode == MODE_EVAL) {
        if (own) a.f[g] = make_float4(fx, fy, fz, pe);
        float v[7] = {own ? pe : 0.f, own ? w0 : 0.f, own ? w1 : 0.f, own ? w2 : 0.f,
                      own ? w3 : 0.f, own ? w4 : 0.f, own ? w5 : 0.f};
        block_reduce_add<7, RC_TILE * lanes_of(TPA)>(v, a.eval_acc + 8 * c);
        return;
    }

    // ---- velocity Verlet + Langevin ----
    float kxx = 0.f, kyy = 0.f, kzz = 0.f, kxy = 0.f, kxz = 0.f, kyz = 0.f;
    if (own) {
        float4 vv = a.v[g];
        float ax = fx * p.fm, ay = fy * p.fm, az = fz * p.fm;
        if (p.inv_tau > 0.0f) {
            const float3 z = rc_normals3((unsigned)a.tag[g], (unsigned)c, a.evals[c] + (unsigned long long)step_index,
                                         p.seed);
            ax += fmaf(-vv.x, p.inv_tau, p.noise * z.x);
            ay += fmaf(-vv.y, p.inv_tau, p.noise * z.y);
            az += fmaf(-vv.z, p.inv_tau, p.noise * z.z);
        }
        const float hdt = 0.5f * p.dt;
        if (mode != MODE_SETUP) {  // complete v(t)
            vv.x = fmaf(hdt, ax, vv.x);
            vv.y = fmaf(hdt, ay, vv.y);
            vv.z = fmaf(hdt, az, vv.z);
            kxx = p.mvv2e * vv.x * vv.x;
            kyy = p.mvv2e * vv.y * vv.y;
            kzz = p.mvv2e * vv.z * vv.z;
            kxy = p.mvv2e * vv.x * vv.y;
            kxz = p.mvv2e * vv.x * vv.z;
            kyz = p.mvv2e * vv.y * vv.z;
        }
        if (mode == MODE_LAST) {
            a.v[g] = vv;
        } else {
            vv.x = fmaf(hdt, ax, vv.x);
            vv.y = fmaf(hdt, ay, vv.y);
            vv.z = fmaf(hdt, az, vv.z);
            if (p.max_step > 0.0f) {
                const float s2 = p.dt * p.dt * (vv.x * vv.x + vv.y * vv.y + vv.z * vv.z);
                if (s2 > p.max_step * p.max_step) {
                    const float f = p.max_step * rsqrtf(s2);
                    vv.x *= f;
                    vv.y *= f;
                    vv.z *= f;
                }
            }
            float4 xn = make_float4(fmaf(p.dt, vv.x, xi.x), fmaf(p.dt, vv.y, xi.y), fmaf(p.dt, vv.z, xi.z), 0.0f);
            a.v[g] = vv;
            (cur ? a.x0 : a.x1)[g] = xn;
            const float4 xr0 = a.xref[g];
            const float ddx = xn.x - xr0.x, ddy = xn.y - xr0.y, ddz = xn.z - xr0.z;
            const float d2 = ddx * ddx + ddy * ddy + ddz * ddz;
            if (d2 > p.skin_half2) a.need_rebuild[c] = 1;
            const float step2 = p.dt * p.dt * (vv.x * vv.x + vv.y * vv.y + vv.z * vv.z);
            if (!(step2 <= p.skin_half2)) rc_set_status(a.status, c, isfinite(step2) ? RC_ELOST : RC_ENAN);
        }
    }
    if (slot >= 0) {
        float v[13] = {kxx, kyy, kzz, kxy, kxz, kyz,
                       own ? w0 : 0.f, own ? w1 : 0.f, own ? w2 : 0.f, own ? w3 : 0.f, own ? w4 : 0.f, own ? w5 : 0.f,
                       own ? pe : 0.f};
        block_reduce_add<13, RC_TILE * lanes_of(TPA)>(v, a.series + ((size_t)c * a.series_cap + slot) * RC_SAMPLE_W);
    }
}

// Eq. PK1 (Sec. 2.2): per cell, the sum over ordered pairs inside rc of
// dE/dr_ij r_ij (x) R_ij / r_ij with R_ij = M r_ij, M = H(0) H^{-1} (upper
// triangular, m[6] per cell: m00 m01 m02 m11 m12 m22), plus the Kremer-Grest
// bonds, each seen from both ends.  FP32 per atom, FP64 per cell into
// acc[9 c + 3 a + b]; the caller scales by 1 / (2 Omega_0).
template <int POT, bool M6>
__global__ void __launch_bounds__(RC_TILE) k_static_pk1(KParams p, KArrays a, int cur, const float *__restrict__ mcell,
                                                        double *acc) {
    const int t = blockIdx.x;
    const int c = a.tile_cell[t];
    if (a.status[c] != 0 || !a.active[c]) return;
    __shared__ ShiftTab s_tab;
    __shared__ float s_H[8];
    rc_load_shifts(s_tab, s_H, a.Hf, c);
    const float *m = mcell + 6 * c;
    const float m00 = m[0], m01 = m[1], m02 = m[2], m11 = m[3], m12 = m[4], m22 = m[5];
    const int n = a.cell_n[c], off = a.cell_off[c];
    const int li = (t - a.cell_tile0[c]) * RC_TILE + threadIdx.x;
    const int g = off + li;
    const float4 *__restrict__ X = cur ? a.x1 : a.x0;
    const float4 *__restrict__ XG = (POT == RC_POT_SC) ? a.xr : X;
    float T[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    auto add = [&](float gr, const float3 &d) {  // gr = dE/dr / r
        const float R0 = fmaf(m00, d.x, fmaf(m01, d.y, m02 * d.z)), R1 = fmaf(m11, d.y, m12 * d.z), R2 = m22 * d.z;
        const float gx = gr * d.x, gy = gr * d.y, gz = gr * d.z;
        T[0] = fmaf(gx, R0, T[0]); T[1] = fmaf(gx, R1, T[1]); T[2] = fmaf(gx, R2, T[2]);
        T[3] = fmaf(gy, R0, T[3]); T[4] = fmaf(gy, R1, T[4]); T[5] = fmaf(gy, R2, T[5]);
        T[6] = fmaf(gz, R0, T[6]); T[7] = fmaf(gz, R1, T[7]); T[8] = fmaf(gz, R2, T[8]);
    };
    if (li < n) {
        const float4 xi = XG[g];
        const int nn = a.nnb[g];
        const int4 *__restrict__ nb =
            reinterpret_cast<const int4 *>(a.nbr) + (size_t)t * (p.max_nb / 4) * RC_TILE + threadIdx.x;
        const float rc2 = p.rc2;
        if (POT == RC_POT_SC) {
            const float a2 = p.sigma * p.sigma, hm = 0.5f * p.sc_m, hn = 0.5f * p.sc_n;
            const float cm2 = 0.5f * p.sc_c * p.sc_m, eps = p.eps, sc_n = p.sc_n, sig = p.sigma;
            for_each_neighbor<1>(nb, nn, 0, GlobalSrc{XG}, xi, s_tab, [&](const float4 &xj, const float3 &d) {
                const float r2 = fmaf(d.x, d.x, fmaf(d.y, d.y, d.z * d.z));
                if (r2 < rc2) {
                    const float ir2 = __fdividef(1.0f, r2), ar2 = a2 * ir2;
                    float arm, arn;
                    if (M6) {
                        arm = ar2 * ar2 * ar2;
                        arn = arm * ar2 * (sig * rsqrtf(r2));
                    } else {
                        arm = powf(ar2, hm);
                        arn = powf(ar2, hn);
                    }
                    add(eps * ir2 * fmaf(cm2 * (xi.w + xj.w), arm, -sc_n * arn), d);
                }
            });
        } else {
            const float s2 = p.sigma * p.sigma, c24 = 24.0f * p.eps;
            for_each_neighbor<1>(nb, nn, 0, GlobalSrc{XG}, xi, s_tab, [&](const float4 &, const float3 &d) {
                const float r2 = fmaf(d.x, d.x, fmaf(d.y, d.y, d.z * d.z));
                if (r2 < rc2) {
                    const float ir2 = __fdividef(1.0f, r2), sr2 = s2 * ir2, sr6 = sr2 * sr2 * sr2;
                    add(-c24 * ir2 * sr6 * (2.0f * sr6 - 1.0f), d);
                }
            });
        }
        if (POT == RC_POT_KG) {
            const int4 pr = a.partner[g];
            const int q[4] = {pr.x, pr.y, pr.z, pr.w};
            const float *Hi = a.Hif + 8 * c;
#pragma unroll
            for (int b = 0; b < RC_MAX_BONDS; b++) {
                if (q[b] < 0) continue;
                const float4 xj = X[off + q[b]];
                const float ex = xj.x - xi.x, ey = xj.y - xi.y, ez = xj.z - xi.z;
                const float f2 = Hi[5] * ez, f1 = Hi[3] * ey + Hi[4] * ez, f0 = Hi[0] * ex + Hi[1] * ey + Hi[2] * ez;
                const int n0 = -(int)rintf(f0), n1 = -(int)rintf(f1), n2 = -(int)rintf(f2);
                if (n0 < -1 || n0 > 1 || n1 < -1 || n1 > 1 || n2 < -1 || n2 > 1) continue;
                const float3 dd = rc_disp(xi, xj, s_tab, rc_image_slot(n0, n1, n2));
                const float r2 = fmaf(dd.x, dd.x, fmaf(dd.y, dd.y, dd.z * dd.z));
                if (!(r2 < p.R02)) continue;
                float gr = p.k_fene / (1.0f - r2 / p.R02);
                if (r2 < p.wca2) {
                    const float sr2 = p.sigma * p.sigma / r2, sr6 = sr2 * sr2 * sr2;
                    gr -= 24.0f * p.eps * sr6 * (2.0f * sr6 - 1.0f) / r2;
                }
                add(gr, dd);
            }
        }
    }
    block_reduce_add<9, RC_TILE>(T, acc + 9 * c);
}

template <class K>
void set_smem(K kernel, int bytes) {
    if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <int POT, bool M6, bool STG, bool SAMPLE>
void launch_force_tpa(const KParams &p, const KArrays &a, int cur, int n_tiles, int tpa, int mode, int slot,
                      int step_index, int smem, cudaStream_t s) {
    switch (tpa) {
    case 0: rc_launch_pdl(k_force<POT, 0, M6, STG, SAMPLE>, pair_grid(p), RC_TILE * 1, smem, s, p, a, cur, mode, slot, step_index); break;
    case 1: rc_launch_pdl(k_force<POT, 1, M6, STG, SAMPLE>, pair_grid(p), RC_TILE * 1, smem, s, p, a, cur, mode, slot, step_index); break;
    case 2: rc_launch_pdl(k_force<POT, 2, M6, STG, SAMPLE>, pair_grid(p), RC_TILE * 2, smem, s, p, a, cur, mode, slot, step_index); break;
    case 4: rc_launch_pdl(k_force<POT, 4, M6, STG, SAMPLE>, pair_grid(p), RC_TILE * 4, smem, s, p, a, cur, mode, slot, step_index); break;
    default: rc_launch_pdl(k_force<POT, 8, M6, STG, SAMPLE>, pair_grid(p), RC_TILE * 8, smem, s, p, a, cur, mode, slot, step_index); break;
    }
}

template <int POT, bool M6, bool STG>
void launch_force_pot(const KParams &p, const KArrays &a, int cur, int n_tiles, int tpa, int mode, int slot,
                      int step_index, int smem, cudaStream_t s) {
    if (slot >= 0 || mode == MODE_EVAL)
        launch_force_tpa<POT, M6, STG, true>(p, a, cur, n_tiles, tpa, mode, slot, step_index, smem, s);
    else
        launch_force_tpa<POT, M6, STG, false>(p, a, cur, n_tiles, tpa, mode, slot, step_index, smem, s);
}

template <bool M6, bool STG>
void launch_density_m(const KParams &p, const KArrays &a, int cur, int n_tiles, int tpa, int smem, cudaStream_t s) {
    switch (tpa) {
    case 0: rc_launch_pdl(k_density<0, M6, STG>, pair_grid(p), RC_TILE * 1, smem, s, p, a, cur); break;
    case 1: rc_launch_pdl(k_density<1, M6, STG>, pair_grid(p), RC_TILE * 1, smem, s, p, a, cur); break;
    case 2: rc_launch_pdl(k_density<2, M6, STG>, pair_grid(p), RC_TILE * 2, smem, s, p, a, cur); break;
    case 4: rc_launch_pdl(k_density<4, M6, STG>, pair_grid(p), RC_TILE * 4, smem, s, p, a, cur); break;
    default: rc_launch_pdl(k_density<8, M6, STG>, pair_grid(p), RC_TILE * 8, smem, s, p, a, cur); break;
    }
}

template <int POT, bool M6, bool SAMPLE>
void prepare_pot_s(int bytes) {
    set_smem(k_force<POT, 0, M6, true, SAMPLE>, bytes);
    set_smem(k_force<POT, 1, M6, true, SAMPLE>, bytes);
    set_smem(k_force<POT, 2, M6, true, SAMPLE>, bytes);
    set_smem(k_force<POT, 4, M6, true, SAMPLE>, bytes);
    set_smem(k_force<POT, 8, M6, true, SAMPLE>, bytes);
}

template <int POT, bool M6>
void prepare_pot(int bytes) {
    prepare_pot_s<POT, M6, true>(bytes);
    prepare_pot_s<POT, M6, false>(bytes);
}

template <bool M6>
void prepare_density(int bytes) {
    set_smem(k_density<0, M6, true>, bytes);
    set_smem(k_density<1, M6, true>, bytes);
    set_smem(k_density<2, M6, true>, bytes);
    set_smem(k_density<4, M6, true>, bytes);
    set_smem(k_density<8, M6, true>, bytes);
}

}  // namespace

int rc_stage_max_atoms() { return RC_STAGE_MAX_ATOMS; }

void rc_prepare_staged(int max_cell_atoms) {
    const int bytes = max_cell_atoms * 16;
    prepare_pot<RC_POT_SC, true>(bytes);
    prepare_pot<RC_POT_SC, false>(bytes);
    prepare_pot<RC_POT_LJ, false>(bytes);
    prepare_pot<RC_POT_KG, false>(bytes);
    prepare_density<true>(bytes);
    prepare_density<false>(bytes);
}

void rc_launch_density(const KParams &p, const KArrays &a, int cur, int n_tiles, int tpa, int stage_atoms,
                       cudaStream_t s) {
    const int smem = stage_atoms * 16;
    if (stage_atoms > 0) {
        if (p.sc_m == 6.0f) launch_density_m<true, true>(p, a, cur, n_tiles, tpa, smem, s);
        else launch_density_m<false, true>(p, a, cur, n_tiles, tpa, smem, s);
    } else {
        if (p.sc_m == 6.0f) launch_density_m<true, false>(p, a, cur, n_tiles, tpa, 0, s);
        else launch_density_m<false, false>(p, a, cur, n_tiles, tpa, 0, s);
    }
}

void rc_launch_force(const KParams &p, const KArrays &a, int cur, int n_tiles, int tpa, int mode, int slot,
                     int step_index, int stage_atoms, cudaStream_t s) {
    const bool m69 = p.sc_m == 6.0f && p.sc_n == 9.0f;
    const int smem = stage_atoms * 16;
    const bool st = stage_atoms > 0;
    if (p.pot == RC_POT_SC) {
        if (m69) {
            if (st) launch_force_pot<RC_POT_SC, true, true>(p, a, cur, n_tiles, tpa, mode, slot, step_index, smem, s);
            else launch_force_pot<RC_POT_SC, true, false>(p, a, cur, n_tiles, tpa, mode, slot, step_index, 0, s);
        } else {
            if (st) launch_force_pot<RC_POT_SC, false, true>(p, a, cur, n_tiles, tpa, mode, slot, step_index, smem, s);
            else launch_force_pot<RC_POT_SC, false, false>(p, a, cur, n_tiles, tpa, mode, slot, step_index, 0, s);
        }
    } else if (p.pot == RC_POT_KG) {
        if (st) launch_force_pot<RC_POT_KG, false, true>(p, a, cur, n_tiles, tpa, mode, slot, step_index, smem, s);
        else launch_force_pot<RC_POT_KG, false, false>(p, a, cur, n_tiles, tpa, mode, slot, step_index, 0, s);
    } else {
        if (st) launch_force_pot<RC_POT_LJ, false, true>(p, a, cur, n_tiles, tpa, mode, slot, step_index, smem, s);
        else launch_force_pot<RC_POT_LJ, false, false>(p, a, cur, n_tiles, tpa, mode, slot, step_index, 0, s);
    }
}

void rc_launch_static_pk1(const KParams &p, const KArrays &a, int cur, int n_tiles, const float *mcell, double *acc,
                          cudaStream_t s) {
    if (p.pot == RC_POT_SC) {
        if (p.sc_m == 6.0f && p.sc_n == 9.0f) k_static_pk1<RC_POT_SC, true><<<n_tiles, RC_TILE, 0, s>>>(p, a, cur, mcell, acc);
        else k_static_pk1<RC_POT_SC, false><<<n_tiles, RC_TILE, 0, s>>>(p, a, cur, mcell, acc);
    } else if (p.pot == RC_POT_KG) {
        k_static_pk1<RC_POT_KG, false><<<n_tiles, RC_TILE, 0, s>>>(p, a, cur, mcell, acc);
    } else {
        k_static_pk1<RC_POT_LJ, false><<<n_tiles, RC_TILE, 0, s>>>(p, a, cur, mcell, acc);
    }
}
