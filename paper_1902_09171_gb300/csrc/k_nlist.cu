// Neighbour-list build for triclinic r-cells (one list per cell, all cells of a
// batch in one launch).
//
//  k_sort  : one CTA per r-cell.  Wraps positions into the current box through
//            fractional coordinates, bins atoms on an n0 x n1 x n2 grid over the
//            fractional cube (n_d = floor(2 w_d / r_list), w_d the perpendicular
//            width: bins at least r_list / 2 wide), counting-sorts them by bin
//            (stable, so the order is deterministic) and permutes every per-atom
//            array.
//  k_nlist : one thread per atom.  Scans the 5 x 5 x 5 bins around its own with
//            explicit periodic image shifts (about 0.58 of the candidates of 27
//            bins r_list wide), a row of five bins as one contiguous range; with
//            n_d >= 2 (w_d >= 2 r_list gives n_d >= 4) the offsets -2..2 map to
//            distinct (bin, image) pairs with images in -1..1, so each (j, image)
//            within r_list is stored exactly once.
#include "rc_internal.cuh"

namespace {

constexpr int SORT_THREADS = 1024, SORT_BATCH = 2;  // atoms per thread whose loads are issued together

// exclusive scan of s[0..n) in place (n <= RC_MAX_BINS_PER_CELL), returns total
__device__ int block_exclusive_scan(int *s, int n) {
    __shared__ int warp_tot[SORT_THREADS / 32];
    const int per = (n + SORT_THREADS - 1) / SORT_THREADS;
    const int lo = threadIdx.x * per;
    int local = 0;
    for (int k = 0; k < per; k++)
        if (lo + k < n) local += s[lo + k];
    // inclusive warp scan of `local`
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int v = local;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += y;
    }
    if (lane == 31) warp_tot[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int w = warp_tot[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += y;
        }
        warp_tot[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    int excl = v - local + (warp > 0 ? warp_tot[warp - 1] : 0);
    int total = warp_tot[31];
    __syncthreads();
    int run = excl;
    for (int k = 0; k < per; k++)
        if (lo + k < n) {
            int c = s[lo + k];
            s[lo + k] = run;
            run += c;
        }
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(SORT_THREADS) k_sort(KParams p, KArrays a, int cur) {
    rc_pdl_wait();
    rc_pdl_trigger();
    const int c = blockIdx.x;
    __shared__ int s_cnt[RC_MAX_BINS_PER_CELL];
    __shared__ int s_go;
    if (threadIdx.x == 0) {
        int go = a.need_rebuild[c] && a.status[c] == 0 && a.active[c];
        a.built[c] = go;
        if (go) {
            a.need_rebuild[c] = 0;
            a.rebuilds[c]++;
        }
        s_go = go;
    }
    __syncthreads();
    if (!s_go) return;

    const int n = a.cell_n[c], off = a.cell_off[c];
    const int nb0 = a.nbins[4 * c], nb1 = a.nbins[4 * c + 1], nb2 = a.nbins[4 * c + 2];
    const int nbt = nb0 * nb1 * nb2;
    const float *H = a.Hf + 8 * c, *Hi = a.Hif + 8 * c;
    const float h00 = H[0], h01 = H[1], h02 = H[2], h11 = H[3], h12 = H[4], h22 = H[5];
    const float i00 = Hi[0], i01 = Hi[1], i02 = Hi[2], i11 = Hi[3], i12 = Hi[4], i22 = Hi[5];
    float4 *X = cur ? a.x1 : a.x0;
    const bool kg = p.pot == RC_POT_KG;

    for (int b = threadIdx.x; b < nbt; b += SORT_THREADS) s_cnt[b] = 0;
    __syncthreads();

    // pass A: wrap, bin, stage a copy of every per-atom array; SORT_BATCH atoms
    // per thread at a time, all their loads issued before any store, so that the
    // loads overlap (the staging arrays are distinct from the sources)
    for (int i0 = threadIdx.x; i0 < n; i0 += SORT_THREADS * SORT_BATCH) {
        float4 xb[SORT_BATCH], vb[SORT_BATCH];
        int tb[SORT_BATCH];
        int4 pb[SORT_BATCH];
#pragma unroll
        for (int k = 0; k < SORT_BATCH; k++) {
            const int i = i0 + k * SORT_THREADS;
            if (i < n) {
                xb[k] = X[off + i];
                vb[k] = a.v[off + i];
                tb[k] = a.tag[off + i];
                if (kg) pb[k] = a.partner[off + i];
            }
        }
#pragma unroll
        for (int k = 0; k < SORT_BATCH; k++) {
            const int i = i0 + k * SORT_THREADS;
            if (i >= n) break;
            const int g = off + i;
            const float4 x = xb[k];
            float s2 = i22 * x.z, s1 = i11 * x.y + i12 * x.z, s0 = i00 * x.x + i01 * x.y + i02 * x.z;
            float f0 = floorf(s0), f1 = floorf(s1), f2 = floorf(s2);
            float w0 = s0 - f0, w1 = s1 - f1, w2 = s2 - f2;
            float xw = x.x - (h00 * f0 + h01 * f1 + h02 * f2);
            float yw = x.y - (h11 * f1 + h12 * f2);
            float zw = x.z - h22 * f2;
            int b0 = min(max((int)(w0 * nb0), 0), nb0 - 1);
            int b1 = min(max((int)(w1 * nb1), 0), nb1 - 1);
            int b2 = min(max((int)(w2 * nb2), 0), nb2 - 1);
            int bin = (b0 * nb1 + b1) * nb2 + b2;
            a.x_tmp[g] = make_float4(xw, yw, zw, 0.0f);
            a.binid[g] = bin;
            a.v_tmp[g] = vb[k];
            a.tag_tmp[g] = tb[k];
            if (kg) a.partner_tmp[g] = pb[k];
            atomicAdd(&s_cnt[bin], 1);
        }
    }
    __syncthreads();

    block_exclusive_scan(s_cnt, nbt);
    int *bs = a.bin_start + a.bin_off[c];
    for (int b = threadIdx.x; b < nbt; b += SORT_THREADS) bs[b] = s_cnt[b];
    if (threadIdx.x == 0) bs[nbt] = n;
    __syncthreads();

    // stable ranking inside bins: one warp walks the atoms in their current
    // order, 32 at a time; the bin ids of the next RANK_BATCH chunks are loaded
    // before the (smem-only) serial pass over them, so that the loads overlap
    if (threadIdx.x < 32) {
        constexpr int RANK_BATCH = 16;
        const int lane = threadIdx.x;
        const unsigned lt = (1u << lane) - 1u;
        for (int base0 = 0; base0 < n; base0 += 32 * RANK_BATCH) {
            int bins[RANK_BATCH];
#pragma unroll
            for (int k = 0; k < RANK_BATCH; k++) {
                const int i = base0 + 32 * k + lane;
                bins[k] = i < n ? a.binid[off + i] : -1 - lane;
            }
#pragma unroll
            for (int k = 0; k < RANK_BATCH; k++) {
                const int i = base0 + 32 * k + lane;
                const bool valid = i < n;
                const int bin = bins[k];
                const unsigned m = __match_any_sync(0xffffffffu, bin);
                const int leader = __ffs(m) - 1;
                int start = 0;
                if (valid && lane == leader) {
                    start = s_cnt[bin];
                    s_cnt[bin] = start + __popc(m);
                }
                start = __shfl_sync(0xffffffffu, start, leader);
                if (valid) a.newpos[off + i] = start + __popc(m & lt);
                __syncwarp();
            }
        }
    }
    __syncthreads();

    // pass B: scatter into sorted order (batched like pass A: the staged
    // arrays are read, the per-atom arrays written)
    for (int i0 = threadIdx.x; i0 < n; i0 += SORT_THREADS * SORT_BATCH) {
        int qb[SORT_BATCH], bb[SORT_BATCH], tb[SORT_BATCH];
        float4 xb[SORT_BATCH], vb[SORT_BATCH];
#pragma unroll
        for (int k = 0; k < SORT_BATCH; k++) {
            const int i = i0 + k * SORT_THREADS;
            if (i < n) {
                const int g = off + i;
                qb[k] = a.newpos[g];
                xb[k] = a.x_tmp[g];
                vb[k] = a.v_tmp[g];
                tb[k] = a.tag_tmp[g];
                bb[k] = a.binid[g];
            }
        }
#pragma unroll
        for (int k = 0; k < SORT_BATCH; k++) {
            const int i = i0 + k * SORT_THREADS;
            if (i >= n) break;
            const int q = off + qb[k];
            X[q] = xb[k];
            a.xref[q] = xb[k];
            a.v[q] = vb[k];
            a.tag[q] = tb[k];
            a.oldidx[q] = i;
            a.bin_of[q] = bb[k];
        }
    }
    if (kg) {
        __syncthreads();
        // bonded partners renumbered: oldidx, partner_tmp and newpos are read,
        // partner written
        for (int i0 = threadIdx.x; i0 < n; i0 += SORT_THREADS * SORT_BATCH) {
            int4 pb[SORT_BATCH];
#pragma unroll
            for (int k = 0; k < SORT_BATCH; k++) {
                const int i = i0 + k * SORT_THREADS;
                if (i < n) pb[k] = a.partner_tmp[off + a.oldidx[off + i]];
            }
#pragma unroll
            for (int k = 0; k < SORT_BATCH; k++) {
                const int i = i0 + k * SORT_THREADS;
                if (i < n) {
                    const int4 pr = pb[k];
                    pb[k] = make_int4(pr.x >= 0 ? a.newpos[off + pr.x] : -1, pr.y >= 0 ? a.newpos[off + pr.y] : -1,
                                      pr.z >= 0 ? a.newpos[off + pr.z] : -1, pr.w >= 0 ? a.newpos[off + pr.w] : -1);
                }
            }
#pragma unroll
            for (int k = 0; k < SORT_BATCH; k++) {
                const int i = i0 + k * SORT_THREADS;
                if (i < n) a.partner[off + i] = pb[k];
            }
        }
    }
}

// compiled for 8 resident CTAs (64 registers): the rebuild is issue-bound, and
// at the 96 registers it takes unbounded only 5 CTAs fit on an SM
__global__ void __launch_bounds__(RC_TILE, 8) k_nlist(KParams p, KArrays a, int cur) {
    rc_pdl_wait();
    rc_pdl_trigger();
    const int t = blockIdx.x;
    const int c = a.tile_cell[t];
    if (!a.built[c]) return;
    __shared__ float s_H[8];
    __shared__ ShiftTab s_tab;
    rc_load_shifts(s_tab, s_H, a.Hf, c);

    const int n = a.cell_n[c], off = a.cell_off[c];
    const int li = (t - a.cell_tile0[c]) * RC_TILE + threadIdx.x;
    const float4 *X = cur ? a.x1 : a.x0;
    // entry k of this atom lives at word 4 * ((t * max_nb/4 + k/4) * TILE + lane) + k%4
    int *nbr = a.nbr + (size_t)t * p.max_nb * RC_TILE + 4 * threadIdx.x;
    int cnt = 0;
    if (li < n) {
        const int g = off + li;
        const float4 xi = X[g];
        const int nb0 = a.nbins[4 * c], nb1 = a.nbins[4 * c + 1], nb2 = a.nbins[4 * c + 2];
        const int bin = a.bin_of[g];
        const int b2 = bin % nb2, b1 = (bin / nb2) % nb1, b0 = bin / (nb1 * nb2);
        const int *bs = a.bin_start + a.bin_off[c];
        int4 pr = make_int4(-1, -1, -1, -1);
        if (p.pot == RC_POT_KG) pr = a.partner[g];
        // two sweeps of the stencil: central-image neighbours first, then the
        // periodic images, so that the lanes of a warp walk long runs of
        // central entries, which skip the shift-table loads.  Bins are numbered
        // with the third index fastest, so the five bins u2 = b2-2..b2+2 of a
        // stencil row are one contiguous range of sorted atoms, split in up to
        // three segments by their image along the third axis: the unwrapped
        // bins (image 0), those wrapped below 0 (image -1) and above nb2 - 1 (+1).
        for (int sweep = 0; sweep < 2; sweep++)
        for (int o0 = -2; o0 <= 2; o0++) {
            int u0 = b0 + o0, s0 = u0 < 0 ? -1 : (u0 >= nb0 ? 1 : 0);
            u0 -= s0 * nb0;
            for (int o1 = -2; o1 <= 2; o1++) {
                int u1 = b1 + o1, s1 = u1 < 0 ? -1 : (u1 >= nb1 ? 1 : 0);
                u1 -= s1 * nb1;
                const int row = (u0 * nb1 + u1) * nb2;
                for (int seg = 0; seg < 3; seg++) {
                    int s2, lo, hi;
                    if (seg == 0) {
                        s2 = 0;
                        lo = max(b2 - 2, 0);
                        hi = min(b2 + 2, nb2 - 1);
                    } else if (seg == 1) {
                        if (b2 >= 2) continue;
                        s2 = -1;
                        lo = nb2 + b2 - 2;
                        hi = nb2 - 1;
                    } else {
                        if (b2 + 2 < nb2) continue;
                        s2 = 1;
                        lo = 0;
                        hi = b2 + 2 - nb2;
                    }
                    const int slot = rc_image_slot(s0, s1, s2);
                    if ((slot == RC_SLOT_CENTRAL) != (sweep == 0)) continue;
                    const int j0 = bs[row + lo], j1 = bs[row + hi + 1];
                    // one shift-table read per segment (it has one image slot); the
                    // candidates' records are loaded NBATCH at a time so that their
                    // loads overlap, then tested in order
                    const float4 sa = s_tab.a[slot], sb = s_tab.b[slot];
                    const float4 xs = make_float4(xi.x - sb.x, xi.y - sb.y, xi.z - sb.z, sb.w);
                    constexpr int NBATCH = 4;
                    for (int jb = j0; jb < j1; jb += NBATCH) {
                        float4 xj[NBATCH];
#pragma unroll
                        for (int k = 0; k < NBATCH; k++) xj[k] = X[off + (jb + k < j1 ? jb + k : j1 - 1)];
#pragma unroll
                        for (int k = 0; k < NBATCH; k++) {
                            const int jl = jb + k;
                            if (jl >= j1) break;
                            const float3 d = rc_disp_pre(xj[k], sa, xs);
                            const float r2 = fmaf(d.x, d.x, fmaf(d.y, d.y, d.z * d.z));
                            // the atom itself and its bond partners are left out; tested on the
                            // quarter of the candidates inside r_list only
                            if (r2 < p.rlist2 && !(jl == li && slot == RC_SLOT_CENTRAL) &&
                                !(jl == pr.x || jl == pr.y || jl == pr.z || jl == pr.w)) {
                                if (cnt < p.max_nb)
                                    nbr[(size_t)(cnt >> 2) * (4 * RC_TILE) + (cnt & 3)] =
                                        (int)((unsigned)(off + jl) | ((unsigned)slot << RC_IDX_BITS));
                                cnt++;
                            }
                        }
                    }
                }
            }
        }
        if (cnt > p.max_nb) {
            rc_set_status(a.status, c, RC_EOVERFLOW);
            cnt = p.max_nb;
        }
    }
    a.nnb[off + li] = cnt;
}

}  // namespace

void rc_launch_sort(const KParams &p, const KArrays &a, int cur, int n_cells, cudaStream_t s) {
    rc_launch_pdl(k_sort, n_cells, SORT_THREADS, 0, s, p, a, cur);
}

void rc_launch_nlist(const KParams &p, const KArrays &a, int cur, int n_tiles, cudaStream_t s) {
    rc_launch_pdl(k_nlist, n_tiles, RC_TILE, 0, s, p, a, cur);
}
