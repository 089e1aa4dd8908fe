// C ABI of the r-cell engine: context set-up, device memory, the per-step
// launch sequence (captured into CUDA graphs), and host accessors.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/surrogate.h"
#include "rc_internal.cuh"

namespace {

// unit conversions from CODATA 2018 constants (metal: eV, Angstrom, ps, amu)
const double kEV = 1.602176634e-19, kAMU = 1.66053906660e-27;
double ftm2v_of(int units) { return units == RC_UNITS_METAL ? kEV / (1e-10 * kAMU) / 1e14 : 1.0; }
double pconv_of(int units) { return units == RC_UNITS_METAL ? kEV / 1e-30 / 1e9 : 1.0; }

}  // namespace

struct rcell_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    rcell_params prm{};
    KParams kp{};
    KArrays ka{};
    int n_cells = 0, n_tiles = 0;
    long n_pad = 0, n_atoms = 0;
    double rlist = 0.0;
    std::vector<int> h_n, h_off, h_tile0, h_ntiles, h_bin_off;
    std::vector<void *> allocs;
    // per-cell device state not in KArrays
    double *d_H = nullptr, *d_H0 = nullptr, *d_Rprev = nullptr, *d_Q = nullptr, *d_R = nullptr, *d_F = nullptr;
    double *d_dR = nullptr, *d_Fin = nullptr;
    float *d_Hf = nullptr, *d_Hif = nullptr;
    int *d_nbins = nullptr, *d_bin_cap = nullptr;
    unsigned long long *d_evals = nullptr;
    double *d_sig_fem = nullptr, *d_sig_se = nullptr, *d_sig_md = nullptr, *d_P = nullptr;
    double *d_rot = nullptr;  // stress reduction scratch, n_cells x series_cap x 6
    int series_cap = 0;
    int last_n_avg = -1;
    int cur = 0;
    int tpa = 1;
    int use_graphs = 1;
    int max_cell = 0;    // largest cell of the batch (atoms)
    int max_nb_alloc = 0;  // neighbour-list entries per atom allocated at creation
    int staged = 0;      // stage whole cells in shared memory (when they fit) -- off by default
    long launches_last = 0;
    // molecular statics (allocated on first use)
    FireState fire{};
    int *d_fire_left = nullptr;
    cudaGraphExec_t fire_graph = nullptr;  // one captured batch of FIRE iterations
    double fire_key[5] = {0, 0, 0, 0, 0};   // f_tol, dt_max, dmax, tpa, cur it was captured with
    float *d_mcell = nullptr;
    double *d_pk_acc = nullptr;
    std::map<std::tuple<int, int, int, int>, cudaGraphExec_t> graphs;
    std::map<std::tuple<int, int, int, int>, long> graph_launches;
    std::string err = "ok";
};

struct fe_ctx {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int nn = 0, ne = 0;
    int npe = 8;  // nodes per element: 8 (hexahedra) or 4 (tetrahedra)
    double rho0 = 0, dt = 0, damping = 0, hg = 0;
    std::vector<void *> allocs;
    double *d_X = nullptr, *d_val = nullptr, *d_gradN = nullptr, *d_V0 = nullptr, *d_mass = nullptr;
    double *d_g = nullptr;    // affine predictor of the load increment (nullptr: none)
    double *d_g_buf = nullptr;
    double lam_last = 0.0;    // load factor of the last boundary-condition update
    double *d_d = nullptr, *d_v = nullptr, *d_fint = nullptr, *d_F = nullptr, *d_P = nullptr;
    int *d_conn = nullptr, *d_mask = nullptr, *d_err = nullptr;
    cudaEvent_t ev = nullptr;
    // surrogate-coupled steps (allocated on first use)
    float *d_u = nullptr, *d_smean = nullptr, *d_spread = nullptr;
    double *d_Pmd = nullptr;
    int *d_nmd = nullptr;
    // per point: deformation gradients of the increments missed while on the
    // surrogate ([RC_REPLAY_MAX][ne][9]), their count, and a replay mask
    double *d_Fhist = nullptr;
    int *d_nfrozen = nullptr, *d_rmask = nullptr;
    std::vector<int> h_flag, h_nfrozen;
    std::string err = "ok";
};

namespace {

template <class T>
cudaError_t dalloc(std::vector<void *> &lst, T **p, size_t count) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    lst.push_back(q);
    *p = static_cast<T *>(q);
    return cudaMemset(q, 0, std::max<size_t>(count, 1) * sizeof(T));
}

int fail(rcell_ctx *c, int code, const std::string &why) {
    if (c) c->err = why;
    return code;
}

#define CKC(ctx, call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) return fail(ctx, RC_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

void free_graphs(rcell_ctx *c) {
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
    c->graph_launches.clear();
    if (c->fire_graph) cudaGraphExecDestroy(c->fire_graph);
    c->fire_graph = nullptr;
}

int first_status(rcell_ctx *c) {
    std::vector<int> st(c->n_cells);
    CKC(c, cudaStreamSynchronize(c->stream));
    CKC(c, cudaMemcpy(st.data(), c->ka.status, sizeof(int) * c->n_cells, cudaMemcpyDeviceToHost));
    for (int i = 0; i < c->n_cells; i++)
        if (st[i] != 0) {
            char buf[96];
            snprintf(buf, sizeof buf, "cell %d reported status %d", i, st[i]);
            c->err = buf;
            return st[i];
        }
    return RC_OK;
}

int stage_atoms(const rcell_ctx *c) {
    return (c->staged && c->max_cell <= rc_stage_max_atoms()) ? c->max_cell : 0;
}

// enqueue the neighbour rebuild (when scheduled) and the force launches of one
// step; returns the number of kernels enqueued
long enqueue_step(rcell_ctx *c, int mode, int slot, int step_index) {
    long k = 0;
    rc_launch_sort(c->kp, c->ka, c->cur, c->n_cells, c->stream);
    rc_launch_nlist(c->kp, c->ka, c->cur, c->n_tiles, c->stream);
    k += 2;
    if (c->kp.pot == RC_POT_SC) {
        rc_launch_density(c->kp, c->ka, c->cur, c->n_tiles, c->tpa, stage_atoms(c), c->stream);
        k++;
    }
    rc_launch_force(c->kp, c->ka, c->cur, c->n_tiles, c->tpa, mode, slot, step_index, stage_atoms(c), c->stream);
    k++;
    return k;
}

long enqueue_run(rcell_ctx *c, int n_steps, int n_avg) {
    long k = 0;
    cudaMemsetAsync(c->ka.series, 0, sizeof(double) * (size_t)c->n_cells * c->series_cap * RC_SAMPLE_W, c->stream);
    for (int s = 0; s <= n_steps; s++) {
        const int mode = s == 0 ? MODE_SETUP : (s == n_steps ? MODE_LAST : MODE_STEP);
        const int slot = (s > 0 && s > n_steps - n_avg) ? s - (n_steps - n_avg) - 1 : -1;
        k += enqueue_step(c, mode, slot, s);
        if (mode != MODE_LAST) c->cur ^= 1;
    }
    if (n_steps & 1) {  // frozen cells: their positions into the buffer that is current now
        rc_launch_keep_frozen(c->ka, c->cur, c->n_tiles, c->stream);
        k++;
    }
    rc_launch_advance(c->d_evals, c->ka.active, c->n_cells, n_steps + 1, c->stream);
    return k + 1;
}

int ensure_series(rcell_ctx *c, int n_avg) {
    if (n_avg <= c->series_cap && c->ka.series) return RC_OK;
    int cap = std::max(n_avg, 256);
    double *p = nullptr;
    CKC(c, cudaStreamSynchronize(c->stream));
    double *rot = nullptr;
    CKC(c, cudaMalloc(&p, sizeof(double) * (size_t)c->n_cells * cap * RC_SAMPLE_W));
    CKC(c, cudaMalloc(&rot, sizeof(double) * (size_t)c->n_cells * cap * 6));
    for (void *old : {(void *)c->ka.series, (void *)c->d_rot}) {
        if (!old) continue;
        auto it = std::find(c->allocs.begin(), c->allocs.end(), old);
        if (it != c->allocs.end()) c->allocs.erase(it);
        cudaFree(old);
    }
    c->allocs.push_back(p);
    c->allocs.push_back(rot);
    c->d_rot = rot;
    c->ka.series = p;
    c->ka.series_cap = cap;
    c->series_cap = cap;
    free_graphs(c);  // graphs hold the old pointer
    return RC_OK;
}

}  // namespace

extern "C" {

int rcell_create(const rcell_params *params, int n_cells, const rcell_init *cells, void *stream, rcell_ctx **out) {
    if (!params || !cells || !out || n_cells <= 0) return RC_EINVAL;
    *out = nullptr;
    const rcell_params &P = *params;
    if (P.potential < RC_POT_LJ || P.potential > RC_POT_KG) return RC_EINVAL;
    if (!(P.rc > 0) || !(P.skin >= 0) || !(P.mass > 0) || !(P.dt > 0) || !(P.sigma > 0)) return RC_EINVAL;
    if (P.potential == RC_POT_KG && !(P.R0 > 0)) return RC_EINVAL;
    rcell_ctx *c = new rcell_ctx();
    c->prm = P;
    c->n_cells = n_cells;
    c->rlist = P.rc + P.skin;
    CKC(c, cudaGetDevice(&c->device));
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        CKC(c, cudaStreamCreate(&c->stream));
        c->own_stream = true;
    }
    // ---- layout: tiles, offsets, bins, capacities ----
    c->h_n.resize(n_cells);
    c->h_off.resize(n_cells);
    c->h_tile0.resize(n_cells);
    c->h_ntiles.resize(n_cells);
    c->h_bin_off.resize(n_cells);
    std::vector<int> bin_cap(n_cells);
    double rho_max = 0.0;
    long tiles = 0, bins = 0;
    for (int i = 0; i < n_cells; i++) {
        const rcell_init &ci = cells[i];
        if (ci.n_atoms <= 0 || !ci.H0 || !ci.x0) { rcell_destroy(c); return RC_EINVAL; }
        // non-finite inputs are refused before anything reaches the device
        bool finite = true;
        for (int k = 0; k < 9; k++) finite = finite && std::isfinite(ci.H0[k]);
        for (long k = 0; k < 3L * ci.n_atoms; k++) {
            finite = finite && std::isfinite(ci.x0[k]);
            if (ci.v0) finite = finite && std::isfinite(ci.v0[k]);
        }
        if (!finite) { rcell_destroy(c); return RC_EINVAL; }
        if (ci.H0[3] != 0.0 || ci.H0[6] != 0.0 || ci.H0[7] != 0.0) { rcell_destroy(c); return RC_EINVAL; }
        const double V = ci.H0[0] * ci.H0[4] * ci.H0[8];
        if (!(V > 0)) { rcell_destroy(c); return RC_EINVAL; }
        rho_max = std::max(rho_max, ci.n_atoms / V);
        c->h_n[i] = ci.n_atoms;
        c->max_cell = std::max(c->max_cell, ci.n_atoms);
        c->h_ntiles[i] = (ci.n_atoms + RC_TILE - 1) / RC_TILE;
        c->h_tile0[i] = (int)tiles;
        c->h_off[i] = (int)(tiles * RC_TILE);
        tiles += c->h_ntiles[i];
        // allocation planning: bins of the initial box (widths of an upper-triangular H)
        const double a = ci.H0[0], b = ci.H0[1], cc = ci.H0[2], d = ci.H0[4], e = ci.H0[5], f = ci.H0[8];
        const double i00 = 1 / a, i01 = -b / (a * d), i02 = (b * e - cc * d) / (a * d * f), i11 = 1 / d,
                     i12 = -e / (d * f), i22 = 1 / f;
        const double w[3] = {1 / std::sqrt(i00 * i00 + i01 * i01 + i02 * i02), 1 / std::sqrt(i11 * i11 + i12 * i12),
                             1 / std::fabs(i22)};
        long prod = 1;
        for (int k = 0; k < 3; k++) prod *= std::max(1L, (long)std::floor(2.0 * w[k] / c->rlist));
        bin_cap[i] = (int)std::min<long>(RC_MAX_BINS_PER_CELL, std::max<long>(64, 3 * prod));
        c->h_bin_off[i] = (int)bins;
        bins += bin_cap[i] + 1;
        c->n_atoms += ci.n_atoms;
    }
    if (tiles * RC_TILE >= (long)RC_IDX_MASK) { rcell_destroy(c); return RC_EINVAL; }
    c->n_tiles = (int)tiles;
    c->n_pad = tiles * RC_TILE;
    const double est = rho_max * 4.0 / 3.0 * M_PI * c->rlist * c->rlist * c->rlist;
    int max_nb = (int)std::ceil(1.6 * est + 32);
    max_nb = (max_nb + 7) / 8 * 8;

    if (c->max_cell <= rc_stage_max_atoms()) rc_prepare_staged(c->max_cell);
    // ---- kernel parameters ----
    KParams &kp = c->kp;
    const double ftm2v = ftm2v_of(P.units);
    kp.pot = P.potential;
    kp.units = P.units;
    kp.eps = (float)P.eps;
    kp.sigma = (float)P.sigma;
    kp.rc2 = (float)(P.rc * P.rc);
    kp.rlist2 = (float)(c->rlist * c->rlist);
    kp.skin_half2 = (float)(0.25 * P.skin * P.skin);
    kp.skin2 = (float)(P.skin * P.skin);
    kp.sc_n = (float)P.n;
    kp.sc_m = (float)P.m;
    kp.sc_c = (float)P.c;
    kp.k_fene = (float)P.k_fene;
    kp.R02 = (float)(P.R0 * P.R0);
    kp.wca2 = (float)(std::pow(2.0, 1.0 / 3.0) * P.sigma * P.sigma);
    kp.dt = (float)P.dt;
    kp.fm = (float)(ftm2v / P.mass);
    kp.inv_tau = P.tau > 0 ? (float)(1.0 / P.tau) : 0.0f;
    kp.noise = P.tau > 0 ? (float)std::sqrt(2.0 * P.kT * ftm2v / (P.mass * P.tau * P.dt)) : 0.0f;
    kp.mvv2e = (float)(P.mass / ftm2v);
    kp.seed = P.seed;
    kp.max_nb = max_nb;
    c->max_nb_alloc = max_nb;
    kp.wait_polls = RC_WAIT_POLLS_DEFAULT;
    kp.n_tiles = c->n_tiles;
    kp.n_sm = 1;
    CKC(c, cudaDeviceGetAttribute(&kp.n_sm, cudaDevAttrMultiProcessorCount, c->device));
    if (kp.n_sm < 1) kp.n_sm = 1;
    kp.max_step = P.max_step > 0 ? (float)P.max_step : 0.0f;

    // ---- device memory ----
    KArrays &A = c->ka;
    auto &L = c->allocs;
    const size_t N = (size_t)c->n_pad;
    int *d_cell_n, *d_cell_off, *d_tile_cell, *d_cell_tile0, *d_bin_off;
    CKC(c, dalloc(L, &d_cell_n, n_cells));
    CKC(c, dalloc(L, &d_cell_off, n_cells));
    CKC(c, dalloc(L, &d_tile_cell, tiles));
    CKC(c, dalloc(L, &d_cell_tile0, n_cells));
    CKC(c, dalloc(L, &d_bin_off, n_cells));
    CKC(c, dalloc(L, &c->d_nbins, 4 * (size_t)n_cells));
    CKC(c, dalloc(L, &c->d_bin_cap, n_cells));
    CKC(c, dalloc(L, &A.bin_start, (size_t)bins));
    CKC(c, dalloc(L, &A.status, n_cells));
    CKC(c, dalloc(L, &A.need_rebuild, n_cells));
    CKC(c, dalloc(L, &A.built, n_cells));
    CKC(c, dalloc(L, &A.rebuilds, n_cells));
    int *d_active = nullptr;
    CKC(c, dalloc(L, &d_active, n_cells));
    {
        std::vector<int> ones(n_cells, 1);
        CKC(c, cudaMemcpy(d_active, ones.data(), sizeof(int) * n_cells, cudaMemcpyHostToDevice));
    }
    A.active = d_active;
    CKC(c, dalloc(L, &c->d_evals, n_cells));
    CKC(c, dalloc(L, &A.eval_acc, 8 * (size_t)n_cells));
    CKC(c, dalloc(L, &c->d_H, 9 * (size_t)n_cells));
    CKC(c, dalloc(L, &c->d_H0, 9 * (size_t)n_cells));
    CKC(c, dalloc(L, &c->d_Rprev, 9 * (size_t)n_cells));
    CKC(c, dalloc(L, &c->d_Q, 9 * (size_t)n_cells));
    CKC(c, dalloc(L, &c->d_R, 9 * (size_t)n_cells));
    CKC(c, dalloc(L, &c->d_F, 9 * (size_t)n_cells));
    CKC(c, dalloc(L, &c->d_dR, 9 * (size_t)n_cells));
    CKC(c, dalloc(L, &c->d_Fin, 9 * (size_t)n_cells));
    CKC(c, dalloc(L, &c->d_Hf, 8 * (size_t)n_cells));
    CKC(c, dalloc(L, &c->d_Hif, 8 * (size_t)n_cells));
    CKC(c, dalloc(L, &c->d_sig_fem, 6 * (size_t)n_cells));
    CKC(c, dalloc(L, &c->d_sig_se, 6 * (size_t)n_cells));
    CKC(c, dalloc(L, &c->d_sig_md, 6 * (size_t)n_cells));
    CKC(c, dalloc(L, &c->d_P, 9 * (size_t)n_cells));
    CKC(c, dalloc(L, &A.x0, N));
    CKC(c, dalloc(L, &A.x1, N));
    CKC(c, dalloc(L, &A.v, N));
    CKC(c, dalloc(L, &A.xref, N));
    CKC(c, dalloc(L, &A.xr, N));
    CKC(c, dalloc(L, &A.f, N));
    CKC(c, dalloc(L, &A.tag, N));
    CKC(c, dalloc(L, &A.partner, N));
    CKC(c, dalloc(L, &A.nnb, N));
    CKC(c, dalloc(L, &A.bin_of, N));
    CKC(c, dalloc(L, &A.x_tmp, N));
    CKC(c, dalloc(L, &A.v_tmp, N));
    CKC(c, dalloc(L, &A.tag_tmp, N));
    CKC(c, dalloc(L, &A.newpos, N));
    CKC(c, dalloc(L, &A.oldidx, N));
    CKC(c, dalloc(L, &A.binid, N));
    CKC(c, dalloc(L, &A.partner_tmp, N));
    CKC(c, dalloc(L, &A.nbr, (size_t)tiles * max_nb * RC_TILE));
    A.cell_n = d_cell_n;
    A.cell_off = d_cell_off;
    A.tile_cell = d_tile_cell;
    A.cell_tile0 = d_cell_tile0;
    A.Hf = c->d_Hf;
    A.Hif = c->d_Hif;
    A.nbins = c->d_nbins;
    A.bin_off = d_bin_off;
    A.evals = c->d_evals;

    // ---- host marshalling of the inputs ----
    std::vector<int> tile_cell(tiles);
    for (int i = 0; i < n_cells; i++)
        for (int t = 0; t < c->h_ntiles[i]; t++) tile_cell[c->h_tile0[i] + t] = i;
    std::vector<float4> hx(N, make_float4(0, 0, 0, 0)), hv(N, make_float4(0, 0, 0, 0));
    std::vector<int> htag(N, -1);
    std::vector<int4> hpart(N, make_int4(-1, -1, -1, -1));
    std::vector<double> hH0(9 * (size_t)n_cells), hI(9 * (size_t)n_cells, 0.0);
    for (int i = 0; i < n_cells; i++) {
        const rcell_init &ci = cells[i];
        const size_t o = c->h_off[i];
        for (int k = 0; k < ci.n_atoms; k++) {
            hx[o + k] = make_float4((float)ci.x0[3 * k], (float)ci.x0[3 * k + 1], (float)ci.x0[3 * k + 2], 0.f);
            if (ci.v0) hv[o + k] = make_float4((float)ci.v0[3 * k], (float)ci.v0[3 * k + 1], (float)ci.v0[3 * k + 2], 0.f);
            htag[o + k] = k;
        }
        if (P.potential == RC_POT_KG) {
            for (int b = 0; b < ci.n_bonds; b++) {
                const int u = ci.bonds[2 * b], w = ci.bonds[2 * b + 1];
                if (u < 0 || w < 0 || u >= ci.n_atoms || w >= ci.n_atoms || u == w) { rcell_destroy(c); return RC_EINVAL; }
                int *pu = &hpart[o + u].x, *pw = &hpart[o + w].x;
                int ku = 0, kw = 0;
                while (ku < 4 && pu[ku] >= 0) ku++;
                while (kw < 4 && pw[kw] >= 0) kw++;
                if (ku == 4 || kw == 4) { rcell_destroy(c); return RC_EINVAL; }
                pu[ku] = w;
                pw[kw] = u;
            }
        }
        for (int k = 0; k < 9; k++) hH0[9 * i + k] = ci.H0[k];
        hI[9 * i] = hI[9 * i + 4] = hI[9 * i + 8] = 1.0;
    }
    CKC(c, cudaMemcpy(d_cell_n, c->h_n.data(), sizeof(int) * n_cells, cudaMemcpyHostToDevice));
    CKC(c, cudaMemcpy(d_cell_off, c->h_off.data(), sizeof(int) * n_cells, cudaMemcpyHostToDevice));
    CKC(c, cudaMemcpy(d_cell_tile0, c->h_tile0.data(), sizeof(int) * n_cells, cudaMemcpyHostToDevice));
    CKC(c, cudaMemcpy(d_tile_cell, tile_cell.data(), sizeof(int) * tiles, cudaMemcpyHostToDevice));
    CKC(c, cudaMemcpy(d_bin_off, c->h_bin_off.data(), sizeof(int) * n_cells, cudaMemcpyHostToDevice));
    CKC(c, cudaMemcpy(c->d_bin_cap, bin_cap.data(), sizeof(int) * n_cells, cudaMemcpyHostToDevice));
    CKC(c, cudaMemcpy(A.x0, hx.data(), sizeof(float4) * N, cudaMemcpyHostToDevice));
    CKC(c, cudaMemcpy(A.v, hv.data(), sizeof(float4) * N, cudaMemcpyHostToDevice));
    CKC(c, cudaMemcpy(A.tag, htag.data(), sizeof(int) * N, cudaMemcpyHostToDevice));
    CKC(c, cudaMemcpy(A.partner, hpart.data(), sizeof(int4) * N, cudaMemcpyHostToDevice));
    CKC(c, cudaMemcpy(c->d_H0, hH0.data(), sizeof(double) * 9 * n_cells, cudaMemcpyHostToDevice));
    CKC(c, cudaMemcpy(c->d_Rprev, hI.data(), sizeof(double) * 9 * n_cells, cudaMemcpyHostToDevice));
    CKC(c, cudaMemcpy(c->d_Fin, hI.data(), sizeof(double) * 9 * n_cells, cudaMemcpyHostToDevice));
    // initial box: the deformation kernel with F = I sets H = H0, the FP32 box copies and the bins
    rc_launch_deform_impl(c->d_Fin, c->d_H, c->d_Rprev, c->d_Q, c->d_R, c->d_F, c->d_dR, c->d_H0, c->d_Hf, c->d_Hif,
                          A.status, A.need_rebuild, c->d_nbins, c->d_bin_cap, A.active, c->rlist, n_cells, c->stream);
    CKC(c, cudaGetLastError());
    int st = first_status(c);
    if (st != RC_OK) {
        rcell_destroy(c);
        return st == RC_EBOX || st == RC_EDEGEN ? RC_EINVAL : st;
    }
    if (ensure_series(c, 256) != RC_OK) { rcell_destroy(c); return RC_ENOMEM; }
    *out = c;
    return RC_OK;
}

int rcell_set_deformation(rcell_ctx *c, const double *F, int where) {
    if (!c || !F) return RC_EINVAL;
    const double *dF = F;
    if (where == RC_HOST) {
        for (long k = 0; k < 9L * c->n_cells; k++)
            if (!std::isfinite(F[k])) return fail(c, RC_EINVAL, "non-finite deformation gradient");
        CKC(c, cudaMemcpyAsync(c->d_Fin, F, sizeof(double) * 9 * c->n_cells, cudaMemcpyHostToDevice, c->stream));
        dF = c->d_Fin;
    } else if (where != RC_DEVICE) {
        return fail(c, RC_EINVAL, "where");
    }
    rc_launch_deform_impl(dF, c->d_H, c->d_Rprev, c->d_Q, c->d_R, c->d_F, c->d_dR, c->d_H0, c->d_Hf, c->d_Hif,
                          c->ka.status, c->ka.need_rebuild, c->d_nbins, c->d_bin_cap, c->ka.active, c->rlist, c->n_cells, c->stream);
    rc_launch_remap(c->ka, c->d_dR, c->cur, c->n_tiles, c->stream);
    CKC(c, cudaGetLastError());
    return RC_OK;
}

int rcell_run(rcell_ctx *c, int n_steps, int n_avg) {
    if (!c || n_steps < 0 || n_avg < 0) return RC_EINVAL;
    if (n_steps == 0) return RC_OK;
    n_avg = std::min(n_avg, n_steps);
    int e = ensure_series(c, n_avg);
    if (e != RC_OK) return e;
    if (c->use_graphs) {
        auto key = std::make_tuple(n_steps, n_avg, c->cur, c->tpa);
        auto it = c->graphs.find(key);
        if (it == c->graphs.end()) {
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ge = nullptr;
            const int cur0 = c->cur;
            CKC(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
            long k = enqueue_run(c, n_steps, n_avg);
            cudaError_t ce = cudaStreamEndCapture(c->stream, &g);
            if (ce != cudaSuccess) { c->cur = cur0; return fail(c, RC_ECUDA, std::string("capture: ") + cudaGetErrorString(ce)); }
            ce = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            if (ce != cudaSuccess) { c->cur = cur0; return fail(c, RC_ECUDA, std::string("instantiate: ") + cudaGetErrorString(ce)); }
            it = c->graphs.emplace(key, ge).first;
            c->graph_launches[key] = k;
            c->cur = cur0;
        }
        c->launches_last = c->graph_launches[key];
        CKC(c, cudaGraphLaunch(it->second, c->stream));
        c->cur ^= (n_steps & 1);
    } else {
        c->launches_last = enqueue_run(c, n_steps, n_avg);
        CKC(c, cudaGetLastError());
    }
    c->last_n_avg = n_avg;
    return RC_OK;
}

int rcell_set_active(rcell_ctx *c, const int *mask, int where) {
    if (!c || !mask) return RC_EINVAL;
    CKC(c, cudaMemcpyAsync((void *)c->ka.active, mask, sizeof(int) * c->n_cells,
                           where == RC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->stream));
    if (where == RC_HOST) CKC(c, cudaStreamSynchronize(c->stream));
    return RC_OK;
}

int rcell_stress(rcell_ctx *c, double *sigma, double *sigma_stderr, double *P, int where) {
    if (!c) return RC_EINVAL;
    if (c->last_n_avg <= 0) return fail(c, RC_ESTATE, "no stress samples: run with n_avg > 0 first");
    rc_launch_stress(c->ka.series, c->last_n_avg, c->series_cap, c->d_H, c->d_Q, c->d_F, pconv_of(c->prm.units),
                     c->d_rot, c->d_sig_fem, c->d_sig_se, c->d_sig_md, c->d_P, c->n_cells, c->stream);
    CKC(c, cudaGetLastError());
    const cudaMemcpyKind kind = where == RC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const size_t n6 = sizeof(double) * 6 * c->n_cells, n9 = sizeof(double) * 9 * c->n_cells;
    if (sigma) CKC(c, cudaMemcpyAsync(sigma, c->d_sig_fem, n6, kind, c->stream));
    if (sigma_stderr) CKC(c, cudaMemcpyAsync(sigma_stderr, c->d_sig_se, n6, kind, c->stream));
    if (P) CKC(c, cudaMemcpyAsync(P, c->d_P, n9, kind, c->stream));
    if (where == RC_HOST) return first_status(c);
    return RC_OK;
}

int rcell_eval(rcell_ctx *c) {
    if (!c) return RC_EINVAL;
    CKC(c, cudaMemsetAsync(c->ka.eval_acc, 0, sizeof(double) * 8 * c->n_cells, c->stream));
    enqueue_step(c, MODE_EVAL, -1, 0);
    CKC(c, cudaGetLastError());
    return RC_OK;
}

int rcell_get_energy(rcell_ctx *c, double *pe, double *W) {
    if (!c) return RC_EINVAL;
    std::vector<double> acc(8 * (size_t)c->n_cells);
    CKC(c, cudaStreamSynchronize(c->stream));
    CKC(c, cudaMemcpy(acc.data(), c->ka.eval_acc, sizeof(double) * acc.size(), cudaMemcpyDeviceToHost));
    for (int i = 0; i < c->n_cells; i++) {
        const double *a = &acc[8 * i];
        if (pe) pe[i] = a[0];
        if (W) {
            double *w = W + 9 * i;
            w[0] = a[1]; w[4] = a[2]; w[8] = a[3];
            w[1] = w[3] = a[4];
            w[2] = w[6] = a[5];
            w[5] = w[7] = a[6];
        }
    }
    return first_status(c);
}

int rcell_get_atoms(rcell_ctx *c, int cell, double *x, double *v, double *f) {
    if (!c || cell < 0 || cell >= c->n_cells) return RC_EINVAL;
    const int n = c->h_n[cell], off = c->h_off[cell];
    std::vector<float4> hx(n), hv(n), hf(n);
    std::vector<int> tag(n);
    CKC(c, cudaStreamSynchronize(c->stream));
    const float4 *X = c->cur ? c->ka.x1 : c->ka.x0;
    CKC(c, cudaMemcpy(tag.data(), c->ka.tag + off, sizeof(int) * n, cudaMemcpyDeviceToHost));
    if (x) CKC(c, cudaMemcpy(hx.data(), X + off, sizeof(float4) * n, cudaMemcpyDeviceToHost));
    if (v) CKC(c, cudaMemcpy(hv.data(), c->ka.v + off, sizeof(float4) * n, cudaMemcpyDeviceToHost));
    if (f) CKC(c, cudaMemcpy(hf.data(), c->ka.f + off, sizeof(float4) * n, cudaMemcpyDeviceToHost));
    for (int k = 0; k < n; k++) {
        const int t = tag[k];
        if (t < 0 || t >= n) return fail(c, RC_ESTATE, "corrupt tag table");
        if (x) { x[3 * t] = hx[k].x; x[3 * t + 1] = hx[k].y; x[3 * t + 2] = hx[k].z; }
        if (v) { v[3 * t] = hv[k].x; v[3 * t + 1] = hv[k].y; v[3 * t + 2] = hv[k].z; }
        if (f) { f[3 * t] = hf[k].x; f[3 * t + 1] = hf[k].y; f[3 * t + 2] = hf[k].z; }
    }
    return RC_OK;
}

int rcell_get_box(rcell_ctx *c, int cell, double *H, double *Q, double *R) {
    if (!c || cell < 0 || cell >= c->n_cells) return RC_EINVAL;
    CKC(c, cudaStreamSynchronize(c->stream));
    if (H) CKC(c, cudaMemcpy(H, c->d_H + 9 * cell, sizeof(double) * 9, cudaMemcpyDeviceToHost));
    if (Q) CKC(c, cudaMemcpy(Q, c->d_Q + 9 * cell, sizeof(double) * 9, cudaMemcpyDeviceToHost));
    if (R) CKC(c, cudaMemcpy(R, c->d_R + 9 * cell, sizeof(double) * 9, cudaMemcpyDeviceToHost));
    return RC_OK;
}

int rcell_get_neighbors(rcell_ctx *c, int cell, int *pairs, long max_pairs, long *count) {
    if (!c || cell < 0 || cell >= c->n_cells || !count) return RC_EINVAL;
    const int n = c->h_n[cell], off = c->h_off[cell], nt = c->h_ntiles[cell], t0 = c->h_tile0[cell];
    const int mx = c->kp.max_nb;
    std::vector<int> tag(n), nnb(n), nbr((size_t)nt * mx * RC_TILE);
    CKC(c, cudaStreamSynchronize(c->stream));
    CKC(c, cudaMemcpy(tag.data(), c->ka.tag + off, sizeof(int) * n, cudaMemcpyDeviceToHost));
    CKC(c, cudaMemcpy(nnb.data(), c->ka.nnb + off, sizeof(int) * n, cudaMemcpyDeviceToHost));
    CKC(c, cudaMemcpy(nbr.data(), c->ka.nbr + (size_t)t0 * mx * RC_TILE, sizeof(int) * nbr.size(),
                      cudaMemcpyDeviceToHost));
    long k = 0;
    for (int i = 0; i < n; i++) {
        const int t = i / RC_TILE, l = i % RC_TILE;
        for (int q = 0; q < nnb[i]; q++) {
            const unsigned e = (unsigned)nbr[((size_t)t * mx + (q & ~3)) * RC_TILE + 4 * l + (q & 3)];
            const int j = (int)(e & RC_IDX_MASK) - off;
            if (j < 0 || j >= n) return fail(c, RC_ESTATE, "neighbour index outside its cell");
            if (pairs && k < max_pairs) {
                pairs[2 * k] = tag[i];
                pairs[2 * k + 1] = tag[j];
            }
            k++;
        }
    }
    *count = k;
    if (k > max_pairs) return fail(c, RC_EOVERFLOW, "pairs buffer too small");
    return first_status(c);
}

int rcell_get_series(rcell_ctx *c, int cell, double *stress, double *pe, double *ke) {
    if (!c || cell < 0 || cell >= c->n_cells) return RC_EINVAL;
    if (c->last_n_avg <= 0) return fail(c, RC_ESTATE, "no samples");
    const int na = c->last_n_avg;
    std::vector<double> rec((size_t)na * RC_SAMPLE_W), H(9);
    CKC(c, cudaStreamSynchronize(c->stream));
    CKC(c, cudaMemcpy(rec.data(), c->ka.series + (size_t)cell * c->series_cap * RC_SAMPLE_W,
                      sizeof(double) * rec.size(), cudaMemcpyDeviceToHost));
    CKC(c, cudaMemcpy(H.data(), c->d_H + 9 * cell, sizeof(double) * 9, cudaMemcpyDeviceToHost));
    const double scale = -pconv_of(c->prm.units) / (H[0] * H[4] * H[8]);
    for (int t = 0; t < na; t++) {
        const double *r = &rec[(size_t)t * RC_SAMPLE_W];
        if (stress)
            for (int k = 0; k < 6; k++) stress[6 * t + k] = scale * (r[k] + r[6 + k]);
        if (pe) pe[t] = r[12];
        if (ke) ke[t] = 0.5 * (r[0] + r[1] + r[2]);
    }
    return RC_OK;
}

int rcell_sync(rcell_ctx *c) {
    if (!c) return RC_EINVAL;
    return first_status(c);
}

int rcell_clear_status(rcell_ctx *c) {
    if (!c) return RC_EINVAL;
    CKC(c, cudaMemsetAsync(c->ka.status, 0, sizeof(int) * c->n_cells, c->stream));
    CKC(c, cudaStreamSynchronize(c->stream));
    c->err = "ok";
    return RC_OK;
}

int rcell_set_staging(rcell_ctx *c, int staged) {
    if (!c) return RC_EINVAL;
    if (staged >= 0 && (staged ? 1 : 0) != c->staged) {
        c->staged = staged ? 1 : 0;
        free_graphs(c);
    }
    return RC_OK;
}

int rcell_set_limits(rcell_ctx *c, int max_neighbors, int wait_polls) {
    if (!c) return RC_EINVAL;
    if (max_neighbors >= 0) {
        const int mx = max_neighbors == 0 ? c->max_nb_alloc : max_neighbors;
        if (mx < 4 || mx % 4 != 0 || mx > c->max_nb_alloc)
            return fail(c, RC_EINVAL, "max_neighbors must be 0 or a multiple of 4 in [4, the allocated capacity]");
        if (mx != c->kp.max_nb) {
            CKC(c, cudaStreamSynchronize(c->stream));
            c->kp.max_nb = mx;
            free_graphs(c);  // graphs hold the old parameters
            std::vector<int> ones(c->n_cells, 1);  // every list is rebuilt with the new capacity
            CKC(c, cudaMemcpy(c->ka.need_rebuild, ones.data(), sizeof(int) * c->n_cells, cudaMemcpyHostToDevice));
        }
    }
    if (wait_polls >= 0 && wait_polls != c->kp.wait_polls) {
        CKC(c, cudaStreamSynchronize(c->stream));
        c->kp.wait_polls = wait_polls;
        free_graphs(c);
    }
    return RC_OK;
}

int rcell_set_tuning(rcell_ctx *c, int threads_per_atom, int use_graphs) {
    if (!c) return RC_EINVAL;
    if (threads_per_atom >= 0) {
        if (threads_per_atom != 0 && threads_per_atom != 1 && threads_per_atom != 2 && threads_per_atom != 4 &&
            threads_per_atom != 8)
            return fail(c, RC_EINVAL, "threads_per_atom must be 0 (lean walk), 1, 2, 4 or 8");
        if (threads_per_atom != c->tpa) free_graphs(c);
        c->tpa = threads_per_atom;
    }
    if (use_graphs >= 0) c->use_graphs = use_graphs ? 1 : 0;
    return RC_OK;
}

int rcell_minimize(rcell_ctx *c, int max_iter, double f_tol, double dt0, double dt_max, double dmax,
                   int *iters_out) {
    if (!c || max_iter < 0 || !(f_tol > 0) || !(dt0 > 0) || !(dt_max >= dt0)) return RC_EINVAL;
    const int nc = c->n_cells;
    if (!c->fire.acc) {
        auto &L = c->allocs;
        FireState &f = c->fire;
        CKC(c, dalloc(L, &f.acc, 4 * (size_t)nc));
        CKC(c, dalloc(L, &f.fmax2, nc));
        CKC(c, dalloc(L, &f.dt, nc));
        CKC(c, dalloc(L, &f.alpha, nc));
        CKC(c, dalloc(L, &f.mixa, nc));
        CKC(c, dalloc(L, &f.mixb, nc));
        CKC(c, dalloc(L, &f.npos, nc));
        CKC(c, dalloc(L, &f.done, nc));
        CKC(c, dalloc(L, &f.iters, nc));
        CKC(c, dalloc(L, &f.it, nc));
        CKC(c, dalloc(L, &f.zero, nc));
        CKC(c, dalloc(L, &f.moving, nc));
        CKC(c, dalloc(L, &c->d_fire_left, 1));
    }
    rc_launch_fire_init(c->fire, c->ka.status, c->ka.active, nc, (float)dt0, c->stream);
    rc_launch_fire_zero_v(c->ka, c->fire, c->n_tiles, 0, c->stream);
    {
    // while minimising, the kernels see the per-cell "still moving" flags as the
    // activity mask, so converged cells cost no more force evaluations; the
    // caller's mask is back in place on every way out of this block
    struct MaskSwap {
        rcell_ctx *c;
        const int *saved;
        ~MaskSwap() { c->ka.active = saved; }
    } swap{c, c->ka.active};
    c->ka.active = c->fire.moving;
    // iterations in batches between convergence checks: forces (MODE_EVAL, after the
    // list and density kernels), then the FIRE power / control / move kernels
    const int batch = 32;
    auto enqueue_batch = [&](int nb) {
        cudaMemsetAsync(c->d_fire_left, 0, sizeof(int), c->stream);
        for (int k = 0; k < nb; k++) {  // the last iteration of the batch counts the cells still moving
            enqueue_step(c, MODE_EVAL, -1, 0);
            rc_launch_fire_iteration(c->kp, c->ka, c->cur, c->fire, c->n_tiles, nc, (float)f_tol, (float)dt_max,
                                     (float)dmax, k == nb - 1 ? c->d_fire_left : nullptr, c->stream);
        }
    };
    const double key[5] = {f_tol, dt_max, dmax, (double)c->tpa, (double)c->cur};
    if (c->use_graphs && (!c->fire_graph || !std::equal(key, key + 5, c->fire_key))) {
        if (c->fire_graph) cudaGraphExecDestroy(c->fire_graph);
        c->fire_graph = nullptr;
        cudaGraph_t g = nullptr;
        CKC(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        enqueue_batch(batch);
        CKC(c, cudaStreamEndCapture(c->stream, &g));
        cudaError_t ce = cudaGraphInstantiate(&c->fire_graph, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) { c->fire_graph = nullptr; return fail(c, RC_ECUDA, "FIRE graph instantiation"); }
        std::copy(key, key + 5, c->fire_key);
    }
    for (int it0 = 0; it0 < max_iter; it0 += batch) {
        const int nb = std::min(batch, max_iter - it0);
        if (c->use_graphs && nb == batch) CKC(c, cudaGraphLaunch(c->fire_graph, c->stream));
        else enqueue_batch(nb);
        CKC(c, cudaGetLastError());
        int left = 0;
        CKC(c, cudaMemcpyAsync(&left, c->d_fire_left, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CKC(c, cudaStreamSynchronize(c->stream));
        if (left == 0) break;
    }
    }
    rc_launch_fire_zero_v(c->ka, c->fire, c->n_tiles, 1, c->stream);
    CKC(c, cudaGetLastError());
    if (iters_out) {
        CKC(c, cudaMemcpyAsync(iters_out, c->fire.iters, sizeof(int) * nc, cudaMemcpyDeviceToHost, c->stream));
    }
    CKC(c, cudaStreamSynchronize(c->stream));
    return first_status(c);
}

int rcell_stress_static(rcell_ctx *c, double *sigma, double *P, int where) {
    if (!c) return RC_EINVAL;
    const int nc = c->n_cells;
    if (!c->d_mcell) {
        CKC(c, dalloc(c->allocs, &c->d_mcell, 6 * (size_t)nc));
        CKC(c, dalloc(c->allocs, &c->d_pk_acc, 9 * (size_t)nc));
    }
    rc_launch_static_prep(c->d_H, c->d_H0, c->d_mcell, c->d_pk_acc, nc, c->stream);
    rc_launch_sort(c->kp, c->ka, c->cur, nc, c->stream);
    rc_launch_nlist(c->kp, c->ka, c->cur, c->n_tiles, c->stream);
    if (c->kp.pot == RC_POT_SC) rc_launch_density(c->kp, c->ka, c->cur, c->n_tiles, 1, 0, c->stream);
    rc_launch_static_pk1(c->kp, c->ka, c->cur, c->n_tiles, c->d_mcell, c->d_pk_acc, c->stream);
    rc_launch_static_finish(c->d_pk_acc, c->d_H0, c->d_Q, c->d_F, pconv_of(c->prm.units), c->d_P, c->d_sig_fem,
                            c->ka.status, nc, c->stream);
    CKC(c, cudaGetLastError());
    const cudaMemcpyKind kind = where == RC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (sigma) CKC(c, cudaMemcpyAsync(sigma, c->d_sig_fem, sizeof(double) * 6 * nc, kind, c->stream));
    if (P) CKC(c, cudaMemcpyAsync(P, c->d_P, sizeof(double) * 9 * nc, kind, c->stream));
    if (where == RC_HOST) return first_status(c);
    return RC_OK;
}

int rcell_get_rebuilds(rcell_ctx *c, unsigned long long *counts) {
    if (!c || !counts) return RC_EINVAL;
    CKC(c, cudaStreamSynchronize(c->stream));
    CKC(c, cudaMemcpy(counts, c->ka.rebuilds, sizeof(unsigned long long) * c->n_cells, cudaMemcpyDeviceToHost));
    return RC_OK;
}

int rcell_info(const rcell_ctx *c, int *n_cells, long *n_atoms, long *launches_last_run) {
    if (!c) return RC_EINVAL;
    if (n_cells) *n_cells = c->n_cells;
    if (n_atoms) *n_atoms = c->n_atoms;
    if (launches_last_run) *launches_last_run = c->launches_last;
    return RC_OK;
}

// checkpoint layout: header {magic, n, cur-independent}, then per cell
// x[n] v[n] (float4), tag[n], partner[n] (int4), H R_prev Q R F (5 x 9 doubles),
// Hf Hif (2 x 8 floats), nbins (4 ints), evals (u64)
static size_t ckpt_size(int n) {
    return 16 + (size_t)n * (2 * sizeof(float4) + sizeof(int) + sizeof(int4)) + 45 * sizeof(double) +
           16 * sizeof(float) + 4 * sizeof(int) + sizeof(unsigned long long);
}

int rcell_checkpoint(rcell_ctx *c, int cell, void *buf, size_t *bytes) {
    if (!c || cell < 0 || cell >= c->n_cells || !bytes) return RC_EINVAL;
    const int n = c->h_n[cell], off = c->h_off[cell];
    const size_t need = ckpt_size(n);
    if (!buf) { *bytes = need; return RC_OK; }
    if (*bytes < need) { *bytes = need; return fail(c, RC_EINVAL, "checkpoint buffer too small"); }
    CKC(c, cudaStreamSynchronize(c->stream));
    char *p = static_cast<char *>(buf);
    const uint64_t magic = 0x52434B5054303031ull;  // "RCKPT001"
    memcpy(p, &magic, 8);
    const int64_t nn = n;
    memcpy(p + 8, &nn, 8);
    p += 16;
    const float4 *X = c->cur ? c->ka.x1 : c->ka.x0;
    CKC(c, cudaMemcpy(p, X + off, sizeof(float4) * n, cudaMemcpyDeviceToHost)); p += sizeof(float4) * n;
    CKC(c, cudaMemcpy(p, c->ka.v + off, sizeof(float4) * n, cudaMemcpyDeviceToHost)); p += sizeof(float4) * n;
    CKC(c, cudaMemcpy(p, c->ka.tag + off, sizeof(int) * n, cudaMemcpyDeviceToHost)); p += sizeof(int) * n;
    CKC(c, cudaMemcpy(p, c->ka.partner + off, sizeof(int4) * n, cudaMemcpyDeviceToHost)); p += sizeof(int4) * n;
    for (double *src : {c->d_H, c->d_Rprev, c->d_Q, c->d_R, c->d_F}) {
        CKC(c, cudaMemcpy(p, src + 9 * cell, sizeof(double) * 9, cudaMemcpyDeviceToHost));
        p += sizeof(double) * 9;
    }
    CKC(c, cudaMemcpy(p, c->d_Hf + 8 * cell, sizeof(float) * 8, cudaMemcpyDeviceToHost)); p += sizeof(float) * 8;
    CKC(c, cudaMemcpy(p, c->d_Hif + 8 * cell, sizeof(float) * 8, cudaMemcpyDeviceToHost)); p += sizeof(float) * 8;
    CKC(c, cudaMemcpy(p, c->d_nbins + 4 * cell, sizeof(int) * 4, cudaMemcpyDeviceToHost)); p += sizeof(int) * 4;
    CKC(c, cudaMemcpy(p, c->d_evals + cell, sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    // the run that follows starts from a fresh neighbour build, exactly as a run
    // after rcell_restore does, so a replay from this checkpoint is bit-identical
    const int one = 1;
    CKC(c, cudaMemcpy(c->ka.need_rebuild + cell, &one, sizeof(int), cudaMemcpyHostToDevice));
    *bytes = need;
    return RC_OK;
}

int rcell_restore(rcell_ctx *c, int cell, const void *buf, size_t bytes) {
    if (!c || cell < 0 || cell >= c->n_cells || !buf) return RC_EINVAL;
    const int n = c->h_n[cell], off = c->h_off[cell];
    if (bytes < ckpt_size(n)) return fail(c, RC_EINVAL, "checkpoint too small");
    const char *p = static_cast<const char *>(buf);
    uint64_t magic;
    int64_t nn;
    memcpy(&magic, p, 8);
    memcpy(&nn, p + 8, 8);
    if (magic != 0x52434B5054303031ull || nn != n) return fail(c, RC_EINVAL, "checkpoint does not match this cell");
    p += 16;
    CKC(c, cudaStreamSynchronize(c->stream));
    float4 *X = c->cur ? c->ka.x1 : c->ka.x0;
    CKC(c, cudaMemcpy(X + off, p, sizeof(float4) * n, cudaMemcpyHostToDevice)); p += sizeof(float4) * n;
    CKC(c, cudaMemcpy(c->ka.v + off, p, sizeof(float4) * n, cudaMemcpyHostToDevice)); p += sizeof(float4) * n;
    CKC(c, cudaMemcpy(c->ka.tag + off, p, sizeof(int) * n, cudaMemcpyHostToDevice)); p += sizeof(int) * n;
    CKC(c, cudaMemcpy(c->ka.partner + off, p, sizeof(int4) * n, cudaMemcpyHostToDevice)); p += sizeof(int4) * n;
    for (double *dst : {c->d_H, c->d_Rprev, c->d_Q, c->d_R, c->d_F}) {
        CKC(c, cudaMemcpy(dst + 9 * cell, p, sizeof(double) * 9, cudaMemcpyHostToDevice));
        p += sizeof(double) * 9;
    }
    CKC(c, cudaMemcpy(c->d_Hf + 8 * cell, p, sizeof(float) * 8, cudaMemcpyHostToDevice)); p += sizeof(float) * 8;
    CKC(c, cudaMemcpy(c->d_Hif + 8 * cell, p, sizeof(float) * 8, cudaMemcpyHostToDevice)); p += sizeof(float) * 8;
    CKC(c, cudaMemcpy(c->d_nbins + 4 * cell, p, sizeof(int) * 4, cudaMemcpyHostToDevice)); p += sizeof(int) * 4;
    CKC(c, cudaMemcpy(c->d_evals + cell, p, sizeof(unsigned long long), cudaMemcpyHostToDevice));
    const int one = 1, zero = 0;
    CKC(c, cudaMemcpy(c->ka.need_rebuild + cell, &one, sizeof(int), cudaMemcpyHostToDevice));
    CKC(c, cudaMemcpy(c->ka.status + cell, &zero, sizeof(int), cudaMemcpyHostToDevice));
    return RC_OK;
}

int rcell_profile_kernels(rcell_ctx *c, int n_steps, double *ms_out) {
    if (!c || !ms_out || n_steps <= 0) return RC_EINVAL;
    for (int k = 0; k < 8; k++) ms_out[k] = 0.0;
    cudaEvent_t ev[6];
    for (auto &e : ev) CKC(c, cudaEventCreate(&e));
    double acc[8] = {0}, cnt[8] = {0};
    auto lap = [&](int a, int b, int slot) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev[a], ev[b]) == cudaSuccess) { acc[slot] += ms; cnt[slot] += 1; }
    };
    // coupling kernels once: re-apply the current F (Delta R = I), then the stress reduction
    CKC(c, cudaEventRecord(ev[0], c->stream));
    rc_launch_deform_impl(c->d_F, c->d_H, c->d_Rprev, c->d_Q, c->d_R, c->d_F, c->d_dR, c->d_H0, c->d_Hf, c->d_Hif,
                          c->ka.status, c->ka.need_rebuild, c->d_nbins, c->d_bin_cap, c->ka.active, c->rlist, c->n_cells, c->stream);
    CKC(c, cudaEventRecord(ev[1], c->stream));
    rc_launch_remap(c->ka, c->d_dR, c->cur, c->n_tiles, c->stream);
    CKC(c, cudaEventRecord(ev[2], c->stream));
    CKC(c, cudaEventSynchronize(ev[2]));
    lap(0, 1, 4);
    lap(1, 2, 5);
    // the steps of a run of n_steps that samples its last half, as rcell_run(n_steps, n_steps / 2)
    const int n_avg = std::min(n_steps / 2, c->series_cap);
    CKC(c, cudaMemsetAsync(c->ka.series, 0, sizeof(double) * (size_t)c->n_cells * c->series_cap * RC_SAMPLE_W,
                           c->stream));
    for (int s = 0; s <= n_steps; s++) {
        const int mode = s == 0 ? MODE_SETUP : (s == n_steps ? MODE_LAST : MODE_STEP);
        const int slot = (s > 0 && s > n_steps - n_avg) ? s - (n_steps - n_avg) - 1 : -1;
        CKC(c, cudaEventRecord(ev[0], c->stream));
        rc_launch_sort(c->kp, c->ka, c->cur, c->n_cells, c->stream);
        CKC(c, cudaEventRecord(ev[1], c->stream));
        rc_launch_nlist(c->kp, c->ka, c->cur, c->n_tiles, c->stream);
        CKC(c, cudaEventRecord(ev[2], c->stream));
        if (c->kp.pot == RC_POT_SC) rc_launch_density(c->kp, c->ka, c->cur, c->n_tiles, c->tpa, stage_atoms(c), c->stream);
        CKC(c, cudaEventRecord(ev[3], c->stream));
        rc_launch_force(c->kp, c->ka, c->cur, c->n_tiles, c->tpa, mode, slot, s, stage_atoms(c), c->stream);
        CKC(c, cudaEventRecord(ev[4], c->stream));
        CKC(c, cudaEventSynchronize(ev[4]));
        lap(0, 1, 0);
        lap(1, 2, 1);
        if (c->kp.pot == RC_POT_SC) lap(2, 3, 2);
        if (s > 0) lap(3, 4, slot >= 0 ? 7 : 3);  // steady-state force launches only
        if (mode != MODE_LAST) c->cur ^= 1;
    }
    if (n_steps & 1) rc_launch_keep_frozen(c->ka, c->cur, c->n_tiles, c->stream);
    rc_launch_advance(c->d_evals, c->ka.active, c->n_cells, n_steps + 1, c->stream);
    c->last_n_avg = n_avg;
    if (c->last_n_avg > 0) {
        CKC(c, cudaEventRecord(ev[0], c->stream));
        rc_launch_stress(c->ka.series, c->last_n_avg, c->series_cap, c->d_H, c->d_Q, c->d_F, pconv_of(c->prm.units),
                         c->d_rot, c->d_sig_fem, c->d_sig_se, c->d_sig_md, c->d_P, c->n_cells, c->stream);
        CKC(c, cudaEventRecord(ev[1], c->stream));
        CKC(c, cudaEventSynchronize(ev[1]));
        lap(0, 1, 6);
    }
    for (auto &e : ev) cudaEventDestroy(e);
    for (int k = 0; k < 8; k++) ms_out[k] = cnt[k] > 0 ? acc[k] / cnt[k] : 0.0;
    CKC(c, cudaGetLastError());
    return first_status(c);
}

const char *rcell_last_error(const rcell_ctx *c) { return c ? c->err.c_str() : "null context"; }

void rcell_destroy(rcell_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_graphs(c);
    for (void *p : c->allocs) cudaFree(p);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

// --------------------------------------------------------------------------
// finite elements
// --------------------------------------------------------------------------
#define CKF(fe, call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) { (fe)->err = cudaGetErrorString(e_); return RC_ECUDA; }   \
    } while (0)

}  // extern "C"

namespace {

void apply_bc(fe_ctx *fe, double lambda, cudaStream_t s) {
    fe_launch_apply_bc(fe->d_mask, fe->d_val, fe->d_g, lambda, lambda - fe->lam_last, fe->d_d, 3 * fe->nn, s);
    fe->lam_last = lambda;
}

int fe_create_npe(int npe, const double *X, int nn, const int *conn, int ne, const int *bc_mask, const double *bc_val,
                  double rho0, double dt, double damping, double hg_coef, void *stream, fe_ctx **out) {
    const int *hex = conn;
    if (!X || !hex || !bc_mask || !bc_val || !out || nn <= 0 || ne <= 0 || !(rho0 > 0) || !(dt > 0)) return RC_EINVAL;
    for (int k = 0; k < npe * ne; k++)
        if (hex[k] < 0 || hex[k] >= nn) return RC_EINVAL;
    fe_ctx *fe = new fe_ctx();
    *out = nullptr;
    fe->npe = npe;
    fe->nn = nn;
    fe->ne = ne;
    fe->rho0 = rho0;
    fe->dt = dt;
    fe->damping = damping;
    fe->hg = hg_coef;
    if (stream) fe->stream = (cudaStream_t)stream;
    else { CKF(fe, cudaStreamCreate(&fe->stream)); fe->own_stream = true; }
    CKF(fe, cudaEventCreateWithFlags(&fe->ev, cudaEventDisableTiming));
    auto &L = fe->allocs;
    const size_t n3 = 3 * (size_t)nn;
    CKF(fe, dalloc(L, &fe->d_X, n3));
    CKF(fe, dalloc(L, &fe->d_val, n3));
    CKF(fe, dalloc(L, &fe->d_d, n3));
    CKF(fe, dalloc(L, &fe->d_v, n3));
    CKF(fe, dalloc(L, &fe->d_fint, n3));
    CKF(fe, dalloc(L, &fe->d_mass, nn));
    CKF(fe, dalloc(L, &fe->d_mask, n3));
    CKF(fe, dalloc(L, &fe->d_conn, (size_t)npe * ne));
    CKF(fe, dalloc(L, &fe->d_gradN, 3 * (size_t)npe * ne));
    CKF(fe, dalloc(L, &fe->d_V0, ne));
    CKF(fe, dalloc(L, &fe->d_F, 9 * (size_t)ne));
    CKF(fe, dalloc(L, &fe->d_P, 9 * (size_t)ne));
    CKF(fe, dalloc(L, &fe->d_err, 1));
    CKF(fe, cudaMemcpy(fe->d_X, X, sizeof(double) * n3, cudaMemcpyHostToDevice));
    CKF(fe, cudaMemcpy(fe->d_val, bc_val, sizeof(double) * n3, cudaMemcpyHostToDevice));
    CKF(fe, cudaMemcpy(fe->d_mask, bc_mask, sizeof(int) * n3, cudaMemcpyHostToDevice));
    CKF(fe, cudaMemcpy(fe->d_conn, hex, sizeof(int) * npe * ne, cudaMemcpyHostToDevice));
    fe_launch_geometry(npe, fe->d_X, fe->d_conn, ne, rho0, fe->d_gradN, fe->d_V0, fe->d_mass, fe->d_err, fe->stream);
    CKF(fe, cudaGetLastError());
    int err = 0;
    CKF(fe, cudaStreamSynchronize(fe->stream));
    CKF(fe, cudaMemcpy(&err, fe->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) { fe_destroy(fe); return RC_EINVAL; }
    *out = fe;
    return RC_OK;
}

}  // namespace

extern "C" {

int fe_create(const double *X, int nn, const int *hex, int ne, const int *bc_mask, const double *bc_val, double rho0,
              double dt, double damping, double hg_coef, void *stream, fe_ctx **out) {
    return fe_create_npe(8, X, nn, hex, ne, bc_mask, bc_val, rho0, dt, damping, hg_coef, stream, out);
}

int fe_create_tet4(const double *X, int nn, const int *tet, int ne, const int *bc_mask, const double *bc_val,
                   double rho0, double dt, double damping, void *stream, fe_ctx **out) {
    return fe_create_npe(4, X, nn, tet, ne, bc_mask, bc_val, rho0, dt, damping, 0.0, stream, out);
}

int fe_apply_bc(fe_ctx *fe, double lambda) {
    if (!fe) return RC_EINVAL;
    apply_bc(fe, lambda, fe->stream);
    CKF(fe, cudaGetLastError());
    return RC_OK;
}

int fe_set_predictor(fe_ctx *fe, const double *g) {
    if (!fe) return RC_EINVAL;
    if (!g) {
        fe->d_g = nullptr;  // the buffer stays allocated with the context
        return RC_OK;
    }
    for (long k = 0; k < 3L * fe->nn; k++)
        if (!std::isfinite(g[k])) return RC_EINVAL;
    static_assert(sizeof(double) == 8, "");
    if (!fe->d_g_buf) CKF(fe, dalloc(fe->allocs, &fe->d_g_buf, 3 * (size_t)fe->nn));
    CKF(fe, cudaMemcpyAsync(fe->d_g_buf, g, sizeof(double) * 3 * fe->nn, cudaMemcpyHostToDevice, fe->stream));
    CKF(fe, cudaStreamSynchronize(fe->stream));
    fe->d_g = fe->d_g_buf;
    return RC_OK;
}

int fe_get_F(fe_ctx *fe, double *F, int where) {
    if (!fe || !F) return RC_EINVAL;
    fe_launch_F(fe->npe, fe->d_conn, fe->d_gradN, fe->d_d, fe->d_F, fe->ne, fe->stream);
    CKF(fe, cudaGetLastError());
    CKF(fe, cudaMemcpyAsync(F, fe->d_F, sizeof(double) * 9 * fe->ne,
                            where == RC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, fe->stream));
    if (where == RC_HOST) CKF(fe, cudaStreamSynchronize(fe->stream));
    return RC_OK;
}

int fe_update(fe_ctx *fe, const double *P, int where) {
    if (!fe || !P) return RC_EINVAL;
    const double *dP = P;
    if (where == RC_HOST) {
        CKF(fe, cudaMemcpyAsync(fe->d_P, P, sizeof(double) * 9 * fe->ne, cudaMemcpyHostToDevice, fe->stream));
        dP = fe->d_P;
    }
    CKF(fe, cudaMemsetAsync(fe->d_fint, 0, sizeof(double) * 3 * fe->nn, fe->stream));
    fe_launch_fint(fe->npe, fe->d_X, fe->d_conn, fe->d_gradN, fe->d_V0, dP, fe->d_d, fe->hg, fe->d_fint, fe->ne,
                   fe->stream);
    fe_launch_update(fe->d_mask, fe->d_mass, fe->d_fint, fe->dt, fe->damping, fe->d_d, fe->d_v, 3 * fe->nn,
                     fe->stream);
    CKF(fe, cudaGetLastError());
    return RC_OK;
}

int fe_step(fe_ctx *fe, rcell_ctx *rc, double lambda, int n_steps, int n_avg, double *u_out) {
    if (!fe || !rc) return RC_EINVAL;
    if (rc->n_cells != fe->ne) { fe->err = "one r-cell per element required"; return RC_EINVAL; }
    int e;
    apply_bc(fe, lambda, fe->stream);
    fe_launch_F(fe->npe, fe->d_conn, fe->d_gradN, fe->d_d, fe->d_F, fe->ne, fe->stream);
    CKF(fe, cudaGetLastError());
    if (fe->stream != rc->stream) {
        CKF(fe, cudaEventRecord(fe->ev, fe->stream));
        CKF(fe, cudaStreamWaitEvent(rc->stream, fe->ev, 0));
    }
    if ((e = rcell_set_deformation(rc, fe->d_F, RC_DEVICE)) != RC_OK) return e;
    if ((e = rcell_run(rc, n_steps, n_avg)) != RC_OK) return e;
    if ((e = rcell_stress(rc, nullptr, nullptr, fe->d_P, RC_DEVICE)) != RC_OK) return e;
    if (fe->stream != rc->stream) {
        CKF(fe, cudaEventRecord(fe->ev, rc->stream));
        CKF(fe, cudaStreamWaitEvent(fe->stream, fe->ev, 0));
    }
    if ((e = fe_update(fe, fe->d_P, RC_DEVICE)) != RC_OK) return e;
    if (u_out) {
        CKF(fe, cudaMemcpyAsync(u_out, fe->d_d, sizeof(double) * 3 * fe->nn, cudaMemcpyDeviceToHost, fe->stream));
        CKF(fe, cudaStreamSynchronize(fe->stream));
        return rcell_sync(rc);
    }
    return RC_OK;
}

int fe_step_surrogate(fe_ctx *fe, rcell_ctx *rc, sur_ctx *sur, double lambda, int n_steps, int n_avg,
                      float spread_on, float spread_off, float s_floor, int force_md, float *h_state, double *F_prev,
                      int *md_flag, float *spread_out, int *n_md, int *n_replayed) {
    if (!fe || !rc || !sur || !h_state || !F_prev || !md_flag) return RC_EINVAL;
    if (rc->n_cells != fe->ne) { fe->err = "one r-cell per element required"; return RC_EINVAL; }
    void *ss = nullptr;
    if (sur_info(sur, nullptr, &ss) != RC_OK) return RC_EINVAL;
    if ((cudaStream_t)ss != fe->stream || rc->stream != fe->stream) {
        fe->err = "fe, r-cell and surrogate contexts must share one stream";
        return RC_EINVAL;
    }
    const int ne = fe->ne;
    cudaStream_t st = fe->stream;
    if (!fe->d_u) {
        CKF(fe, dalloc(fe->allocs, &fe->d_u, 15 * (size_t)ne));
        CKF(fe, dalloc(fe->allocs, &fe->d_smean, 6 * (size_t)ne));
        CKF(fe, dalloc(fe->allocs, &fe->d_spread, ne));
        CKF(fe, dalloc(fe->allocs, &fe->d_Pmd, 9 * (size_t)ne));
        CKF(fe, dalloc(fe->allocs, &fe->d_nmd, 1));
        CKF(fe, dalloc(fe->allocs, &fe->d_Fhist, (size_t)RC_REPLAY_MAX * ne * 9));
        CKF(fe, dalloc(fe->allocs, &fe->d_nfrozen, ne));
        CKF(fe, dalloc(fe->allocs, &fe->d_rmask, ne));
        fe->h_flag.assign(ne, 0);
        fe->h_nfrozen.assign(ne, 0);
    }
    int e;
    // 1. boundary conditions and element F
    apply_bc(fe, lambda, st);
    fe_launch_F(fe->npe, fe->d_conn, fe->d_gradN, fe->d_d, fe->d_F, ne, st);
    // 2. surrogate for every point (keeps every recurrent state current)
    if ((e = sur_features(F_prev, fe->d_F, ne, fe->d_u, st)) != RC_OK) return e;
    if ((e = sur_step(sur, fe->d_u, ne, h_state, s_floor, fe->d_smean, fe->d_spread)) != RC_OK) return e;
    // 3. which points fall back to MD
    CKF(fe, cudaMemsetAsync(fe->d_nmd, 0, sizeof(int), st));
    fe_launch_decide(fe->d_spread, spread_on, spread_off, force_md, md_flag, fe->d_nmd, ne, st);
    if (spread_out)
        CKF(fe, cudaMemcpyAsync(spread_out, fe->d_spread, sizeof(float) * ne, cudaMemcpyDeviceToDevice, st));
    int nmd = 0;
    CKF(fe, cudaMemcpyAsync(&nmd, fe->d_nmd, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKF(fe, cudaMemcpyAsync(fe->h_flag.data(), md_flag, sizeof(int) * ne, cudaMemcpyDeviceToHost, st));
    CKF(fe, cudaMemcpyAsync(fe->h_nfrozen.data(), fe->d_nfrozen, sizeof(int) * ne, cudaMemcpyDeviceToHost, st));
    CKF(fe, cudaStreamSynchronize(st));
    // 4. a point returning to MD resumes from its frozen r-cell state (the state of
    //    its last MD increment) and first replays, increment by increment, the
    //    deformations it missed on the surrogate (R15); points replay side by side,
    //    each masked out once its own history is used up
    int max_k = 0, replayed = 0;
    for (int e = 0; e < ne; e++)
        if (fe->h_flag[e] != 0) {
            max_k = std::max(max_k, fe->h_nfrozen[e]);
            replayed += fe->h_nfrozen[e];
        }
    for (int j = 0; j < max_k; j++) {
        fe_launch_replay_mask(md_flag, fe->d_nfrozen, j, fe->d_rmask, ne, st);
        if ((e = rcell_set_active(rc, fe->d_rmask, RC_DEVICE)) != RC_OK) return e;
        if ((e = rcell_set_deformation(rc, fe->d_Fhist + (size_t)j * ne * 9, RC_DEVICE)) != RC_OK) return e;
        if ((e = rcell_run(rc, n_steps, n_avg)) != RC_OK) return e;  // the all-MD kernel sequence
    }
    // 5. MD for the flagged points at this increment (the others keep their frozen
    //    r-cell state)
    if (nmd > 0) {
        if ((e = rcell_set_active(rc, md_flag, RC_DEVICE)) != RC_OK) return e;
        if ((e = rcell_set_deformation(rc, fe->d_F, RC_DEVICE)) != RC_OK) return e;
        if ((e = rcell_run(rc, n_steps, n_avg)) != RC_OK) return e;
        if ((e = rcell_stress(rc, nullptr, nullptr, fe->d_Pmd, RC_DEVICE)) != RC_OK) return e;
    }
    // 6. merge: MD P where flagged, J sigma_sur F^-T elsewhere; record the missed
    //    increment of every surrogate point; then the FE update
    fe_launch_surrogate_merge(md_flag, fe->d_smean, fe->d_F, fe->d_Pmd, fe->d_P, ne, st);
    fe_launch_track_frozen(md_flag, fe->d_F, fe->d_Fhist, fe->d_nfrozen, ne, RC_REPLAY_MAX, st);
    fe_launch_copy_F(fe->d_F, F_prev, ne, st);
    CKF(fe, cudaGetLastError());
    if ((e = fe_update(fe, fe->d_P, RC_DEVICE)) != RC_OK) return e;
    if (n_md) *n_md = nmd;
    if (n_replayed) *n_replayed = replayed;
    return RC_OK;
}

int fe_get_P(fe_ctx *fe, double *P, int where) {
    if (!fe || !P) return RC_EINVAL;
    CKF(fe, cudaMemcpyAsync(P, fe->d_P, sizeof(double) * 9 * fe->ne,
                            where == RC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, fe->stream));
    if (where == RC_HOST) CKF(fe, cudaStreamSynchronize(fe->stream));
    return RC_OK;
}

int fe_get_state(fe_ctx *fe, double *d, double *v) {
    if (!fe) return RC_EINVAL;
    CKF(fe, cudaStreamSynchronize(fe->stream));
    if (d) CKF(fe, cudaMemcpy(d, fe->d_d, sizeof(double) * 3 * fe->nn, cudaMemcpyDeviceToHost));
    if (v) CKF(fe, cudaMemcpy(v, fe->d_v, sizeof(double) * 3 * fe->nn, cudaMemcpyDeviceToHost));
    return RC_OK;
}

void fe_destroy(fe_ctx *fe) {
    if (!fe) return;
    if (fe->stream) cudaStreamSynchronize(fe->stream);
    for (void *p : fe->allocs) cudaFree(p);
    if (fe->ev) cudaEventDestroy(fe->ev);
    if (fe->own_stream && fe->stream) cudaStreamDestroy(fe->stream);
    delete fe;
}

}  // extern "C"
