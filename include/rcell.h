/*
 * rcell.h -- C ABI of the GB300 r-cell engine for the hierarchical FEM <-> MD
 * coupling of Murashima, Urata & Li (arXiv:1902.09171).
 *
 * Behind every finite-element quadrature point sits a representative cell
 * (r-cell) of atoms.  Per load increment each r-cell takes the local
 * deformation gradient F, splits it as F = Q R (Sec. 2.1), moves its atoms into
 * the triangular box H_MD = R H(0) through Delta R = R(t) R(t-1)^{-1}
 * (Eq. LAMMPS2), runs fixed-box MD, and returns its time-averaged virial stress
 * rotated back to the FE frame (sigma_FEM = Q sigma_MD Q^T) together with the
 * first Piola-Kirchhoff stress P = J sigma_FEM F^{-T} (Eq. Pmd) that the FE
 * internal force (Eq. f) consumes.
 *
 * General rules for every call
 *   - Return value: an rc_status code (RC_OK = 0).  Nothing aborts, throws
 *     across the ABI or traps on the GPU.  After any error other than RC_ECUDA
 *     the context stays usable; rcell_last_error() gives a one-line reason.
 *   - The library owns all device memory it allocates (in rcell_create /
 *     fe_create, plus lazily grown sample buffers in rcell_run).  The caller
 *     owns every array it passes; inputs are copied before the call returns
 *     (host inputs) or before the enqueued work reads them (device inputs must
 *     stay valid until the stream reaches that work).
 *   - All GPU work is enqueued on the CUDA stream given at creation (NULL =
 *     the legacy default stream).  Calls marked "synchronous" wait for it.
 *   - `where` arguments say whether a pointer is host memory (RC_HOST) or
 *     device memory of the current device (RC_DEVICE).
 *   - Matrices are row-major double[9] with F_iJ = dx_i / dX_J; a box matrix H
 *     holds the three box vectors as COLUMNS (r = H s, Eq. LAMMPS1).
 *   - Stresses are tension-positive Cauchy stresses in Voigt order
 *     (xx, yy, zz, xy, xz, yz).  (Table 1 prints the opposite, pressure-like
 *     sign.)  Units: GPa for RC_UNITS_METAL, eps/sigma^3 for RC_UNITS_LJ.
 *   - Device-side failures (degenerate F, box too thin, broken bond, lost atom,
 *     capacity overflow, non-finite energy) are recorded per cell in a status
 *     word; they surface as the return value of the next synchronous call
 *     (rcell_stress, rcell_sync, rcell_get_*).
 */
#ifndef RCELL_H
#define RCELL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rcell_ctx rcell_ctx; /* opaque: a batch of r-cells on one GPU   */
typedef struct fe_ctx fe_ctx;       /* opaque: an explicit hex-8 FE mesh        */

typedef enum {
    RC_OK = 0,
    RC_EINVAL = 1,     /* bad argument (null pointer, size, parameter)           */
    RC_ENOMEM = 2,     /* device or host allocation failed                       */
    RC_ECUDA = 3,      /* CUDA runtime error; the context may be unusable        */
    RC_EDEGEN = 4,     /* det F <= 0: no rotation times positive stretch (Sec. 2.1) */
    RC_EBOX = 5,       /* a perpendicular box width fell below 2 r_list           */
    RC_EBOND = 6,      /* a FENE bond reached r >= R0                             */
    RC_ELOST = 7,      /* an atom moved more than the skin within one step        */
    RC_EOVERFLOW = 8,  /* neighbour / bin capacity exceeded                       */
    RC_ENAN = 9,       /* non-finite force, energy or virial                      */
    RC_ETIMEOUT = 10,  /* a bounded device-side wait gave up                      */
    RC_ESTATE = 11     /* call out of order (e.g. stress before any run)          */
} rc_status;

enum { RC_HOST = 0, RC_DEVICE = 1 };
enum { RC_POT_LJ = 0, RC_POT_SC = 1, RC_POT_KG = 2 };
enum { RC_UNITS_METAL = 0, RC_UNITS_LJ = 1 };

/* Interaction and integration parameters shared by every cell of a batch.
 *   RC_POT_LJ : U = 4 eps [(sigma/r)^12 - (sigma/r)^6] for r < rc, unshifted.
 *   RC_POT_SC : Sutton-Chen EAM, E = eps [1/2 sum_i sum_j!=i (a/r)^n
 *               - c sum_i sqrt(rho_i)], rho_i = sum_j!=i (a/r)^m, r < rc;
 *               `sigma` holds a.
 *   RC_POT_KG : Kremer-Grest bead-spring (Sec. 3.2): LJ (eps, sigma, rc) between
 *               non-bonded pairs; bonded pairs get FENE
 *               -1/2 k_fene R0^2 ln(1 - (r/R0)^2) plus WCA (LJ cut and shifted
 *               at 2^{1/6} sigma) and no non-bonded LJ.
 * Integration: velocity Verlet with time step dt; force-form Langevin
 * thermostat with damping time tau (tau <= 0: none), temperature kT (energy
 * units), noise from Philox4x32-10 keyed by `seed`.  skin: Verlet-list skin
 * (r_list = rc + skin); lists are rebuilt when an atom has moved more than
 * skin/2 since the last build.  max_step > 0 limits every atom's displacement
 * per step to max_step by rescaling its half-step velocity (a soft start for
 * overlapping initial states; 0 = off). */
typedef struct {
    int potential;       /* RC_POT_*                                           */
    int units;           /* RC_UNITS_*                                         */
    double eps, sigma, rc;
    double n, m, c;      /* Sutton-Chen                                        */
    double k_fene, R0;   /* Kremer-Grest bonds                                 */
    double skin;
    double mass, kT, tau, dt;
    uint64_t seed;
    double max_step;
} rcell_params;

/* One r-cell's initial state (host memory).
 *   H0     : 9 doubles, upper-triangular initial box (the paper's H(0) is
 *            orthogonal; a diagonal H0 is the usual case).
 *   x0, v0 : 3 n_atoms doubles, Cartesian positions / velocities (atom-major).
 *   bonds  : 2 n_bonds ints, 0-based atom indices (RC_POT_KG only; at most 4
 *            bonds per atom).
 * Atom index ("tag") order of x0 is the order every per-atom output uses. */
typedef struct {
    int n_atoms;
    const double *H0;
    const double *x0;
    const double *v0;
    int n_bonds;
    const int *bonds;
} rcell_init;

/* Create a batch of n_cells r-cells (uneven atom counts allowed) on the current
 * CUDA device.  stream: a cudaStream_t (NULL = default stream).  Copies all
 * inputs; *out receives the context.  Errors: RC_EINVAL (bad sizes/params,
 * non-finite H0, x0 or v0, box thinner than 2 r_list), RC_ENOMEM, RC_ECUDA.
 * Synchronous. */
int rcell_create(const rcell_params *params, int n_cells, const rcell_init *cells, void *stream, rcell_ctx **out);

/* Sec. 2.1 + Eq. LAMMPS2: for every cell c take F_c (n_cells x 9 doubles,
 * row-major), factor F = Q R with R_ii > 0 (FP64 Gram-Schmidt on the GPU),
 * set the box to R H0, remap atom positions x <- (R R_prev^{-1}) x (FP64 math on
 * the FP32 positions; velocities unchanged) and schedule a neighbour rebuild.
 * where: location of F.  A host F with a non-finite entry is refused with
 * RC_EINVAL before any launch.  Cells with det F <= 0 get RC_EDEGEN and keep
 * their previous state; cells whose new box is thinner than 2 r_list get
 * RC_EBOX.  Asynchronous. */
int rcell_set_deformation(rcell_ctx *ctx, const double *F, int where);

/* Run n_steps fixed-box MD steps on every cell (one setup force evaluation +
 * n_steps velocity-Verlet steps) and record the instantaneous virial stress of
 * the last n_avg steps (0 <= n_avg <= n_steps).  Captured into a CUDA graph
 * per (n_steps, n_avg) after its first use.  Asynchronous. */
int rcell_run(rcell_ctx *ctx, int n_steps, int n_avg);

/* Per-cell activity mask (n_cells ints, `where` memory): cells with mask 0 are
 * skipped by rcell_set_deformation, rcell_run and rcell_eval -- their atoms, box,
 * R(t-1) and random-stream counter stay as they are -- until re-enabled.  All
 * cells start active.  Asynchronous for device masks. */
int rcell_set_active(rcell_ctx *ctx, const int *mask, int where);

/* Time-averaged stress of the last rcell_run, per cell:
 *   sigma        n_cells x 6: mean of Q sigma_MD(t) Q^T over the sampled steps
 *                (sigma_MD(t) = -(sum m v (x) v + W(t)) / det H, W the pair virial);
 *   sigma_stderr n_cells x 6 or NULL: blocking standard error of that mean
 *                (largest over blocking levels that keep >= 16 blocks);
 *   P            n_cells x 9 or NULL: P = J sigma F^{-T} (Eq. Pmd).
 * All outputs in `where` memory.  Synchronous when where == RC_HOST; returns
 * the first per-cell error status, or RC_ESTATE if no samples exist. */
int rcell_stress(rcell_ctx *ctx, double *sigma, double *sigma_stderr, double *P, int where);

/* Evaluate conservative forces, potential energy and pair virial at the current
 * positions (no integration, no thermostat), rebuilding lists as needed.
 * Results are read with rcell_get_atoms / rcell_get_energy.  Asynchronous. */
int rcell_eval(rcell_ctx *ctx);

/* Per-cell potential energy and pair virial W (9, row-major, compression-
 * positive) of the last rcell_eval, host memory (n_cells and n_cells x 9;
 * either may be NULL).  Synchronous. */
int rcell_get_energy(rcell_ctx *ctx, double *pe, double *W);

/* Copy one cell's per-atom state to host memory in tag order: positions
 * (wrapped into the current box), velocities, and the forces of the last
 * rcell_eval (any pointer may be NULL; 3 n_atoms doubles each).  Synchronous. */
int rcell_get_atoms(rcell_ctx *ctx, int cell, double *x, double *v, double *f);

/* Current MD box (9 doubles, upper triangular) and the Q, R of the last
 * deformation (9 each); any may be NULL.  Host memory.  Synchronous. */
int rcell_get_box(rcell_ctx *ctx, int cell, double *H, double *Q, double *R);

/* Neighbour list of one cell as ordered tag pairs (i, j): every pair whose
 * distance (with its periodic image) was below r_list at the last list build.
 * pairs: 2 * max_pairs ints (host); *count receives the number of pairs
 * (RC_EOVERFLOW if it exceeds max_pairs).  Synchronous. */
int rcell_get_neighbors(rcell_ctx *ctx, int cell, int *pairs, long max_pairs, long *count);

/* Per-step samples of the last rcell_run for one cell (host memory, n_avg
 * entries each, any may be NULL): MD-frame stress (n_avg x 6), potential
 * energy, kinetic energy.  Synchronous. */
int rcell_get_series(rcell_ctx *ctx, int cell, double *stress, double *pe, double *ke);

/* Wait for the stream; return the first per-cell error (or RC_OK). */
int rcell_sync(rcell_ctx *ctx);

/* Clear the per-cell error words (after the caller has handled them).  A cell
 * whose error arose inside a run stopped there: it holds the positions of the
 * step that failed or of the one before, so restore a checkpoint of it
 * (rcell_restore) before running it again where that matters. */
int rcell_clear_status(rcell_ctx *ctx);

/* Tuning knobs (chosen by the autotuner; any value < 0 keeps the current):
 *   threads_per_atom : 1, 2, 4 or 8 lanes cooperate on one atom's neighbours,
 *                      walking the list software-pipelined (the next group's
 *                      gathers in flight while a group is evaluated); 0 = one
 *                      lane per atom with a plain walk compiled for more
 *                      resident warps per SM (pays on large batches)
 *   use_graphs       : 0/1, capture rcell_run into CUDA graphs
 * All settings give the same results up to summation order. */
int rcell_set_tuning(rcell_ctx *ctx, int threads_per_atom, int use_graphs);

/* Failure-injection limits, with no counterpart in the paper (any value < 0
 * keeps the current one):
 *   max_neighbors : per-atom Verlet-list capacity used from now on, a multiple
 *                   of 4 in [4, the capacity allocated at creation]; 0 restores
 *                   that capacity.  Lists that would hold more entries are
 *                   truncated and the cell reports RC_EOVERFLOW.  Every list is
 *                   rebuilt at the next step.
 *   wait_polls    : polls of the bounded device-side wait of the shared-memory
 *                   staging (rcell_set_staging) before it gives up with
 *                   RC_ETIMEOUT; RC_WAIT_POLLS_DEFAULT at creation.  A wait
 *                   that gives up still lets the copies it issued land before
 *                   its block exits.
 * RC_EINVAL for a capacity outside the range.  Synchronises the stream when a
 * value changes. */
#define RC_WAIT_POLLS_DEFAULT (1 << 22)
int rcell_set_limits(rcell_ctx *ctx, int max_neighbors, int wait_polls);

/* Shared-memory staging of whole r-cells: with 1, every CTA first copies its
 * r-cell's records into shared memory (TMA bulk copy) and gathers neighbours
 * there -- only for batches whose largest cell has at most 12800 atoms; with 0
 * (the default) neighbours are gathered from global memory through the
 * read-only cache.  Both give the same results up to summation order. */
int rcell_set_staging(rcell_ctx *ctx, int staged);

/* Molecular statics (Sec. 2.2, Eq. CGPR1): relax the atoms of every active
 * cell without an error at fixed box to a local minimum of the potential
 * energy, starting from the current positions (after rcell_set_deformation
 * these are the Cauchy-Born guess F H(0) S of the previous configuration, the
 * r^ge of the paper).  The minimiser is FIRE (Bitzek et al., Phys. Rev. Lett.
 * 97, 170201, 2006; constants n_min 5, f_inc 1.1, f_dec 0.5, alpha 0.1,
 * f_alpha 0.99), one FIRE state per cell, a semi-implicit Euler step with the
 * atom mass: a cell stops once max_i |f_i| < f_tol (force units) at the start
 * of an iteration.  dt0: initial step, dt_max: largest step (time units, dt_max
 * >= dt0 > 0); dmax > 0 caps every atom's move per iteration (its velocity is
 * scaled down; <= 0: no cap).  At most max_iter iterations.  iters_out (n_cells host ints, or
 * NULL) receives each cell's number of moves before convergence (-1: not
 * converged, or skipped).  Velocities are zero afterwards.  Synchronous.
 * RC_EINVAL for bad arguments; cell errors as for rcell_run. */
int rcell_minimize(rcell_ctx *ctx, int max_iter, double f_tol, double dt0, double dt_max, double dmax,
                   int *iters_out);

/* Eq. PK1 / Eq. CGPR2 (Sec. 2.2): the first Piola-Kirchhoff stress of every
 * cell from the pair sum over its current positions,
 *   P_MD = 1/(2 Omega_0) sum_{i != j} dE/dr_ij r_ij (x) R_ij / r_ij,
 * with R_ij = H(0) H^{-1} r_ij the separation in the reference box and
 * Omega_0 = det H(0) (potential part only, no kinetic term); rotated to the FE
 * frame, P = Q P_MD, and sigma = P F^T / J (tension-positive, Voigt xx yy zz
 * xy xz yz with symmetrised off-diagonals).  Stress units as rcell_stress.
 * sigma: n_cells x 6, P: n_cells x 9 row-major; either may be NULL; where:
 * RC_HOST (synchronous, returns the first cell error) or RC_DEVICE. */
int rcell_stress_static(rcell_ctx *ctx, double *sigma, double *P, int where);

/* Neighbour-list builds per cell since creation (the initial build, one after
 * every deformation, and those the skin test triggered): counts receives
 * n_cells host values.  Synchronous.  RC_EINVAL for NULL arguments. */
int rcell_get_rebuilds(rcell_ctx *ctx, unsigned long long *counts);

/* Number of cells, total atoms, and the number of kernels the last rcell_run
 * enqueued (for launch accounting); any pointer may be NULL. */
int rcell_info(const rcell_ctx *ctx, int *n_cells, long *n_atoms, long *launches_last_run);

/* Measurement helper with no counterpart in the paper: the FP32 fused
 * multiply-add throughput (TFLOP/s, FMA = 2 FLOP) this GPU sustains, from a
 * kernel of independent FMA chains filling every SM (about 5 ms), timed with
 * CUDA events on `stream` (NULL: the default stream).  *tflops receives the
 * result (0 on error).  Synchronous.  RC_EINVAL for a NULL tflops, RC_ECUDA
 * if a launch or an event fails. */
int rcell_fp32_peak(void *stream, double *tflops);

/* Measurement helper: run n_steps more MD steps (plus a re-application of the
 * current F and a stress reduction) launching kernels one by one, with CUDA
 * events on the context's stream around every launch; ms_out (8 host doubles)
 * receives the mean duration in ms of one launch of: [0] neighbour sort, [1]
 * list build, [2] Sutton-Chen density pass, [3] force/integrate kernel on a
 * steady-state step that records no stress sample, [4] deformation (QR/box),
 * [5] remap, [6] stress reduction, [7] force/integrate kernel on a step that
 * records a sample (0 when not launched).  The steps are those of
 * rcell_run(n_steps, n_steps / 2): the MD state advances and the stress series
 * holds the samples of this run afterwards.  Synchronous. */
int rcell_profile_kernels(rcell_ctx *ctx, int n_steps, double *ms_out);

/* Per-cell checkpoint (the state the MD engine keeps between FE steps, Sec. 2.1:
 * positions, velocities, box, previous stretch R(t-1), random-stream counter).
 * rcell_checkpoint with buf == NULL returns the needed size in *bytes.  Host
 * buffers; synchronous.  rcell_restore requires the same atom count.  Both
 * schedule a neighbour rebuild for the cell, so a run after rcell_restore
 * repeats bit for bit the run that followed rcell_checkpoint. */
int rcell_checkpoint(rcell_ctx *ctx, int cell, void *buf, size_t *bytes);
int rcell_restore(rcell_ctx *ctx, int cell, const void *buf, size_t bytes);

/* Allocation-free stress reduction, for callers that cannot call cudaMalloc
 * when they need the stress: a host program that reserves the GPU's memory up
 * front for its own pool and forbids later device allocations, or a
 * latency-bound loop that must not take the implicit device synchronisation of
 * cudaFree / a growing cudaMalloc.  The paper has no counterpart: it is the
 * reduction of rcell_stress taken out of the context, with its scratch in a
 * fixed device array of the library instead of memory the context allocated.
 *   series       device, n_cells x n_avg x 6: MD-frame tension-positive stress
 *                samples (Voigt), e.g. what rcell_get_series returns
 *   Q, F         device, n_cells x 9 each: rotation and deformation gradient
 *   sigma        device, n_cells x 6: mean of Q sigma(t) Q^T (required)
 *   sigma_stderr device, n_cells x 6 or NULL: blocking standard error
 *   P            device, n_cells x 9 or NULL: J sigma F^{-T}
 *   stream       cudaStream_t to enqueue on (NULL = default stream)
 * n_cells * n_avg must not exceed 65536 (RC_EINVAL otherwise, nothing runs).
 * Allocates nothing and calls no allocating routine.  All calls share the
 * scratch array, which keeps the last call's contents: calls whose kernels
 * overlap on the GPU race.  The first call on a device looks the array up
 * (device current); make it before any stream capture.  RC_ECUDA when the
 * launch itself fails (an unrelated earlier error is not reported).
 * Asynchronous. */
int rcell_stress_reduce_static(const double *series, int n_cells, int n_avg, const double *Q, const double *F,
                               double *sigma, double *sigma_stderr, double *P, void *stream);

/* One-line description of the last error on this context (never NULL). */
const char *rcell_last_error(const rcell_ctx *ctx);

/* Free all device and host memory of the context (NULL is allowed). */
void rcell_destroy(rcell_ctx *ctx);

/* ---------------------------------------------------------------------------
 * Explicit finite elements (Sec. 2.2, Eq. f): 8-node hexahedra with one
 * centroid quadrature point (one r-cell per element), lumped mass
 * M = sum_e rho0 V_e / 8 per node, Flanagan-Belytschko stiffness hourglass
 * control (coefficient hg_coef, stiffness hg_coef V_e^{1/3}), mass-
 * proportional damping, central-difference update with time step dt.
 *   X       : nn x 3 reference coordinates (host)
 *   hex     : ne x 8 node ids (host), node order (-,-,-) (+,-,-) (+,+,-) (-,+,-)
 *             (-,-,+) (+,-,+) (+,+,+) (-,+,+) in natural coordinates
 *   bc_mask : nn x 3 ints, nonzero = prescribed DOF (host)
 *   bc_val  : nn x 3 doubles; prescribed displacement = lambda * bc_val (host)
 * ------------------------------------------------------------------------- */
int fe_create(const double *X, int nn, const int *hex, int ne, const int *bc_mask, const double *bc_val,
              double rho0, double dt, double damping, double hg_coef, void *stream, fe_ctx **out);

/* The same explicit FE with 4-node tetrahedra, the element the paper uses
 * (C3D4, Sec. 3.2): shape functions N = (1 - xi - eta - zeta, xi, eta, zeta)
 * on the reference tetrahedron, so grad N and F = I + sum_a d_a (x) grad N_a
 * are constant in the element (one quadrature point, one r-cell per element)
 * and there are no hourglass modes (no stabilisation).  Lumped mass
 * rho0 V / 4 per node.  tet: ne x 4 node ids (host) with positive orientation
 * ((X1 - X0) x (X2 - X0)) . (X3 - X0) > 0; other arguments as fe_create.
 * Every other fe_* call works on the returned context unchanged.  RC_EINVAL for
 * bad ids or an element of zero or negative volume. */
int fe_create_tet4(const double *X, int nn, const int *tet, int ne, const int *bc_mask, const double *bc_val,
                   double rho0, double dt, double damping, void *stream, fe_ctx **out);

/* Set the prescribed DOFs to lambda * bc_val.  With a predictor (fe_set_predictor)
 * every free DOF first moves by (lambda - lambda_prev) g, lambda_prev being the
 * load factor of the previous call on this context (0 at creation).
 * Asynchronous. */
int fe_apply_bc(fe_ctx *fe, double lambda);

/* Affine predictor of the load increment, with no counterpart in the paper's
 * explicit scheme: g (host, nn x 3, copied) is the displacement field per unit
 * load factor that the increment would produce in a homogeneous body, e.g.
 * g = (X_x, 0, 0) for uniaxial extension along x with the end face at
 * u_x = lambda L.  Every later boundary-condition update (fe_apply_bc, fe_step,
 * fe_step_surrogate) moves the free DOFs by (lambda - lambda_prev) g before the
 * one explicit update of the increment corrects them, so that a long bar loaded
 * at its end is stretched along its whole length from the first increment on
 * instead of in the elements next to the loaded face.  g = NULL removes the
 * predictor.  RC_EINVAL for a non-finite g.  Synchronous. */
int fe_set_predictor(fe_ctx *fe, const double *g);

/* Element deformation gradients F_e = I + sum_a d_a (x) grad_X N_a (ne x 9) into
 * `where` memory.  Synchronous when where == RC_HOST. */
int fe_get_F(fe_ctx *fe, double *F, int where);

/* Explicit update from element first Piola-Kirchhoff stresses P (ne x 9, in
 * `where` memory): assemble f_int (Eq. f, plus hourglass), then on free DOFs
 * v <- ((1 - c dt/2) v + dt (-f_int/m)) / (1 + c dt/2), d <- d + dt v.
 * Asynchronous. */
int fe_update(fe_ctx *fe, const double *P, int where);

/* One multiscale FE step (Fig. 1 of the paper): apply the BCs at lambda, compute
 * F_e, hand them to the r-cells (rcell_set_deformation), run n_steps MD steps
 * averaging the last n_avg, take P from rcell_stress, update the FE mesh.  The
 * r-cell batch must hold one cell per element.  u_out: nn x 3 host doubles or
 * NULL (synchronous when given).  Everything else stays on the device. */
int fe_step(fe_ctx *fe, rcell_ctx *rc, double lambda, int n_steps, int n_avg, double *u_out);

/* One FE step with the learned surrogate and MD fallback (the paper's Fig. 1
 * loop with the r-cell MD replaced where the ensemble agrees).  For every
 * element: surrogate input from (F_prev, F) and one recurrent step of every
 * member (include/surrogate.h); points whose ensemble spread exceeds spread_on
 * -- or exceeded it before and still exceed spread_off -- or all points when
 * force_md != 0, run n_steps of r-cell MD (rcell_set_active masks the rest) and
 * use its P; the others use P = J sigma_sur F^{-T}.  Then the FE update.
 * While a point uses the surrogate its r-cell stays frozen in the state of its
 * last MD increment, and the F of every increment it misses is recorded (up to
 * RC_REPLAY_MAX; beyond that the first RC_REPLAY_MAX - 1 and the latest are
 * kept).  When it returns to MD it first replays those increments one by one
 * (deformation, n_steps of MD) before running this one, so that its r-cell
 * follows the same per-increment deformation path as under all-MD (Eq. LAMMPS2).
 *   h_state  device, n_members x ne x 128 floats: recurrent states (zero to start)
 *   F_prev   device, ne x 9 doubles: F of the previous step (identity to start);
 *            overwritten with this step's F
 *   md_flag  device, ne ints: 0 surrogate, 1 MD because the spread tripped, 2 MD
 *            because force_md was set (read for the hysteresis, which only
 *            keeps tripped points on MD; then overwritten)
 *   spread_out device, ne floats or NULL: the ensemble spread of every point
 *   n_md     host, may be NULL: number of points that ran MD at this increment
 *   n_replayed host, may be NULL: number of missed increments replayed (r-cell
 *            MD runs of n_steps beyond the n_md of this increment)
 * fe, rc and sur must share one CUDA stream.  Synchronises once per step (to
 * skip the MD launches when no point needs them). */
#define RC_REPLAY_MAX 32
int fe_step_surrogate(fe_ctx *fe, rcell_ctx *rc, struct sur_ctx *sur, double lambda, int n_steps, int n_avg,
                      float spread_on, float spread_off, float s_floor, int force_md, float *h_state, double *F_prev,
                      int *md_flag, float *spread_out, int *n_md, int *n_replayed);

/* First Piola-Kirchhoff stresses (ne x 9) used by the last FE update, into
 * `where` memory.  Synchronous when where == RC_HOST. */
int fe_get_P(fe_ctx *fe, double *P, int where);

/* Displacements and velocities (nn x 3 each, host; either may be NULL). */
int fe_get_state(fe_ctx *fe, double *d, double *v);

void fe_destroy(fe_ctx *fe);

#ifdef __cplusplus
}
#endif
#endif /* RCELL_H */
