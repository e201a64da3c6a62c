/*
 * cfneb.h -- C ABI of the GB300 (sm_103a) cell-filter nudged elastic band
 * library.
 *
 * One relaxation step of a band of images (arXiv 2510.16721) is computed
 * entirely by CUDA kernels of this library:
 *   - cell filter, inverse map (Sec. II.C): B = X_lat / c, D = sqrt(B),
 *     h = h0 D, R = R~ D;
 *   - cell-list build over all periodic images of every atom (the per-atom
 *     energy of Sec. II.B, Eq. U, depends on the neighbours of i in the
 *     periodic crystal);
 *   - Lennard-Jones, Tersoff or NEP-style energy, forces and virial
 *     V = -1/2 sum_ij r^ij (x) f^ij (Sec. II.B, Eqs. V, V2);
 *   - cell filter, forward map: atom rows F D^T and lattice rows
 *     1/2 D^-T V D^-1 / c (Sec. II.C; the 1/2 makes the lattice force the
 *     exact conjugate of B, whose increment is D dD^T + dD D^T);
 *   - NEB force f_NEB = f_real(perp) + f_spring (Sec. II.A) with the upwind
 *     tangent and climbing image the paper cites (Sec. I);
 *   - FIRE update of the interior images (the optimiser is not named by the
 *     paper, Sec. III);
 *   - image insertion / deletion from the spacing of neighbouring images
 *     (Sec. III).
 *
 * Conventions
 *   - Every function returns an int status: 0 = CFNEB_OK, negative = error,
 *     positive = informational.  cfneb_status_string() names it.
 *   - Arrays passed in are caller owned, read during the call and copied;
 *     arrays passed out are caller owned and filled during the call.  All
 *     pointers in this header are HOST pointers.
 *   - Positions are Cartesian, row-major n x 3 (double).  A cell is the 3x3
 *     lattice matrix with the lattice vectors h1, h2, h3 as ROWS (Sec. II.B,
 *     below Eq. epsilon), row-major.
 *   - The image count N includes both endpoints; the endpoints never move.
 *   - A band owns its device memory (allocated at creation, sized for
 *     n_max images) and is bound to the CUDA stream given at creation: the
 *     library orders its own work after the work already queued on that
 *     stream, and work queued on it later runs after the library's.  A band
 *     is not thread safe.
 *   - Units: LJ in reduced units (eps, sigma); Tersoff and NEP-style in eV
 *     and Angstrom.
 */
#ifndef CFNEB_H
#define CFNEB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define CFNEB_OK 0
#define CFNEB_NOT_CONVERGED 1        /* cfneb_relax ran out of steps           */
#define CFNEB_ERR_INVALID_ARG (-1)   /* NULL pointer, bad enum, bad size       */
#define CFNEB_ERR_SHAPE_MISMATCH (-2)/* endpoints differ in atom count/types    */
#define CFNEB_ERR_OUT_OF_MEMORY (-3) /* device allocation failed               */
#define CFNEB_ERR_HBM_BUDGET (-4)    /* batch memory budget exceeded           */
#define CFNEB_ERR_CUDA (-5)          /* a CUDA runtime call failed             */
#define CFNEB_ERR_NONFINITE (-6)     /* NaN/Inf in forces, energies or state   */
#define CFNEB_ERR_NOT_SPD (-7)       /* lattice coordinate B lost positivity   */
#define CFNEB_ERR_NBR_OVERFLOW (-8)  /* more list neighbours than capacity, or a
                                        cell narrower than (rc + skin) / 7     */
#define CFNEB_ERR_TIMEOUT (-9)       /* a bounded device wait gave up          */
#define CFNEB_ERR_STATE (-10)        /* call not valid in the current state    */

/* ---- enums ------------------------------------------------------------- */
#define CFNEB_LJ 0
#define CFNEB_TERSOFF 1
#define CFNEB_NEP 2
/* NEP-style potential: Chebyshev basis size 6, 4 radial and 2 angular
 * functions, Legendre orders 1..4, 16 hidden units: 261 weights. */
#define CFNEB_NEP_N_WEIGHTS 261

/* cell_factor value selecting the scale J = Omega0^(1/3) n^(1/6) of the
 * generalized solid-state NEB (Sheppard et al. 2012): the lattice rows then
 * have the stiffness per unit of X of the atom rows at any n, where c = n
 * makes them ever softer (slower to relax) as n grows (Sec. II.C leaves the
 * scale open) */
#define CFNEB_CELL_FACTOR_J (-1.0)

#define CFNEB_ROTFREE_B 0   /* lattice coordinate B = D D^T (Sec. II.C end)   */
#define CFNEB_DEFGRAD_D 1   /* lattice coordinate D = h0^-1 h (Sec. II.C)     */

#define CFNEB_FP64 0        /* all arithmetic in double                       */
#define CFNEB_MIXED 1       /* FP32 pair/three-body arithmetic and vectors;
                               FP64 energies, reductions and 3x3 cell work    */

/* ---- structures -------------------------------------------------------- */
typedef struct cfneb_band cfneb_band;   /* opaque, owned by the library */

typedef struct {
    int32_t n_atoms;
    const int32_t *types;     /* n_atoms species ids, or NULL; one species  */
    const double *positions;  /* n_atoms x 3, Cartesian, row-major          */
    double cell[9];           /* rows = lattice vectors h1, h2, h3          */
} cfneb_structure;

typedef struct {
    int32_t kind;             /* CFNEB_LJ, CFNEB_TERSOFF or CFNEB_NEP        */
    /* Lennard-Jones: phi = 4 eps [(sigma/r)^12 - (sigma/r)^6], cut at rc,
       minus phi(rc) when shift_energy != 0                                  */
    double eps, sigma, rc;
    int32_t shift_energy;
    /* Tersoff (1988 form, lambda3 = 0): A, B, lambda1, lambda2, beta, n, c,
       d, h, R, D.  All zero selects Tersoff's 1988 carbon parameters.       */
    double tersoff[11];
    /* NEP-style descriptor + neural-network site energy (single species;
       the neuroevolution potential of the paper's examples, Sec. IV, with
       caller-given weights): f_c(r) = (1 + cos(pi r / rc)) / 2; radial
       basis f_k = (T_k(x) + 1)/2 f_c, x = 2 (r/rc - 1)^2 - 1, k < 6;
       g^R_n = sum_k cR[n][k] f_k (n < 4), g^A_n = sum_k cA[n][k] f_k
       (n < 2); descriptors q_n = sum_j g^R_n(r_ij) and q_nl = sum_jk
       g^A_n(r_ij) g^A_n(r_ik) P_l(cos theta_jk), l = 1..4 (order q_0..q_3,
       q_01..q_04, q_11..q_14); U_i = sum_h w1[h] tanh(sum_d W0[h][d] q_d -
       b0[h]) - b1.  nep_weights: CFNEB_NEP_N_WEIGHTS doubles in the order
       cR (4x6), cA (2x6), W0 (16x12), b0 (16), w1 (16), b1; copied at
       creation.  nep_rc: the cutoff (> 0; the neighbour lists hold at most
       16 entries within nep_rc + skin).                                    */
    const double *nep_weights;
    double nep_rc;
} cfneb_potential;

typedef struct {
    int32_t enabled;          /* 0: fixed cell (h = h0 for every image)      */
    int32_t variant;          /* CFNEB_ROTFREE_B (default) or CFNEB_DEFGRAD_D */
    double cell_factor;       /* c in X_lat = c B (> 0); CFNEB_CELL_FACTOR_J
                                 selects J = Omega0^(1/3) n^(1/6) (Omega0 the
                                 initial cell's volume); other values <= 0
                                 select n_atoms                              */
    double pressure;          /* external pressure P: H = U + P Omega        */
} cfneb_cell_filter;

typedef struct {
    double k_spring;          /* spring constant (energy / length^2)         */
    int32_t climb;            /* climbing image on from the first step       */
    int32_t precision;        /* CFNEB_FP64 or CFNEB_MIXED                   */
    double dt, dt_max, maxstep; /* FIRE: initial/maximum step, per-row clamp */
    const double *interior_noise; /* (n_images-2) x n_atoms x 3 displacements
                                     added to the interior images' R~ after
                                     linear interpolation, or NULL           */
    int32_t adaptive;         /* spacing-driven insertion / deletion          */
    int32_t n_min, n_max;     /* image-count bounds; n_max is the capacity   */
    int32_t k_ref, cooldown;  /* refinement check every k_ref steps, at least
                                 cooldown steps after the previous change    */
    double alpha_ins, alpha_del; /* insert if l_s > alpha_ins mean(l); delete
                                 if l_(j-1) + l_j < alpha_del mean(l)        */
    double bin_scale;         /* cell-list bin width / list cutoff (>= 0.25);
                                 0 selects the tuned default                 */
    double skin;              /* neighbour-list skin (length units): cell
                                 lists and lists cover rc + skin and are kept
                                 while no pair can have crossed into rc (a
                                 bound from the largest displacement and the
                                 cell change since the build); 0 rebuilds at
                                 every evaluation; < 0 selects the default
                                 (Tersoff and NEP-style 0.15, LJ 0.12 rc).
                                 At most rc.
                                 LJ bands with a skin and at most 2^17 atoms
                                 keep per-atom neighbour lists; other LJ
                                 bands walk the cell list at every
                                 evaluation.                                 */
} cfneb_options;

/* Fill *opt with the defaults: k 0.1, climb on, FP64, FIRE dt 0.1,
 * dt_max 1.0, maxstep 0.2, no noise, adaptive off, n_min 3, n_max = the
 * image count given at creation, k_ref 10, cooldown 20, alpha_ins 1.5,
 * alpha_del 0.5, bin_scale 0 (tuned), skin -1 (per-potential default).
 * Returns CFNEB_OK. */
int cfneb_default_options(cfneb_options *opt);

/* Create a band between two endpoint structures (Sec. III: the cell filter
 * turns each image into generalised coordinates before forces are taken).
 *   h0 = cell of `initial`; each endpoint is mapped to X = (R~, c B) with
 *   R~ = s h0 and B = D D^T, D = h0^-1 h (Sec. II.C); the final endpoint's
 *   fractional coordinates are unwrapped to the nearest periodic image of
 *   the initial ones; interior images are the linear interpolation of X
 *   plus `interior_noise`.  Endpoint energies are evaluated once.
 * n_images >= 3.  cuda_stream is a cudaStream_t (NULL = legacy default).
 * On success *out owns the band; destroy it with cfneb_destroy_band.
 * Errors: INVALID_ARG (also for coincident endpoints -- every atom on the
 * same periodic site to 1e-12 in fractional coordinates and, with the cell
 * filter on, the same cell -- which leave no path: every tangent would
 * vanish), SHAPE_MISMATCH, OUT_OF_MEMORY, CUDA, NOT_SPD.  Arguments are
 * checked on the host before any CUDA call. */
int cfneb_create_band(const cfneb_structure *initial, const cfneb_structure *final,
                      int32_t n_images, const cfneb_potential *potential,
                      const cfneb_cell_filter *cell_filter, const cfneb_options *options,
                      void *cuda_stream, cfneb_band **out);

/* Run n_steps relaxation steps (map-back, cell list, forces, cell filter,
 * NEB projection, FIRE).  Queued on the band's stream; returns without
 * waiting unless adaptive refinement needs a host decision.  A step whose
 * f_NEB already meets the tolerance of the last cfneb_relax call moves
 * nothing.  Errors raised on the device surface at the next synchronising
 * call (relax, get_path, get_state). */
int cfneb_step(cfneb_band *band, int32_t n_steps);

/* Iterate until fmax = max row norm of f_NEB over the interior images
 * (atom rows and the 3 lattice rows) is below `fmax`, or max_steps steps
 * were taken.  *steps_done = steps taken by this call; *converged = 1 if
 * the tolerance was met.  Returns CFNEB_OK, CFNEB_NOT_CONVERGED or an
 * error.  Synchronises with the device every few steps. */
int cfneb_relax(cfneb_band *band, double fmax, int64_t max_steps, int64_t *steps_done,
                int32_t *converged);

/* Insert the linear midpoint of images after_index and after_index + 1
 * (0 <= after_index < N - 1, N < n_max).  Resets FIRE.  Endpoints are left
 * bit-identical. */
int cfneb_insert_image(cfneb_band *band, int32_t after_index);

/* Delete interior image `index` (0 < index < N - 1, N > n_min).  Resets
 * FIRE. */
int cfneb_delete_image(cfneb_band *band, int32_t index);

/* Copy the current path to the host.  Any output pointer may be NULL.
 *   *n_images  = N
 *   positions  = N x n_atoms x 3 Cartesian positions (R = R~ D)
 *   cells      = N x 9 cells h = h0 D
 *   energies   = N energies (U + P Omega) of these positions and cells,
 *                from an FP64 energy pass (on either precision): barriers
 *                read from them carry FP64 totals
 *   fmax       = largest f_NEB row norm at the last step (0 before any step)
 * Synchronises. */
int cfneb_get_path(const cfneb_band *band, int32_t *n_images, double *positions,
                   double *cells, double *energies, double *fmax);

/* Copy the full state to the host (checkpoints, parity checks).  Any
 * pointer may be NULL.  Rows per image: n_atoms + 3.
 *   X       = N x (n+3) x 3 generalised coordinates (R~ rows, then c B)
 *   F       = N x (n+3) x 3 generalised forces of the last evaluation
 *   Fneb    = N x (n+3) x 3 NEB forces of the last step (endpoints 0)
 *   virials = N x 9 virials V (row-major V_mn)
 *   fire    = 4 doubles: dt, alpha, steps with positive power, steps taken
 *   climbing_index = index of the climbing image of the last step (-1 none)
 * Synchronises. */
int cfneb_get_state(const cfneb_band *band, double *X, double *F, double *Fneb,
                    double *virials, double *fire, int32_t *climbing_index);

/* Restore the generalised coordinates of every image (a checkpoint taken
 * with cfneb_get_state; Sec. II.C coordinates X = (R~, c B)).  X holds
 * N x (n+3) x 3 doubles for the band's current image count N, endpoints
 * included; values are rounded to the band's storage precision.  FIRE is
 * reset (v = 0, dt = dt0), the endpoints are evaluated again and every
 * image rebuilds its cell and neighbour lists at the next evaluation.
 * Errors: INVALID_ARG (NULL or a non-finite entry), NOT_SPD (an endpoint's
 * lattice rows), CUDA.  Synchronises. */
int cfneb_set_state(cfneb_band *band, const double *X);

/* ---- image-range shards ----------------------------------------------------
 * A band of many images can be spread over several devices (or processes)
 * as contiguous image ranges (the paper's scale, Sec. I and Sec. III: ~100
 * images of 1e5 atoms).  Each range is a band of its own whose two end
 * images are ghosts: copies of the neighbouring ranges' boundary images (or
 * the true endpoints).  One step of the whole band, driven by the caller:
 *   1. cfneb_shard_evaluate on every range (energies and forces of its
 *      interior images; energies[N] returned, end images as last set);
 *   2. exchange: each range's first and last interior image (with
 *      cfneb_shard_get_image) go to the neighbours' ghosts
 *      (cfneb_shard_set_ghost);
 *   3. the climbing image is the argmax of every range's interior energies
 *      (lowest global index on ties); each range is told its local index,
 *      or -1;
 *   4. cfneb_shard_project: f_NEB of the interior images (Sec. II.A) and the
 *      range's FIRE sums: sums[4] = F_NEB.v, |F_NEB|^2, |v|^2 and the
 *      largest squared row norm of f_NEB;
 *   5. the caller sums the first three over the ranges and takes the
 *      maximum of the fourth (fmax = its square root; converged if below
 *      the tolerance), then cfneb_shard_move on every range with the same
 *      global sums: the FIRE decision (identical on every range) and move.
 * cfneb_shard_enable turns a band into a range (FIRE reset; not for bands in
 * a batch or with adaptive refinement); set its images first with
 * cfneb_set_state.  Host pointers; every call synchronises.  Errors:
 * INVALID_ARG (not a shard, bad index or side, non-finite X), CUDA, and the
 * band's status bits. */
int cfneb_shard_enable(cfneb_band *band);
int cfneb_shard_evaluate(cfneb_band *band, double *energies);
int cfneb_shard_get_image(const cfneb_band *band, int32_t index, double *X, double *energy);
int cfneb_shard_set_ghost(cfneb_band *band, int32_t side, const double *X, double energy);
int cfneb_shard_project(cfneb_band *band, int32_t climbing_index, double *sums);
int cfneb_shard_move(cfneb_band *band, const double *sums);

/* Per-image scalars of the last step (Sec. II.A): energies[N] the
 * energies (U + P Omega) the step's tangent and climbing image used (in the
 * mixed path from FP32 site energies summed in FP64; cfneb_get_path reports
 * FP64 energies); dots[N x 10] for the interior images |dX+|^2, |dX-|^2,
 * dX+.dX-, F.dX+, F.dX-, F.F, F.v, v.v, dX+.v, dX-.v (dX+ = X_{i+1} - X_i,
 * dX- = X_i - X_{i-1}, F the generalised force, v the FIRE velocity before
 * the move); coef[N x 2] the a, b with f_NEB = F + a dX+ + b dX-.
 * Endpoint entries are 0 (their energy is reported).  Any pointer may be
 * NULL.  Synchronises. */
int cfneb_get_image_scalars(const cfneb_band *band, double *energies, double *dots,
                            double *coef);

/* Release the band and its device memory. */
int cfneb_destroy_band(cfneb_band *band);

/* Single-point evaluation of `count` structures (any cells, any sizes):
 * energies[count], forces[sum n_i x 3] (Cartesian, structures back to
 * back), virials[count x 9].  Forces and virials come from the kernels of a
 * relaxation step in the requested precision; energies from the FP64
 * energy pass.  Output pointers may be NULL.  Synchronises. */
int cfneb_evaluate(const cfneb_structure *structures, int32_t count,
                   const cfneb_potential *potential, int32_t precision, void *cuda_stream,
                   double *energies, double *forces, double *virials);

/* ---- batches: many bands, one launch per kernel --------------------------
 * A batch steps all its member bands together: every kernel of a step is
 * launched once over the tiles of all members (uneven atom and image counts
 * mixed), the steps run as captured CUDA graphs (eight steps per graph; a
 * remainder as one-step graphs), and each band keeps its
 * own FIRE state, convergence test and refinement.  Results of a band do not
 * depend on the other members (reductions use fixed per-band slots).
 * Members must share the precision; LJ, Tersoff and NEP-style bands may be
 * mixed.
 * While a band is a member its work is queued on the batch's stream; the
 * band calls above stay valid on it.  The batch does not own its bands. */
typedef struct cfneb_batch cfneb_batch;

/* Create an empty batch.  budget_bytes bounds the summed device memory of
 * the members (0 = unbounded).  cuda_stream as in cfneb_create_band. */
int cfneb_batch_create(int32_t precision, uint64_t budget_bytes, void *cuda_stream,
                       cfneb_batch **out);

/* Add a band (CFNEB_ERR_HBM_BUDGET if it does not fit the budget,
 * CFNEB_ERR_INVALID_ARG if the precision differs or it is already in a
 * batch). */
int cfneb_batch_add(cfneb_batch *batch, cfneb_band *band);

/* Remove a band; it returns to its own stream.  The band is not destroyed. */
int cfneb_batch_remove(cfneb_batch *batch, cfneb_band *band);

/* n_steps steps of every member (members that converged under the last
 * cfneb_batch_relax or spent their move budget do not move). */
int cfneb_batch_step(cfneb_batch *batch, int32_t n_steps);

/* Relax every member until its fmax < tol or it made max_steps moves
 * (counted per band from this call).  *n_converged = members converged.
 * Synchronises every few steps. */
int cfneb_batch_relax(cfneb_batch *batch, double fmax, int64_t max_steps, int32_t *n_converged);

/* Per-member state, members in the order they were added (removed ones
 * skipped): moves taken, converged flag, fmax of the last step, status
 * (0 or a CFNEB_ERR code).  Arrays of length >= the member count; any may
 * be NULL.  *count = member count.  Synchronises. */
int cfneb_batch_status(cfneb_batch *batch, int32_t *count, int64_t *steps, int32_t *converged,
                       double *fmax, int32_t *status);

/* Device memory of a band, and of a batch's members against its budget. */
int cfneb_band_bytes(const cfneb_band *band, uint64_t *bytes);
int cfneb_batch_bytes(const cfneb_batch *batch, uint64_t *used, uint64_t *budget);

/* Per-kernel CUDA-event timing of batch steps (as cfneb_profile). */
int cfneb_batch_profile(cfneb_batch *batch, int32_t enable);
int cfneb_batch_profile_read(cfneb_batch *batch, int32_t kernel_id, double *total_ms,
                             int64_t *launches);

/* Release the batch (members are removed, not destroyed). */
int cfneb_batch_destroy(cfneb_batch *batch);

/* ---- serving: continuous batching of band requests ------------------------
 * A server keeps one batch on the GPU.  Requests (two endpoints and band
 * options) are submitted with an arrival time on the server's clock (seconds
 * since cfneb_server_create).  cfneb_server_run admits arrived requests in
 * arrival order as the device-memory budget allows (a request that does not
 * fit waits), steps every resident band together, and retires a band as soon
 * as it converges (fmax < its tolerance), spends its move budget or fails;
 * retired bands free their memory for the next admissions, so new bands join
 * while others are mid-relaxation.  Latency = retirement - arrival. */
typedef struct cfneb_server cfneb_server;

int cfneb_server_create(int32_t precision, uint64_t budget_bytes, void *cuda_stream,
                        cfneb_server **out);

/* Queue a request; inputs are copied.  *id receives its id (0, 1, ...). */
int cfneb_server_submit(cfneb_server *server, const cfneb_structure *initial,
                        const cfneb_structure *final, int32_t n_images,
                        const cfneb_potential *potential, const cfneb_cell_filter *cell_filter,
                        const cfneb_options *options, double fmax, int64_t max_steps,
                        double arrival_s, int64_t *id);

/* Serve until every submitted request is retired or the server clock passes
 * until_s.  Returns CFNEB_OK, or CFNEB_NOT_CONVERGED if requests remain. */
int cfneb_server_run(cfneb_server *server, double until_s);

/* Result of a request: *state 0 queued, 1 running, 2 retired; latency in
 * seconds; moves; converged flag; barrier = max E - E(initial) from FP64
 * energies; status of the band (0 or a CFNEB_ERR code). */
int cfneb_server_result(cfneb_server *server, int64_t id, int32_t *state, double *latency_s,
                        int64_t *steps, int32_t *converged, double *barrier, int32_t *status);

/* Latency percentiles over retired requests, retired count, and the served
 * throughput in atom-steps/s (moving images x atoms x moves of every
 * retired request, over the server clock). */
int cfneb_server_stats(cfneb_server *server, double *p50_s, double *p99_s, int64_t *retired,
                       double *atom_steps_per_s);

int cfneb_server_destroy(cfneb_server *server);

/* ---- autotuning of the cell-list bin shape ------------------------------
 * Times `steps` force evaluations of the band (no moves: the state is left
 * as it was) for each candidate bin width (0.5, 0.75, 1.0, 1.3 x cutoff),
 * keeps the fastest for the band and caches it for its class (potential,
 * precision, atom count and density buckets).  Bands created later with
 * options.bin_scale = 0 in a cached class start with the cached width.
 * Bands created with bin_scale = 0 reserve bins for the finest candidate;
 * untuned classes start at 0.5 (LJ) or 1.0 (Tersoff, NEP-style).
 * *best_scale receives the chosen width / cutoff.  Synchronises. */
int cfneb_autotune(cfneb_band *band, int32_t steps, double *best_scale);

/* Autotune one member per class and apply the result to every member of
 * that class.  Synchronises. */
int cfneb_batch_autotune(cfneb_batch *batch, int32_t steps);

/* Per-kernel timing.  With profiling on, each kernel launch of
 * cfneb_step is bracketed by CUDA events on the band's internal stream
 * (the stream the kernels run on; graphs are not used while profiling).
 * cfneb_profile_read returns the summed event time (ms) and launch count of
 * kernel `kernel_id` since profiling was switched on; cfneb_kernel_name
 * names ids 0 .. cfneb_kernel_count()-1. */
int cfneb_profile(cfneb_band *band, int32_t enable);
int cfneb_profile_read(cfneb_band *band, int32_t kernel_id, double *total_ms,
                       int64_t *launches);
int32_t cfneb_kernel_count(void);
const char *cfneb_kernel_name(int32_t kernel_id);

/* Work counters of the last evaluation of the interior images, summed over
 * them: *pairs = neighbour entries (i, j, shift) inside the cutoff,
 * *triples = ordered pairs of distinct neighbour entries of one atom (the
 * three-body terms of Tersoff and NEP-style; 0 for LJ).  Used to turn kernel times into
 * arithmetic rates.  Synchronises. */
int cfneb_get_work(const cfneb_band *band, double *pairs, double *triples);

/* The band's tuning: *bin_scale = cell-list bin width / list cutoff and
 * *blocks_per_sm = resident blocks per SM of the force kernel variant it
 * launches (FP32 LJ with lists: 5-8, FP32 Tersoff: 4-8; 0 where the
 * potential or precision has one variant).  cfneb_autotune picks both: the
 * bin width from timed evaluations with forced rebuilds, then the variant
 * at that width.  Any output pointer may be NULL.  Reads host state only. */
int cfneb_get_tuning(const cfneb_band *band, double *bin_scale, int32_t *blocks_per_sm);

/* Cell-list reuse counters summed over the interior image slots since the
 * band was created: *builds = cell-list (and neighbour-list) builds,
 * *evaluations = force evaluations; *skin = the skin in use.  The paper
 * prints no list policy: a skin is this library's way to skip rebuilds and
 * leaves every force unchanged up to rounding.  Synchronises.  Any output
 * pointer may be NULL. */
int cfneb_get_list_stats(const cfneb_band *band, int64_t *builds, int64_t *evaluations,
                         double *skin);

/* Number of kernel launches one cfneb_step makes for this band when it
 * rebuilds cell and neighbour lists (for launch accounting; a step in which
 * every image keeps its lists skips the 6-7 rebuild kernels). */
int cfneb_launches_per_step(const cfneb_band *band, int32_t *launches);

/* ---- evaluation without device allocation --------------------------------
 * The paper has no counterpart to this entry point.  It serves callers that
 * cannot call cudaMalloc: processes whose allocator owns all of the device
 * memory (a framework's caching pool, a fixed arena sized at start-up), and
 * services that must not allocate once serving (an allocation can fail or
 * stall at any time).
 *
 * Lennard-Jones energy, forces and virial (FP64, the same kernels and
 * results as cfneb_evaluate with CFNEB_FP64) of one periodic structure of
 * n_atoms <= CFNEB_NOALLOC_MAX_ATOMS atoms.  Scratch memory is one
 * file-scope device array of about 8.5 MB, present on every GPU that loads
 * the library until the process exits; nothing is allocated or freed.
 *   d_positions  DEVICE pointer, n_atoms x 3 Cartesian positions (caller owned)
 *   cell         HOST pointer, 9 doubles, rows = lattice vectors
 *   eps, sigma, rc, shift_energy: as in cfneb_potential
 *   d_energy     DEVICE pointer to 1 double, or NULL
 *   d_forces     DEVICE pointer to n_atoms x 3 doubles, or NULL
 *   d_virial     DEVICE pointer to 9 doubles, or NULL
 *   cuda_stream  the stream the work is queued on (NULL = legacy default)
 * Waits for the stream and returns the status the kernels raised:
 * CFNEB_ERR_NONFINITE for a non-finite energy (overlapping atoms).
 * n_atoms above the maximum, a NULL position or cell pointer, a
 * non-finite cell entry or eps, sigma, rc, a singular cell, or a cell
 * narrower than rc / 7 along a lattice direction (the cell list reaches 7
 * bins to each side) return CFNEB_ERR_INVALID_ARG before any GPU work.
 * The array's device address is looked up, and kept, once per CUDA context
 * (the first call in a context, with that context current, does it).
 * Every call shares the one array and leaves its contents behind (the
 * counts that must start at zero are cleared by each call), so calls that
 * overlap on the GPU -- other streams, or unsynchronised host threads --
 * race. */
#define CFNEB_NOALLOC_MAX_ATOMS 32768
int cfneb_lj_evaluate_noalloc(const double *d_positions, int32_t n_atoms, const double *cell,
                              double eps, double sigma, double rc, int32_t shift_energy,
                              double *d_energy, double *d_forces, double *d_virial,
                              void *cuda_stream);

/* Human-readable name of a status code. */
const char *cfneb_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* CFNEB_H */
