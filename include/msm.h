/*
 * msm.h -- C ABI of libmsm_gb300.so: the multilevel summation method (MSM)
 * for Coulomb energies and forces, velocity Verlet dynamics around it and the
 * parareal time-parallel driver, as hand-written sm_103a CUDA kernels.
 *
 * Source of the method: J. Pazurikova and L. Matyska, "Parallel-in-time
 * method for calculation of long-range electrostatic interactions"
 * (arXiv:1309.1889).  Sec. 2 states the problem (inputs q_i, r_i, v_i;
 * outputs trajectories, forces, energy), Sec. 3 the MSM, Sec. 4 parareal.
 *
 * Conventions shared by every entry point
 *   - Units: nm, ps, e, amu, kJ/mol; k_e = 1/(4 pi eps0) = 138.935458 kJ mol^-1 nm e^-2.
 *   - Arrays are plain C-contiguous FP64 (atoms x 3 for vectors).  Array
 *     arguments may be device pointers of the current device or host
 *     pointers (pageable or pinned); the library detects which and stages
 *     host data through its own device buffers.  An array allocated on
 *     another GPU is rejected with MSM_EINVAL before anything is launched.
 *     The caller keeps ownership of every array; the library only borrows
 *     it for the duration of the call.
 *   - box[6] = {x0, y0, z0, Lx, Ly, Lz} (host memory): the open,
 *     non-periodic domain of the grids.  An atom is inside when, on every
 *     axis, t = (x - x0) * (1/h) (IEEE FP64, 1/h rounded once) satisfies
 *     0 <= t < floor(L/h) + 1, i.e. [x0, x0 + L) rounded up to whole cells of
 *     the finest spacing h; any other atom makes the call fail with MSM_ERANGE.
 *   - stream is a cudaStream_t (NULL = legacy default stream).  Every entry
 *     point returns after its results are complete and readable: it
 *     synchronises the stream once at the end to read the device status word.
 *   - Return 0 on success, a negative MSM_E* code on failure;
 *     msm_last_error() gives a message for the calling thread.  No error
 *     leaves a kernel running; no kernel traps.
 */
#ifndef MSM_GB300_H
#define MSM_GB300_H

#include <stdint.h>

#if defined(__GNUC__)
#define MSM_API __attribute__((visibility("default")))
#else
#define MSM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define MSM_OK        0
#define MSM_EINVAL   -1   /* bad parameters, n < 0, NaN/Inf coordinates        */
#define MSM_ERANGE   -2   /* an atom outside box (detected on the device)      */
#define MSM_ENOMEM   -3   /* device allocation failed                          */
#define MSM_ECUDA    -4   /* a CUDA runtime call failed                        */
#define MSM_ETIMEOUT -5   /* a bounded device-side wait ran out                */
#define MSM_ENOCONV  -6   /* SHAKE/RATTLE or parareal did not converge         */

#define MSM_FP64 0        /* every stage in FP64                               */
#define MSM_FP32 1        /* FP32 pair/grid/stencil arithmetic; FP64 state,
                             energy/virial reductions and top level            */

#define MSM_MODEL_CHARGES 0  /* bare point charges: the paper's Coulomb sum     */
#define MSM_MODEL_WATER   1  /* + rigid 3-site water completion (see msm_system) */

/* Electrostatics method (msm_params.method).  The MSM is the fine propagator's
 * method (Sec. 3); Sec. 5 weighs cheaper methods for the parareal coarse
 * propagator and keeps two, both sums over the pairs closer than a (no grids):
 *   MSM_METHOD_CUTOFF  simple cutoff, U = 1/2 sum_{i != j, r_ij < a} k_e q_i q_j / r_ij
 *                      (the paper's chosen coarse propagator)
 *   MSM_METHOD_WOLF    Wolf summation (Wolf, Keblinski, Phillpot & Eggebrecht 1999):
 *                      pair term k_e q_i q_j [erfc(alpha r)/r - erfc(alpha a)/a],
 *                      self term -k_e [erfc(alpha a)/(2a) + alpha/sqrt(pi)] q_i^2,
 *                      alpha = msm_params.wolf_alpha (1/nm)
 * For both, forces are the exact gradient (the shift is constant inside a),
 * potentials phi_i = dU/dq_i, n_levels is ignored, h is only the edge of the
 * cells the pair search uses (and the box contract is the same), and the water
 * completion skips its intramolecular pairs instead of subtracting them. */
#define MSM_METHOD_MSM    0
#define MSM_METHOD_CUTOFF 1
#define MSM_METHOD_WOLF   2

#define MSM_FLAG_GRAPHS   1  /* md_run: steps after the first replay one captured CUDA graph
                                (the first too, when a previous call captured it for the
                                same arrays, geometry and buffers)                         */
#define MSM_FLAG_AUTOTUNE 2  /* time the pair passes' i-group column widths (with
                                MSM_FLAG_BRICKS: brick shapes) on the first evaluation of
                                each geometry and keep the fastest; never changes a result */
#define MSM_FLAG_SCALAR_PAIRS 4  /* diagnostic, FP32 only: the short-range Coulomb and LJ
                                passes take their queued neighbours one at a time instead
                                of two per packed FP32x2 step; the same bits, slower (off
                                by default)                                                */
#define MSM_FLAG_CLUSTER_PAIRS 8  /* FP32, MSM or simple cutoff: the short-range Coulomb pass
                                on cluster pairs (8 i atoms x 4 j atoms from columns of
                                2 x 2 cells, clusters culled by bounding box) instead of
                                32-atom groups; the same sums in another order: agrees
                                with the default pass to rounding, not bitwise; ignored
                                for FP64, Wolf summation and MSM_FLAG_SCALAR_PAIRS (off by
                                default: measured no faster)                               */
#define MSM_FLAG_BRICKS 16  /* diagnostic: the short-range and LJ passes give each warp a brick
                                of cells (~20 atoms) instead of a group of 32 atoms cut from a
                                column of cells; the same bits, slower (off by default)      */

/* Method parameters (Sec. 3).
 *   a          cutoff of the short-range part g* (nm); the level-k lattice
 *              cutoff is 2^{k+1} a (eq. split and the g^k definitions)
 *   h          finest grid spacing (nm); level k has spacing 2^k h
 *   n_levels   number of grids l (levels 0..l-1); level l-1 is summed densely
 *   precision  MSM_FP64 or MSM_FP32
 *   coulomb_k  k_e (0 selects 138.935458)
 *   gamma_kind 0 = C^2 Taylor smoothing (the only one the paper writes out)
 *   basis_kind 0 = cubic C1 numerical Hermite Phi (the paper's p = 3 choice)
 *   model      MSM_MODEL_CHARGES or MSM_MODEL_WATER
 *   lj_sigma, lj_epsilon   O-O Lennard-Jones of the water completion
 *   d_oh, d_hh rigid O-H and H-H distances of the water completion (nm)
 *   wall_k, wall_width     water completion: harmonic flat-bottom wall that
 *              keeps atoms inside the open domain; an atom closer than
 *              wall_width to a box face feels 1/2 wall_k (wall_width - d)^2
 *              (kJ/mol/nm^2, nm; wall_k = 0 disables it)
 *   flags      MSM_FLAG_* bits (default: GRAPHS | AUTOTUNE).  None but
 *              CLUSTER_PAIRS changes a result bit: a graph replays exactly the
 *              launches of an eager step, the short-range sum adds each atom's
 *              neighbours in ascending sorted order whatever the i grouping
 *              (32-atom groups of any column width, or bricks of any shape),
 *              and the packed and scalar pair steps do the same IEEE
 *              operations.  Graphs are not used while the profiler is on.
 *   list_skin  md_run only: Verlet-list skin (nm) of the short-range sum;
 *              lists hold pairs within a + list_skin and are rebuilt when an
 *              atom has moved more than list_skin/2 (0 = cell search every
 *              step; the default).  Exact either way: pairs are still tested against a.
 *   method     MSM_METHOD_* (default MSM_METHOD_MSM)
 *   mts_steps  md_run, md_run_batched and the parareal propagators: multiple
 *              time stepping (Sec. 3 notes that the MSM suits a multiple-
 *              time-step integrator), the impulse method with SHAKE/RATTLE.
 *              The grid part (k_e q_i times the interpolated long-range
 *              gradient, minus the excluded pairs' smooth part) is the slow
 *              force, evaluated once per outer step of mts_steps steps and
 *              applied as two impulses of mts_steps*dt/2 folded into the
 *              outer step's first and last half kicks; the short-range pair
 *              sum, Lennard-Jones and wall are the fast force, every step.
 *              n_steps must be a multiple of mts_steps; the recorded U of a
 *              step inside an outer step is its fast energy plus the last slow
 *              energy (the whole energy at the ends of outer steps).  0 or 1:
 *              plain velocity Verlet (default 0); > 1 needs MSM_METHOD_MSM.
 *   wolf_alpha damping of MSM_METHOD_WOLF (1/nm, >= 0)  */
typedef struct msm_params {
    double  a;
    double  h;
    int32_t n_levels;
    int32_t precision;
    double  coulomb_k;
    int32_t gamma_kind;
    int32_t basis_kind;
    int32_t model;
    int32_t flags;
    double  lj_sigma;
    double  lj_epsilon;
    double  d_oh;
    double  d_hh;
    double  wall_k;
    double  wall_width;
    double  list_skin;
    int32_t method;
    int32_t mts_steps;
    double  wolf_alpha;
} msm_params;

/* An MD system in the library's layout.  Rigid water occupies the first
 * 3*n_mol atoms as (O, H, H) triples; any further atoms are single sites.
 * x, v are updated in place by md_run.  q, m are per-atom; lj (nullable)
 * flags the Lennard-Jones sites (1) of the water completion.  If f is
 * non-NULL, md_run starts from f/energy when f_valid is 1 (skipping the
 * evaluation at the start positions) and leaves F, U of the final positions
 * there with f_valid = 1, so a run split over several calls costs one
 * evaluation per step. */
typedef struct msm_system {
    int64_t        n;
    int64_t        n_mol;
    double        *x;      /* n*3 */
    double        *v;      /* n*3 */
    const double  *q;      /* n   */
    const double  *m;      /* n   */
    const uint8_t *lj;     /* n, nullable */
    double         box[6];
    double        *f;      /* n*3, nullable: forces carried between md_run calls */
    int32_t        f_valid;/* 1: f and energy hold F(x) and U(x) for the current x */
    int32_t        reserved0;
    double         energy; /* U(x) when f_valid (host field) */
} msm_system;

typedef struct msm_handle msm_handle;

/* Fill *p with the defaults: a = 1.2, h = 0.25, 3 levels, FP32, k_e, C^2
 * gamma, cubic Phi, point charges, graphs and autotuning on, TIP3P-like O-O
 * LJ and geometry, no wall, no Verlet lists (skin 0). */
MSM_API void msm_default_params(msm_params *p);

/* Create a handle (validates *p; allocates nothing on the device until the
 * first evaluation).  The handle owns its scratch: sorted atoms, cell lists,
 * grids for every level, stencil and top-level tables.  Not thread-safe:
 * one handle per host thread / stream.  Errors: MSM_EINVAL (among others
 * when n_levels > 1 and the lattice-cutoff radius, the largest r with
 * r h < 2a, exceeds 12 grid points). */
MSM_API int  msm_create(const msm_params *p, msm_handle **out);
MSM_API void msm_destroy(msm_handle *h);

/* One MSM energy/force evaluation (Sec. 3, worked example steps 1-9):
 * short range, anterpolation, restriction and lattice cutoff on levels
 * 0..l-2, top level, prolongation, interpolation.
 *   pos[n*3], q[n]       inputs (device or host)
 *   energy[1]            U = 1/2 sum_i q_i phi_i (device or host, nullable)
 *   forces[n*3]          F_i = -dU/dr_i (nullable)
 *   potentials[n]        phi_i = dU/dq_i, self-interaction removed (nullable)
 *   virial[1]            sum_i r_i . F_i (nullable)
 * Errors: MSM_EINVAL (n < 0, non-finite coordinate), MSM_ERANGE (atom
 * outside box), MSM_ENOMEM, MSM_ECUDA. */
MSM_API int  msm_energy_forces(msm_handle *h, int64_t n, const double *pos, const double *q,
                       const double box[6], double *energy, double *forces,
                       double *potentials, double *virial, void *stream);

/* Same evaluation for independent systems of uneven sizes in one call:
 * system s owns atoms offsets[s] .. offsets[s+1]-1 (host array of n_sys+1,
 * offsets[0] = 0) and box boxes[6*s .. 6*s+5] (host).  energies[n_sys]
 * (device or host); other arrays are concatenated per atom.  All systems go
 * through the same launches (one per stage for the whole batch; the
 * per-system geometry sits in a device table), and each system's results are
 * bitwise those of msm_energy_forces on it alone.  The paper runs its
 * independent fine propagators in parallel (Sec. 4); a batch is the GPU form
 * of that. */
MSM_API int  msm_energy_forces_batched(msm_handle *h, int32_t n_sys, const int64_t *offsets,
                               const double *pos, const double *q, const double *boxes,
                               double *energies, double *forces, double *potentials,
                               void *stream);

/* Energy, forces and potentials of an msm_system under the handle's model
 * (MSM plus, for MSM_MODEL_WATER, intramolecular exclusions and O-O LJ).
 * Same outputs and errors as msm_energy_forces. */
MSM_API int  msm_system_forces(msm_handle *h, const msm_system *sys, double *energy,
                       double *forces, double *potentials, void *stream);

/* Velocity Verlet (Sec. 2: forces F = -dU/dr, move the atoms), with
 * SHAKE/RATTLE for the rigid triples: n_steps steps of length dt (ps) on
 * sys->x, sys->v (device, updated in place).  uk (nullable, device or
 * host) receives (U, K) before the first step and after every step:
 * 2*(n_steps+1) values.  With MSM_FLAG_GRAPHS the first step is launched
 * kernel by kernel and the others replay a CUDA graph of one step (captured
 * on a private stream, launched on the caller's).  Errors as above plus
 * MSM_ENOCONV (constraints). */
MSM_API int  md_run(msm_handle *h, msm_system *sys, double dt, int32_t n_steps, double *uk, void *stream);

/* Energies and forces of n_sys independent msm_systems (uneven sizes and
 * boxes) in one batched evaluation under the handle's model: x, q, lj of each
 * system are gathered (device or host), forces go to systems[s].f (nullable;
 * f_valid and energy are then set), energies[n_sys] (host, nullable).  Each
 * system's results equal msm_system_forces on it alone, bit for bit. */
MSM_API int  msm_system_forces_batched(msm_handle *h, int32_t n_sys, msm_system *systems, double *energies,
                                       void *stream);

/* md_run for n_sys independent systems stepped together: every stage of
 * every step is one launch for the whole batch.  x, v (and f when non-NULL)
 * of each system are updated in place; forces are carried in only if every
 * system has f with f_valid = 1.  uk (nullable, device or host) receives
 * n_sys blocks of 2*(n_steps+1) values, system s first.  Each system's
 * trajectory equals md_run on it alone, bit for bit. */
MSM_API int  md_run_batched(msm_handle *h, int32_t n_sys, msm_system *systems, double dt, int32_t n_steps,
                            double *uk, void *stream);

/* Parareal (Sec. 4): lambda^{k+1}_{n+1} = G(lambda^{k+1}_n) + F(lambda^k_n) - G(lambda^k_n),
 * the fine propagations F of one iteration run as one batch (md_run_batched
 * over the slices not yet exact), G sequentially;
 * evaluated as F + (G_new - G_old) in FP64; F and G are md_run with their own
 * parameters, time steps and step counts (dtG*stepsG must equal dtF*stepsF).
 * state0 gives the system and lambda_0 = (x, v).  slices_x/slices_v
 * (device or host, (n_slices+1)*n*3 each) receive lambda_0..lambda_{n_slices}
 * of the last iterate.  Stops when max |x^{k+1} - x^k| <= tol (nm) or after
 * max_iter iterations; *iters_done and *last_dx (host) report the outcome.
 * The water completion's rigid molecules are projected back onto their
 * constraints after every correction when a correction distorted them by more
 * than 10x the fine propagator's SHAKE tolerance (exact states pass unchanged).
 * Returns MSM_ENOCONV, with a message starting "parareal:", if tol was not met
 * or if the coarse propagator broke down on a corrected state (the iteration
 * diverged); the last complete iterate is written either way.  The correction
 * sweep of an iteration is enqueued without host synchronisation (each coarse
 * propagation's status is kept on the device); the host reads the sweep's
 * outcome once per iteration.  G (or F) may use a cutoff method (msm_params
 * method, Sec. 5). */
MSM_API int  parareal_run(const msm_params *G, double dtG, int32_t stepsG,
                  const msm_params *F, double dtF, int32_t stepsF,
                  const msm_system *state0, int32_t n_slices, int32_t max_iter, double tol,
                  double *slices_x, double *slices_v, int32_t *iters_done, double *last_dx,
                  void *stream);

/* Resume parareal (Sec. 4) from a checkpoint: slices_x/v hold the iterate
 * lambda^k (n_slices + 1 states, slot 0 = state0's x, v) that parareal_run or
 * parareal_resume wrote after k = iters_before iterations (for instance a run
 * stopped by its max_iter, or a saved copy of one).  The coarse propagations
 * G(lambda^k_n) the next correction needs are recomputed from those states (a
 * G sweep), then at most max_iter more iterations run; the iterates equal
 * those of one uninterrupted parareal_run bit for bit.  *iters_done counts
 * all iterations, k included.  state0 supplies q, m, lj, box and the atom
 * counts (its x, v must equal slot 0).  Other arguments, outputs and errors
 * as parareal_run; iters_before < 0 is MSM_EINVAL. */
MSM_API int  parareal_resume(const msm_params *G, double dtG, int32_t stepsG,
                  const msm_params *F, double dtF, int32_t stepsF,
                  const msm_system *state0, int32_t n_slices, int32_t iters_before, int32_t max_iter,
                  double tol, double *slices_x, double *slices_v, int32_t *iters_done,
                  double *last_dx, void *stream);

/* Parareal over a sliding computational window (Sec. 4: the iteration runs on
 * a window of time points).  At most `window` slices [b, e) are iterated at
 * once: each iteration runs F on every window slice as one batch and the
 * correction sweep from lambda_b, which is final.  Then b moves past slice b
 * (its end F(lambda_b) is exact) and past the following slices whose end
 * moved by at most tol (max |x^{k+1} - x^k|, nm), and new slices enter the
 * window with the coarse propagation of its last state as their first
 * iterate.  Device memory holds window + 1 states (plus the batch's copies)
 * instead of n_slices + 1, so long runs fit.  Arguments as parareal_run;
 * max_iter bounds the iterations of the whole run (each iteration finalises
 * at least one slice, so n_slices iterations always suffice).  slices_x/v
 * receive every slice end: final ones for the converged slices, the last
 * iterate for the rest (slices the window never reached are not written).
 * *last_dx is the largest change of the last iteration.  With window =
 * n_slices and tol = 0 the iterates equal parareal_run's; with window = 1 the
 * run is the serial fine propagation.  Returns MSM_ENOCONV ("parareal: ...")
 * if max_iter ran out first or the coarse propagator broke down; the last
 * complete iterate is written either way. */
MSM_API int  parareal_run_window(const msm_params *G, double dtG, int32_t stepsG,
                  const msm_params *F, double dtF, int32_t stepsF,
                  const msm_system *state0, int32_t n_slices, int32_t window, int32_t max_iter,
                  double tol, double *slices_x, double *slices_v, int32_t *iters_done,
                  double *last_dx, void *stream);

/* Budget for the device memory the library allocates: the scratch and staging
 * buffers of every handle in the process (callers' arrays are not counted, nor
 * the static array of msm_cell_list_noalloc).  bytes <= 0 removes the budget
 * (the default).  An allocation that would take the library's holdings past
 * the budget fails as a failed cudaMalloc does: the call that needed it
 * returns MSM_ENOMEM, and the handle stays usable (a later call with room
 * allocates again).  Returns the bytes held when called.  No counterpart in
 * the paper: it lets a caller that shares the GPU with other allocators cap
 * the library's share. */
MSM_API int64_t msm_set_device_budget(int64_t bytes);

/* Inspection of the last evaluation on h (host outputs, synchronous).
 * msm_grid_shape: level k's point counts (nx, ny, nz) and index origin
 * (lo_x, lo_y, lo_z): grid point mu sits at x0 + mu * 2^k h.
 * msm_stage_grid: which = 0 charges q^k, 1 lattice-cutoff potential
 * u^{k,cut} (k < l-1), 2 potential u^k; out[nx*ny*nz] as FP64, x fastest.
 * msm_cell_list: the bit-exact cell binning of the last evaluation: perm[n]
 * (atoms ordered by finest-grid cell, then index) and cell_start[ncells+1],
 * *ncells receiving the cell count (cells floor(L/h)+1 per axis, x fastest).
 * msm_stage_atoms: which = 0 short-range potential sum_j q_j g*(r_ij) (n),
 * 1 short-range force sum (n*3), both before k_e, in original atom order
 * (for the cutoff methods: the pair sums of their pair term).  The cutoff
 * methods have no grids: msm_grid_shape and msm_stage_grid return MSM_EINVAL. */
MSM_API int  msm_grid_shape(msm_handle *h, int32_t level, int64_t shape[3], int64_t lo[3]);
MSM_API int  msm_stage_grid(msm_handle *h, int32_t level, int32_t which, double *out, int64_t count);
MSM_API int  msm_cell_list(msm_handle *h, int64_t *perm, int64_t *cell_start, int64_t *ncells);
MSM_API int  msm_stage_atoms(msm_handle *h, int32_t which, double *out, int64_t count);

/* Per-stage timing with CUDA events recorded on the caller's stream around
 * every stage of every evaluation and step while enabled (off by default).
 * msm_profile_read copies up to max stages' accumulated milliseconds and
 * launch counts (stage i is named by msm_stage_name(i)) and, if reset != 0,
 * clears them.  Returns the number of stages. */
MSM_API int  msm_profile_enable(msm_handle *h, int32_t on);
MSM_API int  msm_profile_read(msm_handle *h, double *ms, int64_t *launches, int32_t max, int32_t reset);
MSM_API const char *msm_stage_name(int32_t stage);

/* Exact number of ordered pairs (i, j), j != i, with r_ij < a in the last
 * evaluation on h: the algorithmic work unit of the short-range sum. */
MSM_API int  msm_count_pairs(msm_handle *h, int64_t *ordered_pairs);

/* Cell binning and stable sort without any device allocation.  The paper has
 * no counterpart: this serves callers that must not allocate device memory,
 * for example a host program whose device memory is owned by another
 * allocator with a fixed budget, or a time-critical loop that cannot afford
 * the device-wide synchronisation that cudaMalloc/cudaFree imply.
 *   pos[n*3]        device, FP64 atom positions
 *   box, h          host; the same binning contract as every other entry
 *                   point (t = (x - x0)*(1/h), cell = floor(t), key =
 *                   (cz*ny + cy)*nx + cx with floor(L/h)+1 cells per axis)
 *   perm[n]         device output: atoms ordered by (cell key, atom index)
 *   cell_start[cell_start_len >= ncells+1]  device output: first slot of each
 *                   cell, cell_start[ncells] = n
 * The output equals msm_cell_list's after an evaluation of the same atoms.
 * Scratch lives in a 24 MiB static device array inside the library, held by
 * every GPU that loads it until the process exits: 4 bytes per atom plus 4
 * per cell must fit (about 1 M atoms with 4 M cells); larger requests return
 * MSM_EINVAL, as do host pointers and arrays on another GPU.  The first call on a device, with that
 * device current, looks up the array's device address; make that first call
 * before any stream capture.  Every call reuses the same array and clears
 * the parts that must start at zero; calls that overlap on the GPU (other
 * streams, other host threads) race on it and must be serialised by the
 * caller.  Synchronises the stream before returning.  Errors: MSM_EINVAL,
 * MSM_ERANGE, MSM_ECUDA. */
MSM_API int  msm_cell_list_noalloc(int64_t n, const double *pos, const double box[6], double h,
                                   int32_t *perm, int32_t *cell_start, int64_t cell_start_len,
                                   void *stream);

/* Verlet-list statistics of h since its creation (up to max values):
 * builds, overflows (a capacity was exceeded or a brick could not be encoded:
 * that step used the cell search and the capacity grew), entries-per-atom
 * capacity, O-O entries-per-atom capacity, row slots per brick, and the
 * largest entries per atom, O-O entries per atom and row count seen at a
 * build. */
MSM_API int  msm_list_stats(msm_handle *h, int64_t *out, int32_t max);

/* Diagnostic: the binary64 <-> binary32 conversions the FP32 kernels use
 * between the FP64 state and FP32 arithmetic, computed (like there) with
 * integer operations on the IEEE 754 bit fields.  x32[i] = x[i] rounded to
 * binary32 (to nearest, ties to even); y64[i] = y[i] as binary64.  Both agree
 * with the hardware conversions except that magnitudes below 2^-126 become
 * signed zero; NaN stays NaN.  x, x32, y, y64 are device arrays of n elements
 * owned by the caller; stream is a cudaStream_t (NULL: the legacy default
 * stream).  Synchronises the stream.  Errors: MSM_EINVAL (n < 0, NULL or host
 * arrays), MSM_ECUDA. */
MSM_API int  msm_diag_convert(int64_t n, const double *x, float *x32, const float *y, double *y64,
                              void *stream);

/* Number of kernels this library launched since load (all handles). */
MSM_API int64_t msm_kernel_launches(void);

/* Message for the last error on the calling thread ("" if none). */
MSM_API const char *msm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MSM_GB300_H */
