/*
 * maze.h - C ABI of the GB300 Poisson MaZe hot path (arxiv 2505.20418).
 *
 * Poisson MaZe treats the grid values of the electrostatic potential phi as
 * zero-mass auxiliary degrees of freedom and enforces the discretised Poisson
 * equation M phi = -4 pi q / h (Sec. II, Eq. linearproblem) as a SHAKE
 * constraint sigma = (h/4pi) M phi + q = 0 (Eq. Constraints) at every MD step.
 * One step (Sec. II, Fig. algorithm; Sec. III velocity Verlet):
 *
 *   S1 v += dt F / 2m, r += dt v (wrapped)        velocity Verlet, first half
 *   S3 q_n = sum_a Q_a W(r_a - r_n)               charge assignment, Sec. II.A
 *   S4 phi_p = 2 phi^k - phi^{k-1},
 *      sigma_p = (h/4pi) M phi_p + q              Eq. SHAKE
 *   S5 solve M y = sigma_p from the previous y    Eq. SHAKEy, App. B / Sec. III.A
 *   S6 phi^{k+1} = phi_p - (4pi/h) y              Eq. SHAKEPhiFinal
 *   S7 F_a = -k_e Q_a sum_n W(r_a - r_n) D phi_n  Eq. F_nostra
 *   S8 Tosi-Fumi pair forces within r_cut         Sec. III
 *   S9 v += dt F / 2m; KE, V_work, 1/2 phi.q      Eq. E_nostra, Eq. energy_discr
 *
 * Units: Angstrom, fs, amu, elementary charge e, eV. Energies and forces carry
 * k_e = e^2 / (4 pi eps0) = 14.3996454784 eV Angstrom (the paper writes
 * Gaussian units). Grid index n = i + j N + k N^2, x fastest (footnote to
 * Eq. linearproblem).
 *
 * Conventions
 *  - Every call returns a maze_status; nothing throws across the ABI.
 *  - A context owns all of its device memory (allocated in maze_create, freed
 *    in maze_destroy). Host pointers passed in are read only during the call.
 *  - Work is issued on the context's CUDA stream. Calls that return data to
 *    the host (maze_get, maze_get_stats, maze_solve, maze_step) synchronise
 *    that stream before returning.
 *  - After a failed maze_step see maze_step for what the context holds.
 *  - The library needs a CUDA device of compute capability 10.3 (sm_103a);
 *    maze_create fails with MAZE_ERR_CUDA when none is present.
 *  - maze_last_error returns a message for the last failing call on the
 *    calling thread (never NULL; empty when there is none).
 */
#ifndef MAZE_H
#define MAZE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MAZE_OK = 0,
  MAZE_ERR_INVALID = 1,        /* bad argument or configuration */
  MAZE_ERR_OOM = 2,            /* device allocation failed */
  MAZE_ERR_NOT_CONVERGED = 3,  /* constraint solve hit max_iter */
  MAZE_ERR_NONFINITE = 4,      /* NaN or Inf in a residual or energy */
  MAZE_ERR_TIMEOUT = 5,        /* a bounded device-side wait gave up */
  MAZE_ERR_CUDA = 6            /* CUDA runtime error (message in maze_last_error) */
} maze_status;

enum { MAZE_SOLVER_CG = 0, MAZE_SOLVER_MG = 1 };
enum { MAZE_FP64 = 0, MAZE_MIXED = 1, MAZE_FP64_FIXMG = 2 };
/* How a step obtains phi^{k+1} (Sec. III.A compares the three):
 *  MAZE_SCHEME_MAZE          SHAKE: phi_p = 2 phi^k - phi^{k-1}, solve M y = sigma_p
 *                            from the previous step's y (Eqs. SHAKE-SHAKEPhiFinal)
 *  MAZE_SCHEME_MG_STATIC     direct solve of M phi = -4 pi q / h (Eq. linearproblem)
 *                            starting from phi^k
 *  MAZE_SCHEME_MG_TIMEPROP   direct solve starting from 2 phi^k - phi^{k-1}
 * The direct schemes stop on max_n |(M phi + (4 pi/h) q)_n| < tol (Eq. res_poisson). */
enum { MAZE_SCHEME_MAZE = 0, MAZE_SCHEME_MG_STATIC = 1, MAZE_SCHEME_MG_TIMEPROP = 2 };
/* Electrostatic force estimator:
 *  MAZE_FORCE_CD      Eq. F_nostra: the assignment weights times the central-
 *                     difference field on the grid (conserves momentum)
 *  MAZE_FORCE_GRADW   Eq. F_Benoit: minus the gradient of the assignment weights
 *                     times phi (the exact gradient of 1/2 phi.q at fixed phi) */
enum { MAZE_FORCE_CD = 0, MAZE_FORCE_GRADW = 1 };

/* Physical constants used by the library (CODATA 2018). */
#define MAZE_KE_EV_ANGSTROM 14.399645478425668  /* e^2/(4 pi eps0) in eV*Angstrom */
#define MAZE_ACC_UNIT 9.648533215665327e-3      /* e/u * 1e-10: 1 eV/(amu*Angstrom) in Angstrom/fs^2 */
#define MAZE_KB_EV_PER_K 8.617333262145179e-5   /* Boltzmann constant k_B / e, eV/K */

/*
 * Run configuration; everything is host memory and is copied by maze_create.
 *
 * n_ions      number of ions N_p (>= 2)
 * grid_N      grid points per box edge N (even, 8 <= N <= 1024); with
 *             MAZE_SOLVER_MG, halving N while it is even and above 8 must
 *             end at an edge <= 8 (the exactly solved coarsest level), e.g.
 *             16, 32, 40, 48, 56, 64, 128, 256; otherwise MAZE_ERR_INVALID
 * box_L       cubic box edge L in Angstrom; grid spacing h = L / N
 * pos, vel    [n_ions * 3] x,y,z per ion (Angstrom, Angstrom/fs); pos may lie
 *             outside [0, L) and is wrapped
 * type        [n_ions] species index, 0 or 1
 * charge,mass per species (e, amu); the system must be neutral:
 *             |sum_a Q_a| <= 1e-9 * sum_a |Q_a|
 * tf_*        Tosi-Fumi pair energy A exp(B (s - r)) - C/r^6 - D/r^8 (Sec. III)
 *             for pair kinds 0 = (0,0), 1 = (0,1), 2 = (1,1); eV and Angstrom;
 *             A >= 0
 * r_cut       pair cutoff (Angstrom), 0 < r_cut <= L/2; the pair energy is
 *             shifted to zero at r_cut, forces are truncated
 * dt          time step (fs)
 * tol         constraint tolerance: the solve stops when
 *             max_n |(M y - sigma_p)_n| < tol (Eq. res_poisson_maze), in e
 * max_iter    iteration cap of one solve (CG iterations or V-cycles)
 * solver      MAZE_SOLVER_CG (Jacobi-PLCG, App. B) or MAZE_SOLVER_MG (V-cycle,
 *             Sec. III.A)
 * mg_pre/post red-black Gauss-Seidel sweeps before/after the coarse correction
 * order_P     assignment order: 2 (linear B-spline over the 8 nearest points)
 *             or 4 (cubic B-spline over 4^3 points), Sec. II.A
 * precision   MAZE_FP64; MAZE_MIXED (FP32 grid arithmetic, FP64 reductions);
 *             or MAZE_FP64_FIXMG (with MAZE_SOLVER_MG only): FP64 state and
 *             FP64 S4/S6, each V-cycle an FP64 defect correction whose
 *             correction is computed in exact 64-bit integers (units of a
 *             power-of-two scale set from the residual), the residual of the
 *             applied corrections tracked exactly; in exact arithmetic the
 *             same iterates as MAZE_FP64
 * scheme      MAZE_SCHEME_* above (0 = MaZe)
 * force_estimator  MAZE_FORCE_* above (0 = Eq. F_nostra)
 * langevin_gamma   friction gamma (1/fs) of the OVRVO Langevin integrator
 *             (Sec. III); 0 gives velocity Verlet (NVE)
 * langevin_T  bath temperature (K) of the O steps
 * seed        key of the counter-based generator (Philox-4x32-10) that draws
 *             the O steps' Gaussian numbers; the counter is (ion, step, stage)
 * cuda_stream cudaStream_t to issue work on; NULL makes the context create
 *             and own a non-blocking stream
 */
typedef struct {
  int32_t n_ions;
  int32_t grid_N;
  double box_L;
  const double* pos;
  const double* vel;
  const int32_t* type;
  double charge[2];
  double mass[2];
  double tf_A[3];
  double tf_B;
  double tf_s[3];
  double tf_C[3];
  double tf_D[3];
  double r_cut;
  double dt;
  double tol;
  int32_t max_iter;
  int32_t solver;
  int32_t mg_pre;
  int32_t mg_post;
  int32_t order_P;
  int32_t precision;
  int32_t scheme;
  int32_t force_estimator;
  double langevin_gamma;
  double langevin_T;
  uint64_t seed;
  void* cuda_stream;
} maze_config;

/* Per-step record, filled on the device at the end of every step. */
typedef struct {
  int64_t step;        /* completed MD steps since maze_create */
  int32_t iters;       /* iterations of the last constraint solve */
  int32_t status;      /* maze_status of the last step */
  double resid;        /* max_n |(M y - sigma_p)_n| at exit of the last solve */
  double ke;           /* kinetic energy, eV */
  double v_tf;         /* Tosi-Fumi energy, eV */
  double v_work;       /* work electrostatic energy V_work (Eq. E_nostra), eV */
  double v_disc;       /* discrete energy 1/2 k_e phi^T q (Eq. energy_discr), eV */
  double e_tot;        /* ke + v_tf + v_work */
  double momentum[3];  /* sum_a m_a v_a, amu Angstrom / fs */
  int64_t total_iters; /* solver iterations summed over all steps */
} maze_stats;

/* Quantities for maze_get / maze_set (layouts in doubles). */
enum {
  MAZE_POS = 0,       /* [n_ions*3], x,y,z per ion, in [0, L) */
  MAZE_VEL = 1,       /* [n_ions*3] */
  MAZE_FORCE = 2,     /* [n_ions*3] total force F_el + F_tf, eV/Angstrom (get only) */
  MAZE_FORCE_EL = 3,  /* [n_ions*3] electrostatic force (Eq. F_nostra) (get only) */
  MAZE_PHI = 4,       /* [N^3] phi^k, e/Angstrom (Gaussian units) */
  MAZE_PHI_PREV = 5,  /* [N^3] phi^{k-1} */
  MAZE_Y = 6,         /* [N^3] last SHAKE solution y (warm start of the next solve) */
  MAZE_CHARGE = 7,    /* [N^3] q on the grid from the last spread, e (get only) */
  MAZE_SIGMA = 8      /* [N^3] sigma_p of the last solve, e (get only) */
};

typedef struct maze_ctx maze_ctx;

/* Create a context: validate cfg, allocate device state, upload the ions and
 * do step 0: spread the charges, solve the constraint from phi = 0 (a zero-mean
 * phi^0) with an iteration cap of max(max_iter, 20000), set phi^{-1} = phi^0
 * and y = 0, and compute F^0 and the energies.
 * On success *out owns the context; on failure *out is NULL. */
maze_status maze_create(const maze_config* cfg, maze_ctx** out);

/* S3 alone: spread the charges of the current positions onto the grid. */
maze_status maze_spread(maze_ctx* ctx);

/* S4-S6 alone, on the charges of the last maze_spread: build sigma_p, solve
 * M y = sigma_p from the stored y, correct phi and rotate phi^{k-1} <- phi^k,
 * phi^k <- phi^{k+1}. Returns the iteration count and the final residual
 * max_n |(M y - sigma_p)_n|. Synchronises. MAZE_ERR_NOT_CONVERGED when
 * max_iter was reached (the state is still updated with the last iterate). */
maze_status maze_solve(maze_ctx* ctx, int32_t* iters, double* resid_inf);

/* S7 + S8 alone: forces F_el (Eq. F_nostra) and Tosi-Fumi forces on the
 * current positions from the current phi^k, plus V_TF and 1/2 phi.q. */
maze_status maze_gather(maze_ctx* ctx);

/* S1..S9 repeated nsteps times (nsteps >= 0). Synchronises and reports the
 * first failing step's status. A step whose solve reaches max_iter still
 * completes with the last iterate (MAZE_ERR_NOT_CONVERGED) and no later step
 * of the call runs; after MAZE_ERR_TIMEOUT or MAZE_ERR_NONFINITE the context
 * state is undefined and it should be destroyed. */
maze_status maze_step(maze_ctx* ctx, int32_t nsteps);

/* As maze_step, but only enqueues the steps on the context's stream and
 * returns without synchronising; device-side failures surface in the next
 * maze_get_stats (field status) or maze_step. */
maze_status maze_step_async(maze_ctx* ctx, int32_t nsteps);

/* Copy a quantity (MAZE_POS ...) to host memory of the documented size. */
maze_status maze_get(maze_ctx* ctx, int32_t what, double* host_out);

/* Overwrite a quantity (MAZE_POS, MAZE_VEL, MAZE_PHI, MAZE_PHI_PREV, MAZE_Y)
 * from host memory. Setting MAZE_POS wraps the positions into [0, L); the
 * forces are not recomputed (call maze_gather). host_in is read during the
 * call; MAZE_POS and MAZE_VEL of a standalone context are then uploaded
 * asynchronously on the context's stream from a pinned copy the context
 * owns (work issued later on the stream sees the new values). */
maze_status maze_set(maze_ctx* ctx, int32_t what, const double* host_in);

/* Copy the per-step record to *out. Synchronises. */
maze_status maze_get_stats(maze_ctx* ctx, maze_stats* out);

/* One exchange of a host-driven simulation in a single call: optional new
 * positions and velocities (host memory, [n][3], as maze_set: positions
 * wrapped into [0, L), forces not recomputed), then nsteps steps (S1..S9 as
 * maze_step), then optional copies of the positions and velocities
 * ([n][3]) and of the per-step record to host memory. Synchronises once.
 * Any of pos_in, vel_in, pos_out, vel_out, stats_out may be NULL. A
 * non-finite input returns MAZE_ERR_INVALID before anything is uploaded or
 * run. The return value is maze_step's; when the steps ran (also with
 * MAZE_ERR_NOT_CONVERGED, MAZE_ERR_NONFINITE or MAZE_ERR_TIMEOUT) the
 * outputs hold the state they left; after a CUDA or argument error they
 * are not written. The results equal maze_set, maze_step, maze_get and
 * maze_get_stats called in that order. */
maze_status maze_step_io(maze_ctx* ctx, const double* pos_in, const double* vel_in, int32_t nsteps,
                         double* pos_out, double* vel_out, maze_stats* stats_out);

/* Checkpoint: the full dynamical state (step, V_work, positions, velocities,
 * forces, phi^k, phi^{k-1}, y) as an opaque blob. With blob == NULL,
 * maze_get_state stores the needed size in *n. Restoring a blob from a
 * context of the same configuration resumes bit-identically. */
maze_status maze_get_state(maze_ctx* ctx, void* blob, size_t* n);
maze_status maze_set_state(maze_ctx* ctx, const void* blob, size_t n);

/* Free everything the context owns. NULL-safe. */
void maze_destroy(maze_ctx* ctx);

/* Message of the last failing call on this thread ("" if none). */
const char* maze_last_error(void);

/* Device timing of the phases of the most recent maze_step / maze_step_async
 * step, in milliseconds, measured with CUDA events on the context's stream:
 * out[0] half kick + drift + spread, out[1] cell list, out[2] constraint
 * solve (S4-S6), out[3] forces + second half kick. (When the pair forces
 * run on a second stream beside the solve - MAZE_FP64_FIXMG boxes of 128^3
 * and more with at least two cells per SM, unless the environment sets
 * MAZE_OVERLAP=0 - out[0] is the half kick + drift, out[1] the cell list and
 * the spread, out[3] the wait for the pairs, the gather and the second half
 * kick.) maze_set_timing(ctx, 1)
 * makes every step record these events (a small cost); maze_get_timing
 * synchronises and fails with MAZE_ERR_INVALID while timing is off. */
maze_status maze_set_timing(maze_ctx* ctx, int32_t on);
maze_status maze_get_timing(maze_ctx* ctx, double* out4);

/* Allocation-free constraint solve. The paper has no counterpart: this entry
 * exists for callers that cannot call cudaMalloc - a host framework that owns
 * all device memory through its own pool, a latency-critical loop that must
 * not take cudaMalloc's implicit device synchronisation, or a process held to
 * a fixed device-memory budget. It solves M y = sigma_p (Eq. SHAKEy) with the
 * same warm-started CG and stopping rule as maze_solve, then removes the mean
 * of y.
 *   grid_N     grid edge N, even, 8 <= N <= 64
 *   sigma_p    [N^3] device pointer, read only, flat index n = i + jN + kN^2;
 *              its entries must sum to zero (the periodic M is singular and
 *              only a zero-mean right-hand side has a solution: a charge-
 *              neutral box gives one), else the call runs to max_iter and
 *              returns MAZE_ERR_NOT_CONVERGED
 *   y          [N^3] device pointer, not overlapping sigma_p (sigma_p == y is
 *              rejected with MAZE_ERR_INVALID); in: warm start, out: zero-mean
 *              solution
 *   tol        stop when max_n |(M y - sigma_p)_n| < tol
 *   max_iter   CG iteration cap
 *   cuda_stream stream to run on (NULL = legacy default stream); the call
 *              synchronises it before returning, so it must never be made
 *              while that stream is being captured into a CUDA graph
 *   iters, resid_inf  optional outputs (host pointers)
 * It allocates nothing: its work vectors live in one file-scope device array
 * of about 6.4 MB (3 x 64^3 doubles plus a small status block), which every
 * GPU that loads the library holds until the process exits. Larger grids are
 * rejected with MAZE_ERR_INVALID. The first call on a device, with that device
 * current, resolves the array's device address and the launch size. A NaN or
 * infinity in sigma_p or in the warm start ends the call with
 * MAZE_ERR_NONFINITE. Every call shares the one array and
 * keeps the last call's contents in it, so calls that overlap on the GPU (on
 * different streams or threads) race and must be serialised by the caller. */
maze_status maze_solve_shake_noalloc(int32_t grid_N, const double* sigma_p, double* y, double tol,
                                     int32_t max_iter, void* cuda_stream, int32_t* iters,
                                     double* resid_inf);

/* ---------------------------------------------------------------------------
 * Batched simulations (many independent MaZe boxes on one GPU).
 *
 * The paper advances one box at a time; these calls are this library's own
 * engine for running many of them together. A batch owns one block of device
 * memory (the arena) from which each admitted simulation takes its buffers,
 * and a set of slots. Every simulation in a batch advances one MaZe step per
 * launch of ONE persistent kernel: each thread-block cluster takes whole
 * boxes, largest first, and runs all phases of that box's step (S1-S9 above)
 * with cluster barriers, so boxes of different sizes share the GPU without
 * waiting for each other. The step is replayed from a captured CUDA graph.
 *
 * Simulations in a batch run precision MAZE_MIXED with MAZE_SOLVER_MG and
 * grid_N <= 64. A simulation advanced in a batch computes bit for bit the
 * positions, velocities, forces and potential it computes alone in a context
 * of the same configuration (energies agree to rounding).
 *
 * Simulation ids are slot indices in [0, max_sims); a removed simulation's id
 * is reused by a later maze_batch_add. The cuda_stream field of the
 * maze_config passed to maze_batch_add is ignored: all work of a batch runs
 * on the batch's stream.
 */
typedef struct maze_batch maze_batch;

typedef struct {
  size_t arena_bytes;    /* device memory reserved for all simulations' buffers (>= 1 MiB) */
  int32_t max_sims;      /* number of slots, in [1, 65536] */
  int32_t cluster_ctas;  /* CTAs per cluster of the step kernel (the tile of one box):
                            1, 2, 4, 8 or 16; 0 selects 4. maze_batch_tune changes it. */
  void* cuda_stream;     /* cudaStream_t for all of the batch's work; NULL = the batch
                            creates its own non-blocking stream */
} maze_batch_config;

/* Create an empty batch: allocates the arena and the per-slot tables.
 * MAZE_ERR_INVALID for a bad config, MAZE_ERR_OOM when the arena cannot be
 * allocated, MAZE_ERR_CUDA without an sm_103a device. *out is NULL on error. */
maze_status maze_batch_create(const maze_batch_config* cfg, maze_batch** out);

/* Arena bytes one simulation of this configuration takes (exact; the
 * admission test of a serving loop). Needs a CUDA device; validates cfg. */
maze_status maze_batch_box_bytes(const maze_config* cfg, size_t* bytes);

/* Largest free block and total free bytes of the arena (either may be NULL). */
maze_status maze_batch_free_bytes(maze_batch* b, size_t* largest_block, size_t* total_free);

/* Admit one simulation: copy its state, take its buffers from the arena and
 * queue its step 0 (as maze_create runs it) on the batch's admission stream,
 * a stream of its own: steps already queued on the batch's stream go on
 * meanwhile, and the call returns without waiting for step 0. On success
 * *id is its slot; it then advances with every maze_batch_step (which first
 * waits for pending admissions) or, once its step 0 has finished, with
 * maze_batch_step_ready_async. A step 0 that fails shows in the
 * simulation's statistics and stops only that simulation.
 * MAZE_ERR_OOM when no slot is free or the arena has no room (nothing is
 * changed; retry after a maze_batch_remove), MAZE_ERR_INVALID for a config
 * maze_create would reject or that the batch cannot run (see above). */
maze_status maze_batch_add(maze_batch* b, const maze_config* cfg, int32_t* id);

/* Retire simulation id and return its buffers to the arena. */
maze_status maze_batch_remove(maze_batch* b, int32_t id);

/* Number of simulations, CTAs per cluster and resident clusters of the step
 * kernel (any pointer may be NULL). */
maze_status maze_batch_info(maze_batch* b, int32_t* count, int32_t* cluster_ctas, int32_t* clusters);

/* Advance every simulation of the batch by nsteps MaZe steps (one kernel
 * launch per step) and synchronise. A simulation whose step fails stops
 * advancing for the rest of the call (as maze_step does for one context)
 * while the others continue; the call then returns the first failing
 * simulation's status and names it in maze_last_error, and
 * maze_batch_get_stats gives each simulation's own status. */
maze_status maze_batch_step(maze_batch* b, int32_t nsteps);

/* As maze_batch_step, without waiting for the GPU or checking statuses. */
maze_status maze_batch_step_async(maze_batch* b, int32_t nsteps);

/* Continuous batching. maze_batch_refresh moves the simulations whose
 * admission (step 0) has finished on the GPU into the work order, without
 * waiting for the others, and lists their ids in joined[0 .. *n_joined)
 * (joined: host array of cap >= max_sims entries). It synchronises the
 * batch's stream. maze_batch_step_ready_async then queues nsteps steps of the
 * simulations in the work order, without waiting for the GPU and without
 * admitting anything new. Pair it with maze_batch_sync. */
maze_status maze_batch_refresh(maze_batch* b, int32_t* joined, int32_t cap, int32_t* n_joined);
maze_status maze_batch_step_ready_async(maze_batch* b, int32_t nsteps);

/* Wait for the steps queued so far and return the first failing status among
 * the simulations they advanced (named in maze_last_error), else MAZE_OK. */
maze_status maze_batch_sync(maze_batch* b);

/* maze_get / maze_set / maze_get_stats for simulation id (synchronise the
 * batch's stream first). */
maze_status maze_batch_get(maze_batch* b, int32_t id, int32_t what, double* host_out);
maze_status maze_batch_set(maze_batch* b, int32_t id, int32_t what, const double* host_in);
maze_status maze_batch_get_stats(maze_batch* b, int32_t id, maze_stats* out);

/* Statistics of every slot in one call: out[id] for id in [0, max_sims)
 * (n >= max_sims); a free slot reads step = -1. */
maze_status maze_batch_get_all_stats(maze_batch* b, maze_stats* out, int32_t n);

/* Autotuner: time steps_per_trial steps with each cluster size the device
 * can co-schedule (1, 2, 4, 8, 16 CTAs per box), keep the fastest. The
 * simulations' state is saved before and restored after every trial, so
 * tuning does not advance them; results do not depend on the cluster size.
 * Needs a temporary device buffer the size of the arena's used part. */
maze_status maze_batch_tune(maze_batch* b, int32_t steps_per_trial, int32_t* chosen_ctas, double* ms_per_step);

/* One row of the per-size-class autotuning table. */
typedef struct {
  int32_t grid_N;               /* the class: boxes of this grid edge */
  int32_t boxes;                /* its boxes in the batch */
  int32_t cluster_ctas;         /* CTAs per box (the tile of the grid one box gets) */
  int32_t mg_pre, mg_post;      /* V-cycle schedule: Gauss-Seidel sweeps before / after */
  int32_t tail_n;               /* levels of at most tail_n^3 points in one CTA (0: the default) */
  double ms_before;             /* batch step time (ms) before this class was tuned */
  double ms_after;              /* ... and after */
} maze_tune_entry;

/* Autotuner per size class (the project's own; the paper has none). Starting
 * from the batch-wide cluster size, it visits the grid sizes of the batch in
 * order of their work and for each picks in turn the CTAs per box (1-16),
 * the size of the V-cycle's one-CTA coarse tail (8^3 or 16^3 points) and the
 * red-black Gauss-Seidel schedule (nu1, nu2 in {(2,2), (1,2), (2,1), (1,1),
 * (3,3)}), each trial timing whole batch steps as they run (one launch per
 * cluster size, the launches side by side); a change must shorten the step
 * by 3 %, so the result is never slower than the start as measured. Cluster size and tail change no result; a schedule other than the
 * configured one changes results within the solve tolerance (every box still
 * meets tol; the mixed-precision path is multigrid only, so there is no CG /
 * multigrid choice to make). State is saved before and restored after every
 * trial. table: host array of cap >= (grid sizes in the batch) entries;
 * *n_entries rows are written. maze_batch_tune undoes these choices. */
maze_status maze_batch_autotune(maze_batch* b, int32_t steps_per_trial, maze_tune_entry* table, int32_t cap,
                                int32_t* n_entries);

/* Free every simulation and the batch (NULL-safe). */
void maze_batch_destroy(maze_batch* b);

/* Library version string, e.g. "maze-gb300 0.1". */
const char* maze_version(void);

/* Diagnostic: drive one of the library's bounded device-side waits to its
 * limit and report what the kernel recorded. The paper has no counterpart;
 * the solves and the batch step synchronise their blocks with three waits
 * (the cooperative grid barrier, the grid reduction of doubles and the one of
 * 64-bit integers), each of which gives up after a fixed number of polls
 * (about a second), records MAZE_ERR_TIMEOUT and returns, so that a block
 * that never arrives cannot hang the GPU. This call launches a small
 * cooperative kernel whose wait can never complete - which = 0: a grid
 * barrier waiting for one more round of arrivals than the grid makes; 1: a
 * grid reduction of doubles in which one block publishes under another
 * round number; 2: the same for the 64-bit integer reduction - and returns
 * the status the kernel recorded in *status_out (MAZE_ERR_TIMEOUT when the
 * wait gave up as designed). The call allocates and frees its own small
 * device buffers and synchronises cuda_stream (NULL = legacy default
 * stream). Returns MAZE_ERR_INVALID for another `which`, MAZE_ERR_CUDA when
 * the launch or a copy fails, else MAZE_OK. */
maze_status maze_wait_probe(int32_t which, void* cuda_stream, int32_t* status_out);

/* Diagnostic: the FP32/FP64 conversions that the FP64 kernels perform on the
 * integer pipe (GB300's conversion instructions occupy the FP64 pipe), beside
 * the conversion instructions, for n host doubles in[]: f_own/f_hw = in
 * rounded to FP32 (nearest even); d_own/d_hw = f_hw widened back to FP64;
 * floor_own/floor_hw = floor(in) as a 64-bit integer (0 where |in| >= 4e18);
 * fix_own/fix_hw = the integer trunc(in 2^20) times 2^-20 as a double (0
 * where |in| >= 4e18). Every array has n elements, host memory, owned by the
 * caller. The call allocates, copies and synchronises on the legacy default
 * stream. Returns MAZE_ERR_INVALID for n < 0 or a NULL array, MAZE_ERR_CUDA
 * when a CUDA call fails, else MAZE_OK. */
maze_status maze_convert_probe(const double* in, int32_t n, float* f_own, float* f_hw, double* d_own, double* d_hw,
                               int64_t* floor_own, int64_t* floor_hw, double* fix_own, double* fix_hw);

/* Diagnostic: the exponential the FP64 Tosi-Fumi pair forces evaluate (a
 * table-driven method, Tang 1989: a 64-entry table of 2^(j/64), a degree-5
 * polynomial, the power of two set in the exponent field; exp() for
 * |x| >= 512 and non-finite x) beside the CUDA math library's exp(), for n
 * host doubles in[]: own[i], ref[i]. Host arrays of n elements owned by the
 * caller; the call allocates, copies and synchronises on the legacy default
 * stream. Returns MAZE_ERR_INVALID for n < 0 or a NULL array, MAZE_ERR_CUDA
 * when a CUDA call fails, else MAZE_OK. */
maze_status maze_exp_probe(const double* in, int32_t n, double* own, double* ref);

/* Diagnostic: the double-float arithmetic that the FP64 boxes' once-per-pair
 * kernel runs on the FP32 pipe (Sec. III's Tosi-Fumi pair, evaluated as an
 * unevaluated sum of two floats to ~1e-14 relative), for n host doubles in[],
 * each split into (hi, lo) floats first (hi = in rounded to FP32, lo = the
 * rest rounded to FP32). what = 0: out0[i] = exp(in[i]) by the double-float
 * table method (out1 and cfg unused, may be NULL). what = 1: in[i] is a
 * squared distance r^2 (A^2) of a pair of kind kind[i] (0 Na-Na, 1 Na-Cl,
 * 2 Cl-Cl) with the Tosi-Fumi table and r_cut of *cfg; out0[i] = -(dV/dr)/r
 * (eV/A^2), out1[i] = V(r) - V(r_cut) (eV), as hi + lo. what = 2: the same
 * pair in FP64 arithmetic (the form of the other force kernels). Only the
 * Tosi-Fumi fields and r_cut of cfg are read. Host arrays of n elements owned
 * by the caller; the call allocates, copies and synchronises on the legacy
 * default stream. Returns MAZE_ERR_INVALID for another what, n < 0, a NULL
 * array that the mode reads or writes, or a kind outside 0..2;
 * MAZE_ERR_CUDA when a CUDA call fails; else MAZE_OK. */
maze_status maze_df_probe(const maze_config* cfg, int32_t what, const double* in, const int32_t* kind, int32_t n,
                          double* out0, double* out1);

#ifdef __cplusplus
}
#endif

#endif /* MAZE_H */
