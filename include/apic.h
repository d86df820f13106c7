/*
 * apic.h -- C ABI of libapic.so: the GB300 (sm_103a) particle-in-cell step of
 * the APIC method (R.D. Smirnov, S.I. Krasheninnikov, "Aspherical PIC code
 * (APIC) for modeling non-spherical dust in plasmas using shape-conforming
 * coordinates", arXiv:2307.11107).
 *
 * One step advances electrons and ions around a conducting grain whose surface
 * is x1 = -1 in the shape-conforming coordinates of Eq. 2,
 *     x1 = -(1/r)(1 + alpha cos(theta)/r),   x2 = cos(theta),
 * in this order (Sec. 1 and Sec. 2 of the paper):
 *   charge weighing of every particle onto the (x1, x2) node grid, divided by
 *   the node volume of Eq. 5;  the Poisson problem of Eqs. 6-7 with fixed
 *   potentials on the grain (x1 = -1) and on the outer surface (x1 = x1_outer);
 *   dphi/dx1, dphi/dx2 at the nodes, interpolated to each particle and turned
 *   into E_R, E_Z by Eq. 10;  the equations of motion of Eq. 9 (leapfrog /
 *   Boris, axial B);  absorption on the grain with per-surface-bin tallies of
 *   charge, momentum, angular momentum and energy;  escape through the outer
 *   surface;  Maxwellian injection through the outer surface weighted by the
 *   area element of Eq. 4.
 *
 * Units (all arguments and results): lengths in R0, time in 1/omega_pe,
 * velocity in lambda_De*omega_pe, potential in Te/e, density in n0, charge of
 * a species in e, mass in m_e, B in m_e omega_pe / e, eps0 = 1.  The unperturbed
 * density n0 is 1 for every species.
 *
 * Grid: n1 x n2 CELLS, nodes (i, j), i = 0..n1 at x1 = -1 + i*(x1_outer+1)/n1,
 * j = 0..n2 at x2 = -1 + 2j/n2; node arrays are row-major [n1+1][n2+1].
 *
 * Ownership and threading: the library owns every device buffer, obtained
 * through the caller's allocator (or cudaMallocAsync when none is given) on the
 * caller's stream; all device work is ordered on that stream.  Host buffers
 * passed in are owned by the caller and are read or written before the call
 * returns.  A simulation object is not thread-safe; distinct objects are
 * independent.
 *
 * Errors: every call returns APIC_OK (0) or a negative APIC_ERR_* code and never
 * throws.  Errors are sticky: after one, every later call on the same object
 * returns it again; apic_last_error() gives a message; only apic_destroy()
 * clears the object.
 */
#ifndef APIC_H
#define APIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define APIC_OK 0
#define APIC_ERR_INVALID_ARG (-1)  /* bad sizes, NULL pointers, bad mode */
#define APIC_ERR_GEOMETRY (-2)     /* |alpha| >= 0.245 or x1_outer not in (-1, 0) */
#define APIC_ERR_CAPACITY (-3)     /* a species outgrew its particle capacity */
#define APIC_ERR_NOT_CONVERGED (-4)/* Poisson iteration limit reached above tolerance */
#define APIC_ERR_NONFINITE (-5)    /* NaN/Inf in the fields or residual, or a tally value beyond its fixed-point
                                      range (|v| >= 11585 v_th for the energy) */
#define APIC_ERR_TIMEOUT (-6)      /* a bounded device wait gave up: a grid barrier of a cooperative solver (2 s of
                                      global time) or a bulk-copy wait; every CTA returns and the context stays
                                      usable, the object keeps the error */
#define APIC_ERR_CUDA (-7)         /* CUDA runtime or allocation failure */

/* precision of the particle arrays and of the Poisson preconditioner */
#define APIC_FP64 0          /* FP64 particles, FP64 multigrid (parity path) */
#define APIC_FP32_REFINED 1  /* FP32 particles; FP32 block cyclic reduction (or FP32 multigrid) inside an
                                FP64 residual loop */

/* apic_inject modes */
#define APIC_LOAD_VOLUME 0   /* n particles uniform in physical volume, Maxwellian at T */
#define APIC_FLUX_SURFACE 1  /* n particles entering through the outer surface (Eq. 4 weighting) */
#define APIC_EXPLICIT 2      /* n caller-given states (x1, x2, vR, vZ, vTheta), FP64 */

/* config flags */
#define APIC_NO_INJECT 1     /* no per-step surface injection */
#define APIC_NO_FIELD 2      /* phi = 0: no Poisson solve, E = 0 (test and baseline use) */
#define APIC_CHORD_ABSORB 4  /* also absorb a particle whose straight chord of the step passes through
                                the grain while its end point lies outside (grazing orbits; the chord is
                                tested at 7 interior points once it comes closer to the origin than the
                                grain's largest radius; impact point by bisection up to the first point
                                inside).  Not with apic_sensitivity (INVALID_ARG). */
#define APIC_FLOATING 8      /* isolated grain: phi_grain is the potential of the first step only; from then
                                on the grain keeps the charge it held then plus every charge it absorbs, and
                                its potential follows (history column 10).  Each step's field is the solve
                                at the last potential plus the multiple of the grain's vacuum field (phi = 1
                                on the grain, 0 outside, computed at creation) that restores that charge.
                                Not with APIC_NO_FIELD, nor with apic_sensitivity (INVALID_ARG);
                                apic_solve_poisson keeps using phi_grain. */
#define APIC_FE_OPERATOR 32  /* the conservative form of Eqs. 6-7 instead of Eq. 7's finite differences: the
                                bilinear finite-element weak form on the logical grid, sum_b K_ab phi_b =
                                rho_a V_a with K_ab = int grad N_a . grad N_b dOmega (3 x 3 Gauss points per cell),
                                symmetric after weighting by V, exact discrete Gauss law; same solvers */
#define APIC_BOLTZMANN 16    /* electrons are not simulated: their density is n0 exp(phi) (Te = 1, potential
                                zero at the outer surface) in Eq. 6, whose nonlinear problem is solved by
                                newton_iters Newton iterations, each a BiCGSTAB solve preconditioned by the
                                multigrid of the linear operator (the species given are the ions).  Forces the
                                multigrid solver (one cooperative launch per Newton iteration for a single
                                instance, per-phase kernels for a batch).  apic_solve_poisson solves the same
                                nonlinear problem for the given ion density.  The grain collects the
                                electrons' one-sided Maxwellian flux exp(phi_grain)/sqrt(2 pi) per unit area
                                and time (history's current).  Not with APIC_NO_FIELD,
                                APIC_FLOATING or apic_sensitivity (INVALID_ARG). */

#define APIC_NT 7  /* tally components per (species, bin): hits, charge, p_R, p_Z, L_z, E_kin, E_kin + E_bind.
                      With APIC_BOLTZMANN the bins hold the simulated ions only: the electrons' flux
                      enters the history's current alone (not its heat flux). */
#define APIC_NH 11 /* history fields per step: t, current, drag F_Z, electric F_Z, torque T_z,
                      heat flux, grain charge Q, resident species 0, resident species 1, absorbed events,
                      grain potential of the step's field */

typedef struct {
  double q;          /* charge in e (electron -1) */
  double m;          /* mass in m_e */
  double T;          /* temperature in Te */
  int64_t n_init;    /* macro-particles that represent density n0 in the whole domain: w = V / n_init */
  int64_t capacity;  /* particle slots reserved for this species */
} apic_species_t;

typedef struct {
  double alpha;          /* shape parameter of Eqs. 1-5, |alpha| < 0.245 */
  double x1_outer;       /* outer boundary x1 = const, in (-1, 0) */
  double phi_grain;      /* potential on x1 = -1 */
  double phi_outer;      /* potential on x1 = x1_outer */
  double B;              /* axial field of Eq. 9 */
  double dt;             /* time step */
  double e_bind_ion;     /* energy deposited per absorbed particle of positive charge, besides E_kin */
  int32_t n1, n2;        /* cells in x1 and x2: n1 >= 4, n2 >= 8 */
  int32_t n_species;     /* 1 or 2 */
  apic_species_t sp[2];
  uint64_t seed;         /* Philox4x32-10 key */
  int32_t instance;      /* Philox counter tag; distinct instances draw distinct streams */
  int32_t precision;     /* APIC_FP64 or APIC_FP32_REFINED */
  int32_t flags;         /* APIC_NO_INJECT | APIC_NO_FIELD | APIC_CHORD_ABSORB | APIC_FLOATING | APIC_BOLTZMANN |
                            APIC_FE_OPERATOR */
  double poisson_tol;    /* relative residual target ||b - A phi|| / ||b|| (0: 1e-10) */
  int32_t poisson_max_iter; /* BiCGSTAB iterations per step (0: 20) */
  int32_t sort_interval; /* sort particles by cell every this many steps (0: never) */
  int32_t history_cap;   /* rows of the per-step history ring (0: 4096) */
  int32_t poisson_guess; /* start of each step's solve: 0 previous phi, 1 linear extrapolation 2 phi^n - phi^n-1 */
  int32_t newton_iters;  /* APIC_BOLTZMANN: Newton iterations per solve (0: 8); the linear solve of each but
                            the last stops once its residual has fallen 1000-fold (inexact Newton); once the
                            nonlinear residual is below poisson_tol the remaining iterations do no solver work */
  int32_t reserved[3];
} apic_config_t;

typedef void* (*apic_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*apic_free_fn)(void* ptr, void* stream, void* ctx);
typedef struct {
  apic_alloc_fn alloc;   /* returns device memory (>= 256-byte aligned) or NULL */
  apic_free_fn free;
  void* ctx;
} apic_allocator_t;

typedef struct apic_sim apic_sim;  /* opaque, owned by the library */

typedef struct {
  /* caller-owned outputs; any pointer may be NULL */
  double* bins;          /* [n_species][n2][APIC_NT] cumulative tallies of absorbed particles */
  double* history;       /* [history_rows][APIC_NH], oldest first */
  int64_t history_rows;  /* in: capacity of history; out: rows written */
  int64_t counts[2][6];  /* out: loaded, injected, absorbed, escaped, resident, dropped */
  int64_t step;          /* out: steps taken */
  double grain_Q;        /* out: grain charge (surface integral of sigma), last field solve */
  double grain_FZ;       /* out: electric force on the grain along Z, last field solve */
  double poisson_res;    /* out: relative residual of the last solve */
  int32_t poisson_iters; /* out: BiCGSTAB iterations of the last solve */
  int32_t pad;
} apic_tallies_t;

/* Create one simulation (batch of one instance).  Sec. 2: grid, node volumes
 * (Eq. 5), sampling tables (Eqs. 4-5) and the finite-difference operator of
 * Eq. 7 are set up here.  stream: a cudaStream_t (NULL = legacy default).
 * allocator: NULL for cudaMallocAsync.  *out receives the object, or NULL on
 * error.  Errors: INVALID_ARG, GEOMETRY, CUDA. */
int apic_create(const apic_config_t* cfg, void* stream, const apic_allocator_t* allocator,
                apic_sim** out);

/* Create n instances that advance together in every kernel launch (each with
 * its own alpha, potentials, B, grid and particle counts).  Instance k is
 * addressed as `instance = k` below.  With FP32 particles the Poisson
 * problems of all instances are solved by one block-cyclic-reduction launch
 * whose blocks are formed here on the host (a few seconds for large batches;
 * up to 24 GB of device memory, and at most 60 % of the free memory, else
 * multigrid is used); an instance computes the same values alone or in the
 * batch.  At most 64 instances share the reduction solve. */
int apic_create_batch(const apic_config_t* cfgs, int32_t n, void* stream,
                      const apic_allocator_t* allocator, apic_sim** out);

/* Release every buffer; safe on NULL. */
int apic_destroy(apic_sim* sim);

/* Add n particles of `species` to `instance` (Sec. 1: Maxwellian plasma of
 * density n0 and temperature T).  explicit_state: host FP64 [n][5] rows
 * (x1, x2, vR, vZ, vTheta) for APIC_EXPLICIT, else NULL.  Draws are
 * counter-based (Philox4x32-10): the same sequence of calls gives the same
 * particles.  Errors: INVALID_ARG, CAPACITY, CUDA. */
int apic_inject(apic_sim* sim, int32_t instance, int32_t species, int64_t n, int32_t mode,
                const double* explicit_state);

/* Advance every instance by n_steps full steps of the method (Sec. 1 and
 * Sec. 2): charge weighing with the node volumes of Eq. 5 -> the Poisson
 * problem of Eqs. 6-7 -> node gradients and the gather of Eq. 10 -> the
 * leapfrog push of Eq. 9 -> absorption on the grain x1 = -1 with its tallies
 * -> escape through x1 = x1_outer -> Maxwellian injection through the outer
 * surface weighted by Eq. 4.  Work is queued on the stream and the call waits
 * for it once at the end to read the status word.  Errors: CAPACITY,
 * NOT_CONVERGED, NONFINITE, TIMEOUT, CUDA. */
int apic_step(apic_sim* sim, int32_t n_steps);

/* Copy tallies, counts and the history of `instance` into caller buffers
 * (Sec. 1: the charge, momentum, angular momentum and energy that absorbed
 * particles transfer to the grain at the point of impact, binned by the x2
 * of the impact; Sec. 2 after Eq. 10: the grain charge and electric force).
 * The bins are sums of fixed-point values (scaled by the species' thermal
 * speed, 36 fraction bits, 128-bit accumulators): they do not depend on the
 * order of the absorption events, and each event's value is rounded by at
 * most 7.3e-12 of m w v_th (momenta), m w v_th R0 (L_z) or m w v_th^2
 * (energy).  Waits for the stream.  Errors: INVALID_ARG, those of earlier
 * calls (sticky). */
int apic_tallies(apic_sim* sim, int32_t instance, apic_tallies_t* out);

/* ---- Checkpoint / resume (no counterpart in the paper) ----------------------
 * A checkpoint holds what the next apic_step calls depend on, for every
 * instance of the object: each population's live particle slots (the five
 * state arrays of Sec. 2's macro-particles) and free-slot stack, its counts,
 * Philox draws consumed and injection carry, the solver and step scalars
 * (step index, grain charge and force), phi (the next solve's start), the
 * deposit accumulators of the last step, the node gradients, the fixed-point
 * tallies and the history ring, and the step counter and sort interval of the
 * object.  Because every random draw is a counter-based Philox draw, steps
 * after apic_checkpoint_load give the tallies, fields and particle set of the
 * uninterrupted run bit for bit (particles may sit in other slots: the sort's
 * placement within a row depends on scheduling).  A sensitivity window in
 * progress is not part of a checkpoint.  The buffer is plain host memory in
 * the layout of this library version (a header, then the arrays); its size
 * depends on the particle counts at the time of the call.
 *
 * apic_checkpoint_size: *bytes = the size a checkpoint of the current state
 *   takes.  Errors: INVALID_ARG (NULL), a sticky error.
 * apic_checkpoint_save: waits for the work in flight and copies the state into
 *   buf (host, bytes long).  Errors: INVALID_ARG (NULL, bytes too small), a
 *   sticky error, CUDA.
 * apic_checkpoint_load: replaces this object's state with the checkpoint in
 *   buf, made by an object created with the same configurations (the same
 *   instances, grids, species capacities and history sizes).  Errors:
 *   INVALID_ARG (NULL, a buffer that is not a checkpoint of this layout, or
 *   of an object with other sizes, counts above a capacity), a sticky error,
 *   CUDA.  A refused checkpoint leaves the object unchanged. */
int apic_checkpoint_size(apic_sim* sim, int64_t* bytes);
int apic_checkpoint_save(apic_sim* sim, void* buf, int64_t bytes);
int apic_checkpoint_load(apic_sim* sim, const void* buf, int64_t bytes);

/* Solve Eqs. 6-7 for `instance` with the GPU solver.  rho: host [n1+1][n2+1]
 * charge density, or NULL for the density of the current particles.
 * phi_out: host [n1+1][n2+1].  The simulation's own potential is unchanged. */
int apic_solve_poisson(apic_sim* sim, int32_t instance, const double* rho, double* phi_out);

/* Diagnostics: copy the live particles of (instance, species) as FP64 rows
 * (x1, x2, vR, vZ, vTheta) into out [capacity][5]; slots of absorbed or escaped
 * particles are skipped.  *n_out receives the row count (<= capacity). */
int apic_get_particles(apic_sim* sim, int32_t instance, int32_t species, double* out,
                       int64_t capacity, int64_t* n_out);

/* Diagnostics: node field `which` of `instance` into out [n1+1][n2+1]:
 * 0 rho (last deposit), 1 phi, 2 dphi/dx1, 3 dphi/dx2, 4 node volume. */
int apic_get_field(apic_sim* sim, int32_t instance, int32_t which, double* out);

/* Message of the last error (static storage of the object; never NULL). */
const char* apic_last_error(const apic_sim* sim);

/* Number of instances of the batch. */
int32_t apic_num_instances(const apic_sim* sim);

#define APIC_NPHASE 6 /* deposit->rho, Poisson, node gradients + surface, push, inject, bookkeeping */

typedef struct {
  int64_t steps;                /* steps taken by the batch */
  int64_t poisson_loop_iters;   /* Krylov-loop iterations executed, summed over steps */
  int32_t kernels_per_step;     /* kernel launches per step outside the Krylov loop */
  int32_t kernels_per_iter;     /* kernel launches per Krylov-loop iteration (incl. its test) */
  int64_t timed_steps;          /* steps run by apic_step_timed */
  double phase_ms[APIC_NPHASE]; /* CUDA-event time per phase, summed over timed steps */
  int32_t solver;               /* Poisson solver in use: APIC_SOLVER_* */
  int32_t kernels_per_sort;     /* kernel launches of one particle sort */
  int64_t sorts;                /* particle sorts launched (every sort_interval steps) */
  int32_t sort_interval;        /* steps between particle sorts in use (0: none) */
  int32_t win_rows;             /* node rows of the push's shared-memory deposit window in use */
  int32_t chunk_group;          /* consecutive particle chunks a push CTA takes at a time */
  int32_t chunk_items;          /* FP32 push: particles per thread of a chunk (16: 4096 per chunk, 32: 8192) */
  int64_t timed_sorts;          /* particle sorts run inside apic_step_timed */
  double sort_ms;               /* CUDA-event time of those sorts, summed */
} apic_stats_t;

/* Poisson solvers (chosen at creation) */
#define APIC_SOLVER_MG_KERNELS 0 /* BiCGSTAB + multigrid V-cycle, one kernel per phase (FP64 batches) */
#define APIC_SOLVER_MG_COOP 1    /* the same in one cooperative launch per solve (FP64, one instance) */
#define APIC_SOLVER_BCR 2        /* FP64 iterative refinement around an FP32 block cyclic reduction of
                                    every instance in one cooperative launch (FP32 particles, any n1,
                                    grids up to 543 cells in x2): the default when the whole batch's
                                    reduction blocks fit in L2 (e.g. one 256 x 128 grid) */
#define APIC_SOLVER_ND 3         /* the same refinement around an FP32 nested-dissection factorisation (formed
                                    once at creation on the host in FP64) for some or all instances: the
                                    default otherwise (larger grids, batches); APIC_DIRECT=bcr / nd / wide
                                    (nested dissection only for grids wider than 256 cells) override */

/* Counters of the batch (launch counts, Krylov iterations, phase times). */
int apic_stats(apic_sim* sim, apic_stats_t* out);

/* As apic_step, but each phase is launched as its own CUDA graph with CUDA
 * events recorded between phases on the simulation's stream, and the elapsed
 * times are added to apic_stats_t.phase_ms.  Results are identical to
 * apic_step. */
int apic_step_timed(apic_sim* sim, int32_t n_steps);

/* ---- Autotuning ------------------------------------------------------------
 * Four schedules of the step trade against each other: the particle sort's
 * interval (the sort's cost against the push's locality: the push deposits
 * through a shared-memory window of grid rows, which works best on recently
 * sorted particles), the node rows of that window (a wider window catches
 * more of a chunk's deposits, a narrower one leaves more L1 to the field
 * gather), the chunks a push CTA takes from the shared counter at a time and
 * the size of a chunk (fewer barriers per particle against a coarser load
 * balance).  apic_autotune first runs, for each of APIC_TUNE_CANDIDATES
 * intervals c (2, 4, 6, 8, 12, 16, 24), whole sort intervals, c *
 * ceil(steps_per_trial / c) full steps each starting with a sort, timed with
 * CUDA events on the simulation's stream, and keeps the fastest; then, at
 * that interval, chunk groups 2, 4, 8, window rows 2, 4, 6, 8, 12, 16 and (FP32)
 * chunks of 16 or 32 particles per thread (the step graphs recaptured for
 * each, one warm-up interval and then the same timed steps), keeping the
 * fastest of each.  apic_stats reports the choices.  The simulation
 * advances by the steps run (results as apic_step).  Without sorting
 * (sort_interval = 0 at creation) nothing runs and 0 is returned in
 * *sort_interval.
 * ms_per_step: [APIC_TUNE_CANDIDATES] host array (or NULL) for the sort
 * intervals' measured times.  Errors: INVALID_ARG (NULL sort_interval,
 * steps_per_trial < 1), those of apic_step. */
#define APIC_TUNE_CANDIDATES 7
int apic_autotune(apic_sim* sim, int32_t steps_per_trial, int32_t* sort_interval, double* ms_per_step);

/* Apply a schedule chosen earlier (by apic_autotune on the same workload, as
 * apic_stats reported it) without measuring again.  Each argument 0 leaves
 * that setting unchanged; otherwise sort_interval >= 1 (the simulation must
 * have been created with sorting: sort_interval > 0 in some instance's
 * config, which allocates the second particle buffer), win_rows 2..16 node
 * rows of the push's deposit window, chunk_group 1..64 chunks per claim,
 * chunk_items 16 or 32 particles per thread of a push chunk (FP32; ignored
 * for FP64).  Waits for the work in flight, then recaptures the step graphs
 * at the next step; results are those of apic_step under any schedule (the
 * deposits are fixed-point sums).  Errors: INVALID_ARG (a value out of
 * range, sort_interval > 0 without sorting), a sticky error. */
int apic_set_schedule(apic_sim* sim, int32_t sort_interval, int32_t win_rows, int32_t chunk_group,
                      int32_t chunk_items);

/* ---- Sensitivity window (forward mode) and its adjoint (reverse mode) ------
 * Derivatives of window-averaged grain outputs with respect to the grain
 * shape alpha (Eqs. 2-5, 7), the grain potential phi_g (boundary value of
 * Eq. 6) and the axial magnetic field B (Eq. 9).
 *
 * Runs n_steps full steps from the current state (the state itself, in
 * (x1, x2, vR, vZ, vTheta), is held fixed: its derivatives start at zero) and
 * carries, per particle and per node, the derivatives along the three
 * parameters through every step: deposit (node volumes and the macro-weight
 * w = V_domain / n_init depend on alpha), the Poisson problem (three tangent
 * problems with the step's operator, the alpha-derivative of the Eq. 7
 * operator applied to phi on the right-hand side, d phi_g on the grain row),
 * node gradients, the gather of Eq. 10, the Boris push, the chord and Eq. 2,
 * absorption tallies, the surface field, and the injection of Eq. 4 at the
 * same random numbers.  Branch decisions (absorbed, escaped, injection
 * counts, cells) follow the values and carry no derivative (frozen-decision
 * derivative).  The window advances the simulation by n_steps steps (the
 * same state as apic_step up to rounding; particles are not re-sorted inside
 * the window).
 *
 * values:   [n_instances][APIC_NOUT] window means (NULL: not returned)
 * jacobian: [n_instances][APIC_NOUT][APIC_NPAR] derivatives of those means
 *           (NULL: not returned); host arrays owned by the caller.
 * Errors: INVALID_ARG (n_steps < 1), those of apic_step, CUDA. */
#define APIC_NPAR 3  /* parameters: alpha, phi_g, B */
#define APIC_NOUT 5  /* outputs: drag F_Z (absorbed Z momentum / dt), electric F_Z on the grain,
                        current (absorbed charge / dt), torque T_z (absorbed L_z / dt), grain charge Q */
int apic_sensitivity(apic_sim* sim, int32_t n_steps, double* values, double* jacobian);

/* Gradient of L = sum_o dL_dout[o] * output_o (window means over n_steps
 * steps from the current state) with respect to (alpha, phi_g, B), by a
 * reverse sweep with per-step checkpoints: a forward pass of the window keeps,
 * for every step, the particle state at its start, rho and phi, each slot's
 * fate and each injection draw's slot; the backward pass then transposes the
 * step's operations from the last step to the first (injection of Eq. 4,
 * the push of Eqs. 10, 9 and 2 with each particle's local Jacobian, the
 * surface charge and force, the node gradients, the Poisson problem of
 * Eqs. 6-7 solved transposed by a nested-dissection factorisation of the
 * operator in FP64, and the charge weighing with the node volumes of Eq. 5).
 * Decisions are frozen as in apic_sensitivity (the same derivative: this is
 * the transpose of its Jacobian).  The window advances the simulation by
 * n_steps steps.  Memory: 5 n_steps particle arrays of checkpoints, 2 n_steps
 * FP64 node arrays and a factorisation of each instance's operator (formed at
 * the first call, a few seconds for 1024 x 512 cells).
 * dL_dout: [n_instances][APIC_NOUT]; values (or NULL): [n_instances][APIC_NOUT]
 * window means; grad: [n_instances][APIC_NPAR]; host arrays owned by the
 * caller.  Errors: as apic_sensitivity; INVALID_ARG for NULL dL_dout or grad. */
int apic_adjoint_window(apic_sim* sim, int32_t n_steps, const double* dL_dout, double* values, double* grad);

/* apic_adjoint_window without the window means. */
int apic_adjoint(apic_sim* sim, int32_t n_steps, const double* dL_dout, double* grad);

/* ---- Charge deposit without device allocation --------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory (a component living inside another
 * program's fixed device-memory budget, a framework that only hands out the
 * buffers it manages, a loop that must not enter the allocator).
 *
 * rho[i][j] = qw * sum_p S_ij(p) / volume[i][j]: the cloud-in-cell weights S
 * of the n particles at (x1[p], x2[p]) on the grid `grid` (n1 x n2 cells,
 * x1 in [-1, x1_outer], x2 in [-1, 1]), the same weighing as the deposit of
 * an FP64 (APIC_FP64) instance's apic_step, with 64-bit fixed-point sums (an
 * FP32 instance rounds the cell fractions to 16 bits first, a difference of
 * up to 2^-17 of a particle's charge per node).  A particle outside
 * [-1, x1_outer] x [-1, 1] or with a non-finite coordinate is skipped (it adds
 * no charge), as a freed or escaped slot of a simulation is.  x1, x2 (n doubles), volume and rho
 * ((n1+1)(n2+1) doubles, row-major) are device pointers owned by the caller;
 * work is queued on `stream` (a cudaStream_t) and the call returns without
 * waiting.  No cudaMalloc, cudaFree or other allocating call is made.
 *
 * Scratch: one static accumulator of 2^20 nodes (8 MiB) per device, held
 * from library load until process exit; grids with (n1+1)(n2+1) > 2^20 are
 * rejected with APIC_ERR_INVALID_ARG.  Every call shares that accumulator and
 * clears it first: calls that overlap on the GPU (different streams or host
 * threads without ordering) race and give wrong densities.  The first call on
 * each device looks up the accumulator's device address; make that first
 * call before any stream capture.
 * Errors: INVALID_ARG (NULL pointer, bad grid, too many nodes), CUDA. */
typedef struct {
  int32_t n1, n2;   /* cells in x1 and x2 */
  double x1_outer;  /* outer boundary x1, in (-1, 0) */
} apic_grid_t;

int apic_deposit_static(const apic_grid_t* grid, const double* x1, const double* x2, int64_t n, double qw,
                        const double* volume, double* rho, void* stream);

/* Failure-detection check: launches four CTAs that wait at a grid barrier
 * of the kind the cooperative solvers use, set up so that it never completes
 * (one arrival more than there are CTAs), with the wait limited to limit_ns
 * of global time (1e3 .. 1e10) instead of the solvers' 2 s.  Each wait gives up
 * at the limit, sets the status word's time-out bit and its CTA returns; the
 * call then reads the status word as apic_step does and returns
 * APIC_ERR_TIMEOUT, which the object keeps (sticky).  The CUDA context stays
 * usable: other objects are unaffected.  Errors: INVALID_ARG, TIMEOUT (the
 * expected result), CUDA. */
int apic_check_wait_limit(apic_sim* sim, int64_t limit_ns);

/* FP32 CUDA-core throughput of the current device in TFLOP/s: independent fused
 * multiply-add chains (2 FLOPs each) over every SM, reps iterations per chain,
 * timed with CUDA events on `stream` (a cudaStream_t; NULL: the default stream)
 * after one warm-up launch.  It is the ALU ceiling that the push's arithmetic
 * is compared with (the measured peaks hold only memory bandwidth and tensor
 * throughput).  Waits for the stream.
 * Errors: INVALID_ARG (NULL tflops, reps < 1), CUDA. */
int apic_probe_fp32_fma(void* stream, int32_t reps, double* tflops);

#ifdef __cplusplus
}
#endif
#endif /* APIC_H */
