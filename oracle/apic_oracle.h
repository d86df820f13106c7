/*
 * FP64 CPU oracle for the APIC particle-in-cell step (Smirnov & Krasheninnikov,
 * "Aspherical PIC code (APIC) ...", arXiv:2307.11107).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the plain, slow reference the CUDA
 * path is checked against.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load it; the product library never does.
 * It shares no source, header, table or constant generator with the CUDA path.
 *
 * Units: lengths in R0, time in 1/omega_pe, velocity in lambda_De*omega_pe,
 * potential in Te/e, density in n0, eps0 = 1 (so Eq. 6 reads Lap(phi) = -rho).
 * Grid: n1 x n2 CELLS, nodes (i, j) with i = 0..n1 (x1 = -1 + i*h1) and
 * j = 0..n2 (x2 = -1 + j*h2); node index = i*(n2+1) + j.
 *
 * Functions whose value is pinned only by invariants of the method (not by a
 * printed number) are marked in apic_oracle.c; the paper prints no numbers.
 */
#ifndef APIC_ORACLE_H
#define APIC_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

#define OR_NO_INJECT 1   /* skip surface injection (Sec. 1 injection) */
#define OR_NO_FIELD 2    /* phi == 0 everywhere: no deposit/Poisson feed-back */
#define OR_CHORD 4       /* also absorb when the step's chord passes through the grain */
#define OR_CHORD_SAMPLES 8 /* the chord is tested at s = k / OR_CHORD_SAMPLES, k = 1..7 */
#define OR_FLOATING 8    /* isolated grain: its potential follows the charge it collects */
#define OR_BOLTZMANN 16  /* electrons not simulated: n_e = exp(phi) in Eq. 6, solved by Newton; the grain
                            collects their Maxwellian flux exp(phi_g) sqrt(1/2pi) per unit area */
#define OR_FE 32         /* conservative (bilinear finite-element) form of Eqs. 6-7 instead of Eq. 7's differences */

#define OR_NT 7          /* tally components per bin */
#define OR_NH 11         /* history fields per step (the last: the grain potential used) */

typedef struct {
  double q, m, T;
  int64_t n_init;        /* macro-particles of the initial volume load; sets w */
} or_species;

typedef struct {
  double alpha, x1_out, phi_g, phi_out, B, dt, e_bind_ion;
  int32_t n1, n2, n_species;
  or_species sp[2];
  uint64_t seed;
  int32_t instance;
  int32_t flags;
} or_config;

typedef struct or_sim or_sim;

/* ---- pieces exported for the pin tests ---- */
double or_r_of(double alpha, double x1, double x2);             /* Eq. 3 */
double or_x1_of(double alpha, double r, double x2);             /* Eq. 2 */
void or_metric(double alpha, double r, double x2, double out[4]);/* dx1/dR, dx1/dZ, dx2/dR, dx2/dZ */
double or_dA_dx2(double alpha, double x1, double x2);           /* Eq. 4, R0 = 1 */
double or_dOmega(double alpha, double x1, double x2);           /* Eq. 5, R0 = 1 */
void or_philox4x32(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void or_gauss_legendre(int n, double* x, double* w);            /* nodes/weights on [-1,1] */

/* ---- simulation ---- */
or_sim* or_create(const or_config* cfg);
void or_destroy(or_sim* s);
int or_load_volume(or_sim* s, int sp, int64_t n);
int or_add_particles(or_sim* s, int sp, int64_t n, const double* state5);
int or_step(or_sim* s, int n_steps);
int or_deposit(or_sim* s);                  /* rho from the current particles */
int or_solve(or_sim* s, const double* rho_or_null, double* phi_out);
int or_solve_linear(or_sim* s, const double* rho, double* phi_out); /* Eqs. 6-7 with rho, any electron model */
int or_newton_iterations(const or_sim* s);  /* Boltzmann electrons: Newton iterations of the last step's solve */
void or_apply_operator(const or_sim* s, const double* phi, double* out); /* L phi per node (see apic_oracle.c) */
void or_set_phi(or_sim* s, const double* phi); /* phi := caller values [n1+1][n2+1] (pin tests) */
void or_gradients(or_sim* s);               /* G1, G2 from the current phi */
int or_push_only(or_sim* s);                /* gather + push + absorb + escape, no inject */

/* ---- accessors ---- */
int64_t or_count(const or_sim* s, int sp);
int or_get_particles(const or_sim* s, int sp, double* state5, int64_t* ids);
void or_get_grid(const or_sim* s, int which, double* out); /* 0 rho,1 phi,2 G1,3 G2,4 V */
void or_get_bins(const or_sim* s, double* out);            /* [n_species][n2][OR_NT] */
int64_t or_get_history(const or_sim* s, double* out);      /* [steps][OR_NH]; returns steps */
void or_get_counts(const or_sim* s, int64_t* out); /* [2][6] loaded, injected, absorbed, escaped, resident, draws */
void or_get_scalars(const or_sim* s, double* out);         /* w0,w1,V_dom,A_out,A_grain,lam0,lam1,Q,FZ */
void or_surface(or_sim* s, double* En_out, double* Q, double* FZ);
double or_sample_table(const or_sim* s, int which, double u); /* 0 volume, 1 surface */

/* ---- decision tape: frozen-decision runs for finite-difference derivatives ---- */
#define OR_TAPE_OFF 0
#define OR_TAPE_RECORD 1  /* store every absorb/escape/keep decision, injection count, cell and table interval */
#define OR_TAPE_REPLAY 2  /* take them from the tape instead of the geometry */
void or_tape_mode(or_sim* s, int mode);
int64_t or_tape_get(const or_sim* s, uint8_t* st, int64_t* nk, int64_t* n_nk); /* returns status count */
void or_tape_set(or_sim* s, const uint8_t* st, int64_t n, const int64_t* nk, int64_t n_nk);
int or_tape_status(const or_sim* s); /* -1 if a replay ran past the end of its tape */
int64_t or_tape_ix_get(const or_sim* s, int32_t* out);          /* cells and table intervals; returns the count */
void or_tape_ix_set(or_sim* s, const int32_t* ix, int64_t n);

#ifdef __cplusplus
}
#endif
#endif
