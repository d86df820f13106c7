/*
 * FP64 CPU oracle of the APIC particle-in-cell step (arXiv:2307.11107).
 *
 * TEST INFRASTRUCTURE ONLY: the plain, slow, obviously-correct definition the
 * CUDA path is compared with.  It is loaded only by the tests, the smoke check
 * and the benchmark's CPU-baseline leg.  Compile with -ffp-contract=off so that
 * no multiply-add is fused behind the reader's back.
 *
 * Every function cites the passage of the paper it follows.  Where the paper is
 * silent the reading taken is stated at the function.  The paper prints no
 * numeric results (Figs. 1-3 are plots), so all dynamic quantities are pinned
 * only by invariants (round trips, closed forms, conservation laws); the tests
 * say which invariant pins which function.
 *
 * Options beside the paper's method, each off by default and pinned by its own
 * tests: chord-intersection absorption of grazing orbits (OR_CHORD), the
 * isolated grain whose potential follows the collected charge (OR_FLOATING),
 * Boltzmann electrons solved by Newton (OR_BOLTZMANN; the paper mentions the
 * option in Sec. 2), and the conservative finite-element form of Eqs. 6-7
 * (OR_FE).
 */
#include "apic_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846
#define TABLE_M 4096 /* intervals of the inverse-CDF sampling tables */
#define BISECT_IT 40 /* bisection steps for the impact point */

/* ------------------------------------------------------------------------ */
/* Geometry: Eqs. 2-5, 8 and the metric needed by Eq. 10.                    */
/* ------------------------------------------------------------------------ */

/* Eq. 3: r(x1, x2) = -(1 + sqrt(1 - 4 alpha x1 x2)) / (2 x1). */
double or_r_of(double alpha, double x1, double x2) {
  return -(1.0 + sqrt(1.0 - 4.0 * alpha * x1 * x2)) / (2.0 * x1);
}

/* Eq. 2: x1 = -(1/r)(1 + alpha cos(theta)/r), with x2 = cos(theta). */
double or_x1_of(double alpha, double r, double x2) {
  return -(1.0 / r) * (1.0 + alpha * x2 / r);
}

/* Grain surface x1 = -1 (Eq. 3): r_g(x2) = (1 + sqrt(1 + 4 alpha x2)) / 2. */
static double r_grain(double alpha, double x2) {
  return (1.0 + sqrt(1.0 + 4.0 * alpha * x2)) / 2.0;
}

/* Grazing orbits (option OR_CHORD): the step's straight chord P(s) = (R + s dx,
 * s dy, Z + s dz), s in [0, 1], in the local Cartesian frame of the start
 * point, may pass through the grain although its end point lies outside.
 * Returns the first of the points s = k / OR_CHORD_SAMPLES (k = 1..7) that
 * lies inside the grain, or 0 if none does.  Chords whose closest approach
 * to the origin stays beyond the grain's largest radius (1 + sqrt(1 +
 * 4 |alpha|)) / 2 are not sampled. */
static double chord_entry(double al, double R, double Z, double dx, double dy, double dz) {
  double dd = dx * dx + dy * dy + dz * dz;
  double s0 = dd > 0.0 ? -(R * dx + Z * dz) / dd : 0.0;
  if (s0 < 0.0) s0 = 0.0;
  if (s0 > 1.0) s0 = 1.0;
  double px = R + s0 * dx, py = s0 * dy, pz = Z + s0 * dz;
  double rmax = 0.5 * (1.0 + sqrt(1.0 + 4.0 * fabs(al)));
  if (px * px + py * py + pz * pz >= rmax * rmax) return 0.0;
  for (int k = 1; k < OR_CHORD_SAMPLES; ++k) {
    double sk = (double)k / OR_CHORD_SAMPLES;
    double qx = R + sk * dx, qy = sk * dy, qz = Z + sk * dz;
    double rr = sqrt(qx * qx + qy * qy + qz * qz);
    if (rr < r_grain(al, qz / rr)) return sk;
  }
  return 0.0;
}

/* Partial derivatives of (x1, x2) with respect to the cylindrical (R, Z) of
 * Eq. 8, obtained by the chain rule from Eq. 2 with r^2 = R^2 + Z^2 and
 * x2 = Z/r.  They are the "coordinate derivatives found analytically" that
 * Eq. 10 multiplies with the numerical dphi/dx_i (Sec. 2, after Eq. 10).
 * s = sin(theta) = sqrt((1 - x2)(1 + x2)). */
void or_metric(double alpha, double r, double x2, double out[4]) {
  double s2 = (1.0 - x2) * (1.0 + x2);
  double s = sqrt(s2);
  double r3 = r * r * r;
  out[0] = s * (r + 3.0 * alpha * x2) / r3;                        /* dx1/dR */
  out[1] = (r * x2 + alpha * (3.0 * x2 * x2 - 1.0)) / r3;          /* dx1/dZ */
  out[2] = -x2 * s / r;                                            /* dx2/dR */
  out[3] = s2 / r;                                                 /* dx2/dZ */
}

/* Eq. 4 (R0 = 1): dA/dx2 on the surface x1 = const. */
double or_dA_dx2(double alpha, double x1, double x2) {
  double r = or_r_of(alpha, x1, x2);
  double s2 = (1.0 - x2) * (1.0 + x2);
  double t = alpha / (r + 2.0 * alpha * x2);
  return 2.0 * OR_PI * r * r * sqrt(1.0 + s2 * t * t);
}

/* Eq. 5 (R0 = 1): dOmega / (dx1 dx2). */
double or_dOmega(double alpha, double x1, double x2) {
  double r = or_r_of(alpha, x1, x2);
  return 2.0 * OR_PI * r * r * r * r / (1.0 + 2.0 * alpha * x2 / r);
}

/* Coefficients of the Laplacian of Eq. 7 at (x1, x2):
 * c[0] d2/dx1^2 + c[1] d2/dx2^2 + c[2] d2/dx1dx2 + c[3] d/dx2. */
static void lap_coef(double alpha, double x1, double x2, double c[4]) {
  double r = or_r_of(alpha, x1, x2);
  double s2 = (1.0 - x2) * (1.0 + x2);
  double r2 = r * r, r4 = r2 * r2, r6 = r4 * r2;
  double a = r + 2.0 * alpha * x2;
  c[0] = (a * a + alpha * alpha * s2) / r6;
  c[1] = s2 / r2;
  c[2] = -2.0 * alpha * s2 / r4;
  c[3] = -2.0 * x2 / r2;
}

/* Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n
 * (textbook construction; used only for the quadratures below). */
void or_gauss_legendre(int n, double* x, double* w) {
  for (int k = 0; k < n; ++k) {
    double z = cos(OR_PI * (k + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int l = 2; l <= n; ++l) {
        double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
        p0 = p1;
        p1 = p2;
      }
      /* p1 = P_n(z), p0 = P_{n-1}(z) */
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int l = 2; l <= n; ++l) {
      double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[k] = z;
    w[k] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its definition:   */
/* round: (hi0,lo0) = M0*c0, (hi1,lo1) = M1*c2;                              */
/*        c <- (hi1^c1^k0, lo1, hi0^c3^k1, lo0); key += (W0, W1) per round.  */
/* ------------------------------------------------------------------------ */
void or_philox4x32(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* 32-bit integer to a uniform in (0,1): (u + 1/2) / 2^32, exact in FP64. */
static double u01(uint32_t u) { return ((double)u + 0.5) * (1.0 / 4294967296.0); }

/* Box-Muller: two uniforms to two standard normals. */
static void box_muller(double ua, double ub, double* z0, double* z1) {
  double rad = sqrt(-2.0 * log(ua));
  *z0 = rad * cos(2.0 * OR_PI * ub);
  *z1 = rad * sin(2.0 * OR_PI * ub);
}

/* ------------------------------------------------------------------------ */
/* Simulation state.                                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
  double *x1, *x2, *vR, *vZ, *vT;
  int64_t* id;
  int64_t n, cap, next_id;
  int64_t draws; /* Philox draw counter (one per sampled particle) */
  int64_t loaded, injected, absorbed, escaped;
  double carry; /* fractional injection carry */
} species_state;

struct or_sim {
  or_config c;
  int N1, N2;   /* nodes per direction = cells + 1 */
  double h1, h2;
  double *rho, *phi, *G1, *G2, *V;
  /* banded LU of the Eq. 6-7 finite-difference matrix */
  int nu, kl, ku, ld;
  double* band;
  int* piv;
  /* sampling tables: CDF on TABLE_M intervals of x2 */
  double cdf_vol[TABLE_M + 1], cdf_surf[TABLE_M + 1];
  double V_dom, A_out, A_grain, w[2], lam[2];
  species_state sp[2];
  double* bins; /* [n_species][n2][OR_NT], cumulative */
  double* hist;
  int64_t hist_n, hist_cap, step;
  double Q, FZ;
  double step_tally[5]; /* this step's charge, pZ, Lz, heat, events (history) */
  /* isolated grain (OR_FLOATING): potential of this step, collected charge,
   * and the vacuum field of a grain at potential 1 (outer boundary at 0) */
  double phig, Qg, C_vac;
  int qg_set;
  int newton_its; /* Boltzmann electrons: Newton iterations of the last solve (-1: no convergence) */
  double* phi_vac;
  /* decision tape: one status byte per particle update and per injection
   * draw, in processing order, and one injection count per step and species */
  int tape_mode;        /* OR_TAPE_OFF, OR_TAPE_RECORD, OR_TAPE_REPLAY */
  int tape_short;       /* a replay ran past the end of its tape */
  uint8_t* tape_st;
  int64_t tape_n, tape_cap, tape_pos;
  int64_t* tape_nk;
  int64_t tape_nk_n, tape_nk_cap, tape_nk_pos;
  /* cells and table intervals: every locate (packed i (n2+1) + j) and every
   * injection's table interval, in the order they are taken */
  int32_t* tape_ix;
  int64_t tape_ix_n, tape_ix_cap, tape_ix_pos;
};

/* Decision of one particle update or injection draw under the tape: the
 * natural decision (record mode stores it), or the recorded one (replay). */
static int tape_status(or_sim* s, int natural) {
  if (s->tape_mode == OR_TAPE_RECORD) {
    if (s->tape_n == s->tape_cap) {
      s->tape_cap = s->tape_cap ? 2 * s->tape_cap : 4096;
      s->tape_st = (uint8_t*)realloc(s->tape_st, (size_t)s->tape_cap);
    }
    s->tape_st[s->tape_n++] = (uint8_t)natural;
    return natural;
  }
  if (s->tape_mode == OR_TAPE_REPLAY) {
    if (s->tape_pos < s->tape_n) return s->tape_st[s->tape_pos++];
    s->tape_short = 1;
  }
  return natural;
}

/* An integer choice (a particle's cell, a table interval) under the tape:
 * record mode stores the natural one, replay returns the recorded one. */
static int tape_int(or_sim* s, int natural) {
  if (s->tape_mode == OR_TAPE_RECORD) {
    if (s->tape_ix_n == s->tape_ix_cap) {
      s->tape_ix_cap = s->tape_ix_cap ? 2 * s->tape_ix_cap : 65536;
      s->tape_ix = (int32_t*)realloc(s->tape_ix, sizeof(int32_t) * (size_t)s->tape_ix_cap);
    }
    s->tape_ix[s->tape_ix_n++] = natural;
    return natural;
  }
  if (s->tape_mode == OR_TAPE_REPLAY) {
    if (s->tape_ix_pos < s->tape_ix_n) return s->tape_ix[s->tape_ix_pos++];
    s->tape_short = 1;
  }
  return natural;
}

static int64_t tape_count(or_sim* s, int64_t natural) {
  if (s->tape_mode == OR_TAPE_RECORD) {
    if (s->tape_nk_n == s->tape_nk_cap) {
      s->tape_nk_cap = s->tape_nk_cap ? 2 * s->tape_nk_cap : 256;
      s->tape_nk = (int64_t*)realloc(s->tape_nk, sizeof(int64_t) * (size_t)s->tape_nk_cap);
    }
    s->tape_nk[s->tape_nk_n++] = natural;
    return natural;
  }
  if (s->tape_mode == OR_TAPE_REPLAY) {
    if (s->tape_nk_pos < s->tape_nk_n) return s->tape_nk[s->tape_nk_pos++];
    s->tape_short = 1;
  }
  return natural;
}

static double x1_node(const or_sim* s, int i) { return i == s->c.n1 ? s->c.x1_out : -1.0 + i * s->h1; }
static double x2_node(const or_sim* s, int j) { return j == s->c.n2 ? 1.0 : -1.0 + j * s->h2; }

/* Hat-weighted node volumes V_ij = integral of S_ij dOmega (Eq. 5), where S_ij
 * is the bilinear (cloud-in-cell) weight of node (i,j) in (x1, x2).  Reading of
 * "volume-weighted charge weighing" (Sec. 2, after Eq. 5): charge is shared by
 * CIC in the logical (x1, x2) grid and divided by this volume, so that a
 * uniform density gives rho = n0 in expectation.  8x8 Gauss-Legendre per cell. */
static void build_volumes(or_sim* s) {
  double gx[8], gw[8];
  or_gauss_legendre(8, gx, gw);
  int N2 = s->N2;
  memset(s->V, 0, sizeof(double) * (size_t)s->N1 * N2);
  for (int ci = 0; ci < s->c.n1; ++ci) {
    double xa = x1_node(s, ci), xb = x1_node(s, ci + 1);
    for (int cj = 0; cj < s->c.n2; ++cj) {
      double ya = x2_node(s, cj), yb = x2_node(s, cj + 1);
      double acc[4] = {0, 0, 0, 0};
      for (int a = 0; a < 8; ++a) {
        double f1 = 0.5 * (gx[a] + 1.0);
        double x1 = xa + f1 * (xb - xa);
        for (int b = 0; b < 8; ++b) {
          double f2 = 0.5 * (gx[b] + 1.0);
          double x2 = ya + f2 * (yb - ya);
          double wq = 0.25 * gw[a] * gw[b] * (xb - xa) * (yb - ya) * or_dOmega(s->c.alpha, x1, x2);
          acc[0] += wq * (1.0 - f1) * (1.0 - f2);
          acc[1] += wq * f1 * (1.0 - f2);
          acc[2] += wq * (1.0 - f1) * f2;
          acc[3] += wq * f1 * f2;
        }
      }
      s->V[ci * N2 + cj] += acc[0];
      s->V[(ci + 1) * N2 + cj] += acc[1];
      s->V[ci * N2 + cj + 1] += acc[2];
      s->V[(ci + 1) * N2 + cj + 1] += acc[3];
    }
  }
}

/* Cumulative tables on x2 in [-1, 1] (TABLE_M intervals, 8-point GL each):
 *  - volume density dV/dx2 = (2 pi / 3)(r_out^3 - r_g^3), from integrating
 *    Eq. 5 over x1 (dOmega = 2 pi r^2 dr dx2 along a line of constant x2);
 *  - surface density dA/dx2 of Eq. 4 at x1 = x1_out (injection, Sec. 1). */
static double vol_density(const or_sim* s, double x2) {
  double ro = or_r_of(s->c.alpha, s->c.x1_out, x2), rg = r_grain(s->c.alpha, x2);
  return 2.0 * OR_PI / 3.0 * (ro * ro * ro - rg * rg * rg);
}

static void build_tables(or_sim* s) {
  double gx[8], gw[8];
  or_gauss_legendre(8, gx, gw);
  double ht = 2.0 / TABLE_M;
  s->cdf_vol[0] = 0.0;
  s->cdf_surf[0] = 0.0;
  double ag = 0.0;
  for (int k = 0; k < TABLE_M; ++k) {
    double a = -1.0 + k * ht;
    double sv = 0.0, ss = 0.0, sg = 0.0;
    for (int q = 0; q < 8; ++q) {
      double x2 = a + 0.5 * (gx[q] + 1.0) * ht;
      sv += 0.5 * ht * gw[q] * vol_density(s, x2);
      ss += 0.5 * ht * gw[q] * or_dA_dx2(s->c.alpha, s->c.x1_out, x2);
      sg += 0.5 * ht * gw[q] * or_dA_dx2(s->c.alpha, -1.0, x2);
    }
    s->cdf_vol[k + 1] = s->cdf_vol[k] + sv;
    s->cdf_surf[k + 1] = s->cdf_surf[k] + ss;
    ag += sg;
  }
  s->V_dom = s->cdf_vol[TABLE_M];
  s->A_out = s->cdf_surf[TABLE_M];
  s->A_grain = ag;
}

/* Inverse CDF with linear interpolation inside the table interval (under a
 * decision tape the interval is recorded or replayed, the interpolation
 * follows the parameters). */
static double sample_table_in(or_sim* s, const double* cdf, double u) {
  double t = u * cdf[TABLE_M];
  int lo = 0, hi = TABLE_M;
  while (hi - lo > 1) {
    int mid = (lo + hi) / 2;
    if (cdf[mid] <= t) lo = mid; else hi = mid;
  }
  if (s) lo = tape_int(s, lo);
  double ht = 2.0 / TABLE_M;
  double d = cdf[lo + 1] - cdf[lo];
  double f = d > 0.0 ? (t - cdf[lo]) / d : 0.5;
  return -1.0 + lo * ht + f * ht;
}

static double sample_table(const double* cdf, double u) { return sample_table_in(NULL, cdf, u); }

double or_sample_table(const or_sim* s, int which, double u) {
  return sample_table(which == 0 ? s->cdf_vol : s->cdf_surf, u);
}

/* ------------------------------------------------------------------------ */
/* Poisson problem, Eqs. 6-7, second-order finite differences (Sec. 2).      */
/* Unknowns: nodes i = 1..n1-1, j = 0..n2; Dirichlet phi = phi_g at i = 0    */
/* (grain, x1 = -1) and phi = phi_out at i = n1 (outer surface), Sec. 1.     */
/* Interior j: central differences; the cross derivative uses the four       */
/* diagonal neighbours / (4 h1 h2).  Pole rows j = 0, n2 (x2 = -+1): the     */
/* d2/dx2^2 and cross coefficients of Eq. 7 vanish there and d/dx2 is taken  */
/* one-sided to second order (reading: the paper does not state the pole     */
/* treatment).  Solved by banded LU with partial pivoting, factorised once   */
/* (the matrix is constant in time), as the paper's LAPACK LU (Sec. 2).      */
/* ------------------------------------------------------------------------ */
#define UIDX(s, i, j) (((i) - 1) * (s)->N2 + (j))
#define BANDA(a, s, r, c) (a)[(size_t)(c) * (s)->ld + ((r) - (c) + (s)->kl + (s)->ku)]

/* Conservative form (option OR_FE; the paper discretises Eq. 7 by finite
 * differences, Sec. 2): the weak form of Eq. 6 with the bilinear hat
 * functions N_a of the logical grid, whose own weights are the charge
 * assignment, int rho N_a dOmega = rho_a V_a (Eq. 5's V_a):
 *   sum_b K_ab phi_b = rho_a V_a,
 *   K_ab = int grad N_a . grad N_b dOmega
 *        = int (J g^kl dN_a/dx_k dN_b/dx_l) dx1 dx2,
 * g^kl = grad x_k . grad x_l from the chain rule of Eq. 2 (or_metric) and
 * J = dOmega / (dx1 dx2) of Eq. 5, integrated per cell by quadrature.  K is
 * symmetric, and its rows over all nodes sum to zero (the hat functions sum
 * to one), so the discrete Gauss law holds exactly.  Cell (ci, cj) has the
 * corners p = px + 2 py at nodes (ci + px, cj + py). */
static void fe_cell(const or_sim* s, int ci, int cj, double K[4][4]) {
  /* 3 x 3 Gauss-Legendre points of the cell; in the two cells next to a pole
   * the x2 points are placed in t = sqrt(distance to the pole), where J's
   * sqrt(1 - x2^2) growth becomes smooth */
  static const double gx[3] = {-0.7745966692414834, 0.0, 0.7745966692414834};
  static const double gw[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
  double xa = x1_node(s, ci), xb = x1_node(s, ci + 1), ya = x2_node(s, cj), yb = x2_node(s, cj + 1);
  memset(K, 0, sizeof(double) * 16);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double f1 = 0.5 * (gx[a] + 1.0), x1 = xa + f1 * (xb - xa);
      double wq = 0.25 * gw[a] * gw[b] * (xb - xa) * (yb - ya);
      double f2 = 0.5 * (gx[b] + 1.0), x2;
      if (cj == 0) {          /* x2 = -1 + h2 t^2, dx2 = 2 h2 t dt */
        x2 = ya + (yb - ya) * f2 * f2;
        wq *= 2.0 * f2;
        f2 = f2 * f2;
      } else if (cj == s->c.n2 - 1) {  /* x2 = 1 - h2 t^2 */
        double t = f2;
        x2 = yb - (yb - ya) * t * t;
        wq *= 2.0 * t;
        f2 = 1.0 - t * t;
      } else {
        x2 = ya + f2 * (yb - ya);
      }
      double m[4];
      or_metric(s->c.alpha, or_r_of(s->c.alpha, x1, x2), x2, m);
      double g11 = m[0] * m[0] + m[1] * m[1], g22 = m[2] * m[2] + m[3] * m[3], g12 = m[0] * m[2] + m[1] * m[3];
      double J = or_dOmega(s->c.alpha, x1, x2);
      /* derivatives of the bilinear corner functions at (f1, f2) */
      double d1[4], d2[4];
      for (int p = 0; p < 4; ++p) {
        int px = p & 1, py = p >> 1;
        double sx = px ? 1.0 : -1.0, sy = py ? 1.0 : -1.0;
        double ex = px ? f1 : 1.0 - f1, ey = py ? f2 : 1.0 - f2;
        d1[p] = sx * ey / (xb - xa);
        d2[p] = sy * ex / (yb - ya);
      }
      for (int p = 0; p < 4; ++p)
        for (int q = 0; q < 4; ++q)
          K[p][q] += wq * J * (g11 * d1[p] * d1[q] + g12 * (d1[p] * d2[q] + d2[p] * d1[q]) + g22 * d2[p] * d2[q]);
    }
}

/* Row (i, j) of the conservative form divided by -V_ij, in the layout of
 * stencil(): sum_b w_b phi_b = -rho_ij. */
static void stencil_fe(const or_sim* s, int i, int j, double w[3][5]) {
  memset(w, 0, sizeof(double) * 15);
  double V = s->V[i * s->N2 + j];
  for (int ci = i - 1; ci <= i; ++ci)
    for (int cj = j - 1; cj <= j; ++cj) {
      if (ci < 0 || ci >= s->c.n1 || cj < 0 || cj >= s->c.n2) continue;
      double K[4][4];
      fe_cell(s, ci, cj, K);
      int pa = (i - ci) | ((j - cj) << 1);
      for (int q = 0; q < 4; ++q) {
        int di = ci + (q & 1) - i, dj = cj + (q >> 1) - j;
        w[di + 1][dj + 2] -= K[pa][q] / V;
      }
    }
}

/* The nine stencil weights of node (i, j): w[di+1][dj+2] for di in -1..1,
 * dj in -2..2 (the pole rows reach two nodes in j). */
static void stencil(const or_sim* s, int i, int j, double w[3][5]) {
  if (s->c.flags & OR_FE) {
    stencil_fe(s, i, j, w);
    return;
  }
  memset(w, 0, sizeof(double) * 15);
  double c[4];
  lap_coef(s->c.alpha, x1_node(s, i), x2_node(s, j), c);
  double ih1 = 1.0 / (s->h1 * s->h1);
  double a1 = c[0] * ih1;
  w[0][2] += a1;
  w[2][2] += a1;
  w[1][2] += -2.0 * a1;
  if (j == 0 || j == s->c.n2) {
    double e = c[3] / (2.0 * s->h2);
    double sg = (j == 0) ? 1.0 : -1.0; /* forward at x2 = -1, backward at +1 */
    w[1][2] += e * sg * (-3.0);
    w[1][2 + (int)sg] += e * sg * 4.0;
    w[1][2 + 2 * (int)sg] += e * sg * (-1.0);
  } else {
    double a2 = c[1] / (s->h2 * s->h2);
    double e = c[3] / (2.0 * s->h2);
    double d = c[2] / (4.0 * s->h1 * s->h2);
    w[1][1] += a2 - e;
    w[1][3] += a2 + e;
    w[1][2] += -2.0 * a2;
    w[2][3] += d;
    w[0][1] += d;
    w[2][1] -= d;
    w[0][3] -= d;
  }
}

/* The matrix of the interior unknowns in band storage, plus shift[node] on
 * the diagonal (NULL: none), then its LU factors with partial pivoting
 * (column c keeps rows c-(kl+ku) .. c+kl; fill-in from row swaps stays inside
 * that band). */
static void assemble_factor(or_sim* s, const double* shift, double* band, int* piv) {
  memset(band, 0, sizeof(double) * (size_t)s->ld * s->nu);
  for (int i = 1; i < s->c.n1; ++i)
    for (int j = 0; j < s->N2; ++j) {
      double w[3][5];
      stencil(s, i, j, w);
      int r = UIDX(s, i, j);
      if (shift) w[1][2] += shift[i * s->N2 + j];
      for (int di = -1; di <= 1; ++di)
        for (int dj = -2; dj <= 2; ++dj) {
          double v = w[di + 1][dj + 2];
          if (v == 0.0) continue;
          int ii = i + di, jj = j + dj;
          if (ii < 1 || ii > s->c.n1 - 1) continue; /* Dirichlet: goes to the rhs */
          BANDA(band, s, r, UIDX(s, ii, jj)) += v;
        }
    }
  int n = s->nu, kl = s->kl, kuu = s->kl + s->ku;
  for (int j = 0; j < n; ++j) {
    int km = kl < n - 1 - j ? kl : n - 1 - j;
    int p = j;
    double best = fabs(BANDA(band, s, j, j));
    for (int r = j + 1; r <= j + km; ++r)
      if (fabs(BANDA(band, s, r, j)) > best) { best = fabs(BANDA(band, s, r, j)); p = r; }
    piv[j] = p;
    int cmax = j + kuu < n - 1 ? j + kuu : n - 1;
    if (p != j)
      for (int c = j; c <= cmax; ++c) {
        double t = BANDA(band, s, j, c);
        BANDA(band, s, j, c) = BANDA(band, s, p, c);
        BANDA(band, s, p, c) = t;
      }
    double inv = 1.0 / BANDA(band, s, j, j);
    for (int r = j + 1; r <= j + km; ++r) BANDA(band, s, r, j) *= inv;
    for (int c = j + 1; c <= cmax; ++c) {
      double u = BANDA(band, s, j, c);
      if (u == 0.0) continue;
      for (int r = j + 1; r <= j + km; ++r) BANDA(band, s, r, c) -= BANDA(band, s, r, j) * u;
    }
  }
}

/* b <- A^-1 b with the factors of assemble_factor. */
static void lu_solve(const or_sim* s, const double* band, const int* piv, double* b) {
  int n = s->nu, kl = s->kl, kuu = s->kl + s->ku;
  for (int j = 0; j < n; ++j) {
    int p = piv[j];
    if (p != j) { double t = b[j]; b[j] = b[p]; b[p] = t; }
    int km = kl < n - 1 - j ? kl : n - 1 - j;
    for (int r = j + 1; r <= j + km; ++r) b[r] -= BANDA(band, s, r, j) * b[j];
  }
  for (int j = n - 1; j >= 0; --j) {
    b[j] /= BANDA(band, s, j, j);
    int r0 = j - kuu > 0 ? j - kuu : 0;
    for (int r = r0; r < j; ++r) b[r] -= BANDA(band, s, r, j) * b[j];
  }
}

static void build_matrix(or_sim* s) {
  s->nu = (s->c.n1 - 1) * s->N2;
  s->kl = s->N2 + 2;
  s->ku = s->N2 + 2;
  s->ld = 2 * s->kl + s->ku + 1;
  s->band = (double*)calloc((size_t)s->ld * s->nu, sizeof(double));
  s->piv = (int*)calloc((size_t)s->nu, sizeof(int));
  assemble_factor(s, NULL, s->band, s->piv);
}

/* Right-hand side of row (i, j): -rho plus the Dirichlet terms moved from
 * the grain row (phig) and the outer row (phiout). */
static double row_rhs(const or_sim* s, int i, int j, double rho, double phig, double phiout) {
  double w[3][5];
  stencil(s, i, j, w);
  double rhs = -rho;
  for (int dj = -2; dj <= 2; ++dj) {
    if (i - 1 == 0) rhs -= w[0][dj + 2] * phig;
    if (i + 1 == s->c.n1) rhs -= w[2][dj + 2] * phiout;
  }
  return rhs;
}

/* The Dirichlet problem of Eqs. 6-7 for charge density rho (NULL: zero) with
 * phi = phig on the grain and phi = phiout on the outer surface. */
static void solve_dirichlet(or_sim* s, const double* rho, double phig, double phiout, double* phi) {
  double* b = (double*)malloc(sizeof(double) * (size_t)s->nu);
  for (int i = 1; i < s->c.n1; ++i)
    for (int j = 0; j < s->N2; ++j) b[UIDX(s, i, j)] = row_rhs(s, i, j, rho ? rho[i * s->N2 + j] : 0.0, phig, phiout);
  lu_solve(s, s->band, s->piv, b);
  for (int j = 0; j < s->N2; ++j) {
    phi[j] = phig;
    phi[s->c.n1 * s->N2 + j] = phiout;
  }
  for (int i = 1; i < s->c.n1; ++i)
    for (int j = 0; j < s->N2; ++j) phi[i * s->N2 + j] = b[UIDX(s, i, j)];
  free(b);
}

/* Boltzmann electrons (the paper's Sec. 2 option; n0 = 1, Te = 1 units, with
 * the sign of a negative electron charge): Eq. 6 becomes
 * Delta phi = -(rho_i - exp(phi)), rho_i the particles' charge density, with
 * the same Dirichlet values.  Solved by Newton's method: each iteration
 * solves (L - diag(exp(phi_k))) phi_{k+1} = -rho_i + exp(phi_k)(1 - phi_k)
 * (plus the Dirichlet terms) by banded LU, until the largest update is below
 * 1e-13 (1 + max |phi|).  phi holds the start on entry.  Returns the
 * iterations, or -1 without convergence in 100. */
static int solve_boltzmann(or_sim* s, const double* rho, double* phi) {
  size_t nn = (size_t)s->N1 * s->N2;
  double* band = (double*)malloc(sizeof(double) * (size_t)s->ld * s->nu);
  int* piv = (int*)malloc(sizeof(int) * (size_t)s->nu);
  double* shift = (double*)calloc(nn, sizeof(double));
  double* b = (double*)malloc(sizeof(double) * (size_t)s->nu);
  int it, ok = 0;
  for (int j = 0; j < s->N2; ++j) {
    phi[j] = s->c.phi_g;
    phi[s->c.n1 * s->N2 + j] = s->c.phi_out;
  }
  for (it = 1; it <= 100; ++it) {
    for (int i = 1; i < s->c.n1; ++i)
      for (int j = 0; j < s->N2; ++j) {
        double p = phi[i * s->N2 + j], e = exp(p);
        shift[i * s->N2 + j] = -e;
        b[UIDX(s, i, j)] = row_rhs(s, i, j, rho[i * s->N2 + j], s->c.phi_g, s->c.phi_out) + e * (1.0 - p);
      }
    assemble_factor(s, shift, band, piv);
    lu_solve(s, band, piv, b);
    double dmax = 0.0, pmax = 0.0;
    for (int i = 1; i < s->c.n1; ++i)
      for (int j = 0; j < s->N2; ++j) {
        double* p = &phi[i * s->N2 + j];
        double nw = b[UIDX(s, i, j)];
        if (fabs(nw - *p) > dmax) dmax = fabs(nw - *p);
        if (fabs(nw) > pmax) pmax = fabs(nw);
        *p = nw;
      }
    if (dmax <= 1e-13 * (1.0 + pmax)) { ok = 1; break; }
  }
  free(band); free(piv); free(shift); free(b);
  return ok ? it : -1;
}

/* out = L phi at every node where the operator has a row: the interior rows
 * of Eq. 7's differences (boundary rows 0), or, with OR_FE, every node's
 * -(K phi)_a / V_a including the boundary rows (their sum weighted by V is
 * the total flux, zero for any phi). */
void or_apply_operator(const or_sim* s, const double* phi, double* out) {
  size_t nn = (size_t)s->N1 * s->N2;
  memset(out, 0, sizeof(double) * nn);
  if (s->c.flags & OR_FE) {
    for (int ci = 0; ci < s->c.n1; ++ci)
      for (int cj = 0; cj < s->c.n2; ++cj) {
        double K[4][4];
        fe_cell(s, ci, cj, K);
        for (int p = 0; p < 4; ++p) {
          size_t a = (size_t)(ci + (p & 1)) * s->N2 + cj + (p >> 1);
          for (int q = 0; q < 4; ++q) out[a] -= K[p][q] * phi[(size_t)(ci + (q & 1)) * s->N2 + cj + (q >> 1)];
        }
      }
    for (size_t a = 0; a < nn; ++a) out[a] /= s->V[a];
    return;
  }
  for (int i = 1; i < s->c.n1; ++i)
    for (int j = 0; j < s->N2; ++j) {
      double w[3][5], acc = 0.0;
      stencil(s, i, j, w);
      for (int di = -1; di <= 1; ++di)
        for (int dj = -2; dj <= 2; ++dj) {
          int jj = j + dj;
          if (w[di + 1][dj + 2] != 0.0 && jj >= 0 && jj < s->N2) acc += w[di + 1][dj + 2] * phi[(i + di) * s->N2 + jj];
        }
      out[i * s->N2 + j] = acc;
    }
}

/* The configured boundary values (phi_g, phi_out); with Boltzmann electrons
 * the nonlinear problem, from phi = 0 inside. */
int or_solve(or_sim* s, const double* rho_in, double* phi_out) {
  if (!s->band) return -1;
  const double* rho = rho_in ? rho_in : s->rho;
  double* phi = phi_out ? phi_out : s->phi;
  if (s->c.flags & OR_BOLTZMANN) {
    memset(phi, 0, sizeof(double) * (size_t)s->N1 * s->N2);
    return solve_boltzmann(s, rho, phi) > 0 ? 0 : -2;
  }
  solve_dirichlet(s, rho, s->c.phi_g, s->c.phi_out, phi);
  return 0;
}

/* The linear problem of Eqs. 6-7 whatever the electron model. */
int or_solve_linear(or_sim* s, const double* rho, double* phi_out) {
  if (!s->band) return -1;
  solve_dirichlet(s, rho, s->c.phi_g, s->c.phi_out, phi_out);
  return 0;
}

/* Replace the simulation's potential by the caller's node values (pin tests:
 * the gather, the push in a field and the surface quantities are then
 * checked on potentials whose gradient and surface integrals are known in
 * closed form). */
void or_set_phi(or_sim* s, const double* phi) {
  memcpy(s->phi, phi, sizeof(double) * (size_t)s->N1 * s->N2);
}

/* Node gradients dphi/dx1, dphi/dx2 (Sec. 2 after Eq. 10: derivatives taken
 * numerically at the grid nodes): central in the interior, one-sided second
 * order on the four edges. */
void or_gradients(or_sim* s) {
  int n1 = s->c.n1, n2 = s->c.n2, N2 = s->N2;
  const double* p = s->phi;
  for (int i = 0; i <= n1; ++i)
    for (int j = 0; j <= n2; ++j) {
      double g1, g2;
      if (i == 0) g1 = (-3.0 * p[j] + 4.0 * p[N2 + j] - p[2 * N2 + j]) / (2.0 * s->h1);
      else if (i == n1) g1 = (3.0 * p[n1 * N2 + j] - 4.0 * p[(n1 - 1) * N2 + j] + p[(n1 - 2) * N2 + j]) / (2.0 * s->h1);
      else g1 = (p[(i + 1) * N2 + j] - p[(i - 1) * N2 + j]) / (2.0 * s->h1);
      int b = i * N2;
      if (j == 0) g2 = (-3.0 * p[b] + 4.0 * p[b + 1] - p[b + 2]) / (2.0 * s->h2);
      else if (j == n2) g2 = (3.0 * p[b + n2] - 4.0 * p[b + n2 - 1] + p[b + n2 - 2]) / (2.0 * s->h2);
      else g2 = (p[b + j + 1] - p[b + j - 1]) / (2.0 * s->h2);
      s->G1[b + j] = g1;
      s->G2[b + j] = g2;
    }
}

/* Surface charge and electric force on the grain (Sec. 2 after Eq. 10):
 * E_n = -(dphi/dx1)|grad x1| on x1 = -1 (phi is constant along the surface),
 * sigma = eps0 E_n, F_Z = surface integral of (sigma^2 / 2 eps0) n_Z dA with
 * dA of Eq. 4; trapezoid rule over the x2 nodes. */
void or_surface(or_sim* s, double* En_out, double* Q, double* FZ) {
  double q = 0.0, fz = 0.0;
  for (int j = 0; j <= s->c.n2; ++j) {
    double x2 = x2_node(s, j);
    double r = r_grain(s->c.alpha, x2);
    double m[4];
    or_metric(s->c.alpha, r, x2, m);
    double g = sqrt(m[0] * m[0] + m[1] * m[1]);
    double En = -s->G1[j] * g;
    double nZ = m[1] / g;
    double dA = or_dA_dx2(s->c.alpha, -1.0, x2);
    double tw = (j == 0 || j == s->c.n2) ? 0.5 * s->h2 : s->h2;
    if (En_out) En_out[j] = En;
    q += tw * En * dA;
    fz += tw * 0.5 * En * En * nZ * dA;
  }
  *Q = q;
  *FZ = fz;
}

/* The grain charge Q of or_surface for an arbitrary potential phi (its rows
 * i = 0..2 enter through the one-sided dphi/dx1 on the grain). */
static double grain_charge(const or_sim* s, const double* phi) {
  int N2 = s->N2;
  double q = 0.0;
  for (int j = 0; j <= s->c.n2; ++j) {
    double x2 = x2_node(s, j);
    double m[4];
    or_metric(s->c.alpha, r_grain(s->c.alpha, x2), x2, m);
    double g1 = (-3.0 * phi[j] + 4.0 * phi[N2 + j] - phi[2 * N2 + j]) / (2.0 * s->h1);
    double En = -g1 * sqrt(m[0] * m[0] + m[1] * m[1]);
    double tw = (j == 0 || j == s->c.n2) ? 0.5 * s->h2 : s->h2;
    q += tw * En * or_dA_dx2(s->c.alpha, -1.0, x2);
  }
  return q;
}

/* ------------------------------------------------------------------------ */
/* Particles.                                                               */
/* ------------------------------------------------------------------------ */
static void sp_reserve(species_state* p, int64_t need) {
  if (need <= p->cap) return;
  int64_t nc = p->cap ? p->cap : 1024;
  while (nc < need) nc *= 2;
  p->x1 = (double*)realloc(p->x1, sizeof(double) * nc);
  p->x2 = (double*)realloc(p->x2, sizeof(double) * nc);
  p->vR = (double*)realloc(p->vR, sizeof(double) * nc);
  p->vZ = (double*)realloc(p->vZ, sizeof(double) * nc);
  p->vT = (double*)realloc(p->vT, sizeof(double) * nc);
  p->id = (int64_t*)realloc(p->id, sizeof(int64_t) * nc);
  p->cap = nc;
}

static void sp_append(species_state* p, double x1, double x2, double vR, double vZ, double vT) {
  sp_reserve(p, p->n + 1);
  int64_t k = p->n++;
  p->x1[k] = x1; p->x2[k] = x2; p->vR[k] = vR; p->vZ[k] = vZ; p->vT[k] = vT;
  p->id[k] = p->next_id++;
}

/* Philox counter of draw g for species sp: (g_lo, g_hi, kind, inst<<16 | sp<<8 | block). */
static void draw(const or_sim* s, int sp, int64_t g, uint32_t kind, uint32_t block, double u[4]) {
  uint32_t ctr[4] = {(uint32_t)((uint64_t)g & 0xffffffffu), (uint32_t)((uint64_t)g >> 32), kind,
                     ((uint32_t)s->c.instance << 16) | ((uint32_t)sp << 8) | block};
  uint32_t key[2] = {(uint32_t)(s->c.seed & 0xffffffffu), (uint32_t)(s->c.seed >> 32)};
  uint32_t o[4];
  or_philox4x32(ctr, key, o);
  for (int k = 0; k < 4; ++k) u[k] = u01(o[k]);
}

/* Initial volume load: positions uniform in physical volume (Eq. 5 integrated
 * along x1: x2 from the inverse CDF of r_out^3 - r_g^3, then r by inverting the
 * r^3 cumulative), velocities Maxwellian at T_s (Sec. 1, "unperturbed
 * Maxwellian with a prescribed particle density and temperature"). */
int or_load_volume(or_sim* s, int spi, int64_t n) {
  species_state* p = &s->sp[spi];
  double vth = sqrt(s->c.sp[spi].T / s->c.sp[spi].m);
  for (int64_t k = 0; k < n; ++k) {
    int64_t g = p->draws + k;
    double a[4], b[4];
    draw(s, spi, g, 1u, 0u, a);
    draw(s, spi, g, 1u, 1u, b);
    double x2 = sample_table(s->cdf_vol, a[0]);
    double rg = r_grain(s->c.alpha, x2), ro = or_r_of(s->c.alpha, s->c.x1_out, x2);
    double r = cbrt(rg * rg * rg + a[1] * (ro * ro * ro - rg * rg * rg));
    double z0, z1, z2, z3;
    box_muller(a[2], a[3], &z0, &z1);
    box_muller(b[0], b[1], &z2, &z3);
    sp_append(p, or_x1_of(s->c.alpha, r, x2), x2, vth * z0, vth * z1, vth * z2);
  }
  p->draws += n;
  p->loaded += n;
  return 0;
}

int or_add_particles(or_sim* s, int spi, int64_t n, const double* st) {
  species_state* p = &s->sp[spi];
  for (int64_t k = 0; k < n; ++k)
    sp_append(p, st[5 * k], st[5 * k + 1], st[5 * k + 2], st[5 * k + 3], st[5 * k + 4]);
  p->loaded += n;
  return 0;
}

/* Cell and bilinear fractions of a point; the same weights serve charge
 * weighing and field interpolation (Sec. 1).  Under a decision tape the cell
 * is recorded, or replayed with the fractions left unclamped, so that a
 * replayed run's weights are the same bilinear functions of the position
 * (the frozen-decision map is then smooth in the parameters). */
static void locate(or_sim* s, double x1, double x2, int* i, int* j, double* f1, double* f2) {
  double u1 = (x1 + 1.0) / s->h1, u2 = (x2 + 1.0) / s->h2;
  int a = (int)floor(u1), b = (int)floor(u2);
  if (a < 0) a = 0;
  if (a > s->c.n1 - 1) a = s->c.n1 - 1;
  if (b < 0) b = 0;
  if (b > s->c.n2 - 1) b = s->c.n2 - 1;
  if (s->tape_mode != OR_TAPE_OFF) {
    int packed = tape_int(s, a * s->N2 + b);
    a = packed / s->N2;
    b = packed % s->N2;
  }
  double g1 = u1 - a, g2 = u2 - b;
  if (s->tape_mode != OR_TAPE_REPLAY) {
    if (g1 < 0.0) g1 = 0.0;
    if (g1 > 1.0) g1 = 1.0;
    if (g2 < 0.0) g2 = 0.0;
    if (g2 > 1.0) g2 = 1.0;
  }
  *i = a; *j = b; *f1 = g1; *f2 = g2;
}

/* Charge weighing (Sec. 1, Eq. 5): rho_ij = sum_s q_s w_s sum_p S_ij(p) / V_ij. */
int or_deposit(or_sim* s) {
  int N2 = s->N2;
  size_t nn = (size_t)s->N1 * N2;
  memset(s->rho, 0, sizeof(double) * nn);
  for (int spi = 0; spi < s->c.n_species; ++spi) {
    species_state* p = &s->sp[spi];
    double qw = s->c.sp[spi].q * s->w[spi];
    for (int64_t k = 0; k < p->n; ++k) {
      int i, j;
      double f1, f2;
      locate(s, p->x1[k], p->x2[k], &i, &j, &f1, &f2);
      s->rho[i * N2 + j] += qw * (1.0 - f1) * (1.0 - f2);
      s->rho[(i + 1) * N2 + j] += qw * f1 * (1.0 - f2);
      s->rho[i * N2 + j + 1] += qw * (1.0 - f1) * f2;
      s->rho[(i + 1) * N2 + j + 1] += qw * f1 * f2;
    }
  }
  for (size_t k = 0; k < nn; ++k) s->rho[k] /= s->V[k];
  return 0;
}

/* Deposit of one tally event at the grain (Sec. 1: charge, momentum, angular
 * momentum and energy are transferred locally at the point of impact). */
static void tally(or_sim* s, int spi, double R, double Z, double vR, double vZ, double vT, double dt_chord) {
  /* Impact point by bisection on the straight chord of this step, in the local
   * Cartesian frame (x = R-hat, y = Theta-hat, z = Z) of the start point. */
  double lo = 0.0, hi = 1.0;
  for (int it = 0; it < BISECT_IT; ++it) {
    double mid = 0.5 * (lo + hi);
    double px = R + vR * dt_chord * mid, py = vT * dt_chord * mid, pz = Z + vZ * dt_chord * mid;
    double rr = sqrt(px * px + py * py + pz * pz);
    if (rr < r_grain(s->c.alpha, pz / rr)) hi = mid; else lo = mid;
  }
  double sm = 0.5 * (lo + hi);
  double px = R + vR * dt_chord * sm, py = vT * dt_chord * sm, pz = Z + vZ * dt_chord * sm;
  double Ri = sqrt(px * px + py * py);
  double ri = sqrt(Ri * Ri + pz * pz);
  double x2i = pz / ri;
  double c = 1.0, sn = 0.0;
  if (Ri > 0.0) { c = px / Ri; sn = py / Ri; }
  double vRi = c * vR + sn * vT;
  int bin = (int)floor((x2i + 1.0) / s->h2);
  if (bin < 0) bin = 0;
  if (bin > s->c.n2 - 1) bin = s->c.n2 - 1;
  double q = s->c.sp[spi].q, m = s->c.sp[spi].m, w = s->w[spi];
  double ek = 0.5 * m * (vR * vR + vZ * vZ + vT * vT) * w;
  double eb = q > 0.0 ? s->c.e_bind_ion * w : 0.0;
  double ev[OR_NT] = {1.0, q * w, m * vRi * w, m * vZ * w, m * R * vT * w, ek, ek + eb};
  double* b = s->bins + ((size_t)spi * s->c.n2 + bin) * OR_NT;
  for (int k = 0; k < OR_NT; ++k) b[k] += ev[k];
  s->step_tally[0] += q * w;
  s->step_tally[1] += m * vZ * w;
  s->step_tally[2] += m * R * vT * w;
  s->step_tally[3] += ek + eb;
  s->step_tally[4] += 1.0;
}

/* One particle over one step: field gather (Eq. 10), Boris push of Eq. 9,
 * straight chord in the local Cartesian frame, rotation back to the (R, Z)
 * half plane, new (x1, x2) by Eq. 2.  Returns 0 alive, 1 absorbed, 2 escaped.
 *
 * Reading of "explicit leapfrog" (Sec. 2): the standard time-centred Boris
 * scheme.  The Lorentz term of Eq. 9 (E_R - V_Theta B, +V_R B) is the force
 * of a field B_vec = -B z-hat; the V_Theta^2/R and -V_R V_Theta/R terms of
 * Eq. 9 are produced exactly by moving on the Cartesian chord and rotating the
 * velocity back into the meridional plane. */
static int push_one(or_sim* s, int spi, int64_t k) {
  species_state* p = &s->sp[spi];
  double al = s->c.alpha, dt = s->c.dt;
  double x1 = p->x1[k], x2 = p->x2[k];
  double r = or_r_of(al, x1, x2);
  double sn = sqrt((1.0 - x2) * (1.0 + x2));
  double R = r * sn, Z = r * x2;
  /* gather */
  int i, j;
  double f1, f2;
  locate(s, x1, x2, &i, &j, &f1, &f2);
  int N2 = s->N2;
  int n00 = i * N2 + j, n10 = (i + 1) * N2 + j, n01 = i * N2 + j + 1, n11 = (i + 1) * N2 + j + 1;
  double w00 = (1.0 - f1) * (1.0 - f2), w10 = f1 * (1.0 - f2), w01 = (1.0 - f1) * f2, w11 = f1 * f2;
  double g1 = w00 * s->G1[n00] + w10 * s->G1[n10] + w01 * s->G1[n01] + w11 * s->G1[n11];
  double g2 = w00 * s->G2[n00] + w10 * s->G2[n10] + w01 * s->G2[n01] + w11 * s->G2[n11];
  double m[4];
  or_metric(al, r, x2, m);
  double ER = -(m[0] * g1 + m[2] * g2);
  double EZ = -(m[1] * g1 + m[3] * g2);
  /* Boris, local frame (x, y, z) = (R-hat, Theta-hat, Z-hat) */
  double qm = s->c.sp[spi].q / s->c.sp[spi].m;
  double h = 0.5 * qm * dt;
  double vx = p->vR[k] + h * ER, vy = p->vT[k], vz = p->vZ[k] + h * EZ;
  double tz = h * (-s->c.B);
  double sz = 2.0 * tz / (1.0 + tz * tz);
  double px_ = vx + vy * tz, py_ = vy - vx * tz; /* v' = v- + v- x t */
  vx = vx + py_ * sz;                            /* v+ = v- + v' x s */
  vy = vy - px_ * sz;
  vx = vx + h * ER;
  vz = vz + h * EZ;
  /* chord and rotation */
  double X = R + vx * dt, Y = vy * dt, Zn = Z + vz * dt;
  double Rn = sqrt(X * X + Y * Y);
  double c = 1.0, s_ = 0.0;
  if (Rn > 0.0) { c = X / Rn; s_ = Y / Rn; }
  double vRn = c * vx + s_ * vy, vTn = -s_ * vx + c * vy;
  double rn = sqrt(Rn * Rn + Zn * Zn);
  double x2n = Zn / rn;
  double x1n = or_x1_of(al, rn, x2n);
  double tau = dt; /* chord time up to a point inside the grain */
  int st = rn < r_grain(al, x2n) ? 1 : 0;
  if (!st && (s->c.flags & OR_CHORD)) {
    double se = chord_entry(al, R, Z, vx * dt, vy * dt, vz * dt);
    if (se > 0.0) {
      st = 1;
      tau = dt * se;
    }
  }
  if (!st && x1n > s->c.x1_out) st = 2;
  st = tape_status(s, st);
  if (st == 1) {
    tally(s, spi, R, Z, vx, vz, vy, tau);
    return 1;
  }
  if (st == 2) return 2;
  p->x1[k] = x1n; p->x2[k] = x2n; p->vR[k] = vRn; p->vZ[k] = vz; p->vT[k] = vTn;
  return 0;
}

static void compact_push(or_sim* s) {
  for (int spi = 0; spi < s->c.n_species; ++spi) {
    species_state* p = &s->sp[spi];
    int64_t wpos = 0;
    for (int64_t k = 0; k < p->n; ++k) {
      int st = push_one(s, spi, k);
      if (st == 1) { p->absorbed++; continue; }
      if (st == 2) { p->escaped++; continue; }
      if (wpos != k) {
        p->x1[wpos] = p->x1[k]; p->x2[wpos] = p->x2[k]; p->vR[wpos] = p->vR[k];
        p->vZ[wpos] = p->vZ[k]; p->vT[wpos] = p->vT[k]; p->id[wpos] = p->id[k];
      }
      ++wpos;
    }
    p->n = wpos;
  }
}

/* Surface injection (Sec. 1, Eq. 4): per step lam_s = Gamma_s A_out dt / w_s,
 * Gamma_s = n0 sqrt(T_s / 2 pi m_s) (one-sided Maxwellian flux); the integer
 * count is the floor of a running fractional carry (reading: the paper does
 * not say whether the count is random).  x2 from the inverse CDF of Eq. 4 at
 * x1_out; velocity: flux-weighted half-Maxwellian along the inward normal
 * -grad x1/|grad x1|, Maxwellian along the meridional tangent and Theta; free
 * flight for a uniform fraction of dt, then the boundary tests. */
static void inject(or_sim* s) {
  double al = s->c.alpha;
  for (int spi = 0; spi < s->c.n_species; ++spi) {
    species_state* p = &s->sp[spi];
    p->carry += s->lam[spi];
    int64_t nk = (int64_t)floor(p->carry);
    p->carry -= (double)nk;
    nk = tape_count(s, nk);
    double vth = sqrt(s->c.sp[spi].T / s->c.sp[spi].m);
    for (int64_t k = 0; k < nk; ++k) {
      int64_t g = p->draws + k;
      double a[4], b[4];
      draw(s, spi, g, 2u, 0u, a);
      draw(s, spi, g, 2u, 1u, b);
      double x2 = sample_table_in(s, s->cdf_surf, a[0]);
      double vn = vth * sqrt(-2.0 * log(a[1]));
      double z0, z1;
      box_muller(a[2], a[3], &z0, &z1);
      double vt = vth * z0, vth_ = vth * z1;
      double tau = b[0] * s->c.dt;
      double r = or_r_of(al, s->c.x1_out, x2);
      double sn = sqrt((1.0 - x2) * (1.0 + x2));
      double R = r * sn, Z = r * x2;
      double m[4];
      or_metric(al, r, x2, m);
      double gn = sqrt(m[0] * m[0] + m[1] * m[1]);
      double nR = -m[0] / gn, nZ = -m[1] / gn; /* inward normal */
      double tR = nZ, tZ = -nR;                /* meridional tangent */
      double vx = vn * nR + vt * tR, vz = vn * nZ + vt * tZ, vy = vth_;
      double X = R + vx * tau, Y = vy * tau, Zn = Z + vz * tau;
      double Rn = sqrt(X * X + Y * Y);
      double c = 1.0, s_ = 0.0;
      if (Rn > 0.0) { c = X / Rn; s_ = Y / Rn; }
      double rn = sqrt(Rn * Rn + Zn * Zn);
      double x2n = Zn / rn;
      double x1n = or_x1_of(al, rn, x2n);
      double tau_in = tau; /* flight time up to a point inside the grain */
      int st = rn < r_grain(al, x2n) ? 1 : 0;
      if (!st && (s->c.flags & OR_CHORD)) {
        double se = chord_entry(al, R, Z, vx * tau, vy * tau, vz * tau);
        if (se > 0.0) {
          st = 1;
          tau_in = tau * se;
        }
      }
      if (!st && x1n > s->c.x1_out) st = 2;
      st = tape_status(s, st);
      if (st == 1) {
        tally(s, spi, R, Z, vx, vz, vy, tau_in);
        p->absorbed++;
        continue;
      }
      if (st == 2) { p->escaped++; continue; }
      sp_append(p, x1n, x2n, c * vx + s_ * vy, vz, -s_ * vx + c * vy);
    }
    p->draws += nk;
    p->injected += nk;
  }
}

static void record_history(or_sim* s) {
  if (s->hist_n == s->hist_cap) {
    s->hist_cap = s->hist_cap ? 2 * s->hist_cap : 256;
    s->hist = (double*)realloc(s->hist, sizeof(double) * OR_NH * s->hist_cap);
  }
  double* h = s->hist + OR_NH * s->hist_n++;
  double dt = s->c.dt;
  h[0] = (s->step + 1) * dt;
  h[1] = s->step_tally[0] / dt;
  h[2] = s->step_tally[1] / dt;
  h[3] = s->FZ;
  h[4] = s->step_tally[2] / dt;
  h[5] = s->step_tally[3] / dt;
  h[6] = s->Q;
  h[7] = (double)s->sp[0].n;
  h[8] = s->c.n_species > 1 ? (double)s->sp[1].n : 0.0;
  h[9] = s->step_tally[4];
  h[10] = s->phig;
}

static void field_phase(or_sim* s) {
  size_t nn = (size_t)s->N1 * s->N2;
  or_deposit(s);
  if (s->c.flags & OR_NO_FIELD) {
    memset(s->phi, 0, sizeof(double) * nn);
    memset(s->G1, 0, sizeof(double) * nn);
    memset(s->G2, 0, sizeof(double) * nn);
    s->Q = 0.0;
    s->FZ = 0.0;
    return;
  }
  if (s->c.flags & OR_FLOATING) {
    /* Isolated grain (an option; the paper holds phi_g fixed, Sec. 1): the
     * grain is an equipotential whose charge is what it has collected.  The
     * problem is linear, so phi = phi_0 + phi_g phi_vac, with phi_0 the
     * solution for this rho with the grain at 0 and phi_vac the vacuum field
     * of a grain at 1 (outer boundary at 0); phi_g follows from
     * Q(phi) = Q_grain, Q being linear in phi.  The first step fixes
     * Q_grain as the charge that holds the grain at the configured phi_g. */
    size_t nn = (size_t)s->N1 * s->N2;
    solve_dirichlet(s, s->rho, 0.0, s->c.phi_out, s->phi);
    double q0 = grain_charge(s, s->phi);
    if (!s->qg_set) {
      s->Qg = q0 + s->c.phi_g * s->C_vac;
      s->qg_set = 1;
    }
    s->phig = (s->Qg - q0) / s->C_vac;
    for (size_t k = 0; k < nn; ++k) s->phi[k] += s->phig * s->phi_vac[k];
  } else if (s->c.flags & OR_BOLTZMANN) {
    /* Newton from the previous step's potential */
    s->newton_its = solve_boltzmann(s, s->rho, s->phi);
  } else {
    or_solve(s, NULL, NULL);
  }
  or_gradients(s);
  or_surface(s, NULL, &s->Q, &s->FZ);
}

/* Step order: deposit(x^n) -> Poisson -> node gradients -> gather + push ->
 * absorb -> escape -> inject (Sec. 1 and Sec. 2). */
int or_step(or_sim* s, int n_steps) {
  for (int it = 0; it < n_steps; ++it) {
    field_phase(s);
    memset(s->step_tally, 0, sizeof(s->step_tally));
    compact_push(s);
    if (!(s->c.flags & OR_NO_INJECT)) inject(s);
    if (s->c.flags & OR_BOLTZMANN) {
      /* Boltzmann electrons reach the grain as the one-sided flux of a
       * Maxwellian of density n0 exp(phi_g) at the surface (Te = me = 1):
       * exp(phi_g) sqrt(1 / 2 pi) per unit area and time, charge -1 each */
      s->step_tally[0] -= exp(s->c.phi_g) * sqrt(1.0 / (2.0 * OR_PI)) * s->A_grain * s->c.dt;
    }
    if (s->c.flags & OR_FLOATING) s->Qg += s->step_tally[0]; /* charge collected this step */
    record_history(s);
    s->step++;
  }
  return 0;
}

int or_push_only(or_sim* s) {
  memset(s->step_tally, 0, sizeof(s->step_tally));
  compact_push(s);
  return 0;
}

or_sim* or_create(const or_config* cfg) {
  if (cfg->n1 < 2 || cfg->n2 < 2 || cfg->n_species < 1 || cfg->n_species > 2) return NULL;
  if (!(cfg->x1_out > -1.0 && cfg->x1_out < 0.0) || !(fabs(cfg->alpha) < 0.245)) return NULL;
  or_sim* s = (or_sim*)calloc(1, sizeof(or_sim));
  s->c = *cfg;
  s->N1 = cfg->n1 + 1;
  s->N2 = cfg->n2 + 1;
  s->h1 = (cfg->x1_out + 1.0) / cfg->n1;
  s->h2 = 2.0 / cfg->n2;
  size_t nn = (size_t)s->N1 * s->N2;
  s->rho = (double*)calloc(nn, sizeof(double));
  s->phi = (double*)calloc(nn, sizeof(double));
  s->G1 = (double*)calloc(nn, sizeof(double));
  s->G2 = (double*)calloc(nn, sizeof(double));
  s->V = (double*)calloc(nn, sizeof(double));
  build_volumes(s);
  build_tables(s);
  if (!(cfg->flags & OR_NO_FIELD)) build_matrix(s);
  s->phig = cfg->phi_g;
  /* an isolated grain's charge-restoring correction is a superposition,
   * which the nonlinear Boltzmann problem does not allow */
  if (((cfg->flags & (OR_FLOATING | OR_BOLTZMANN)) && (cfg->flags & OR_NO_FIELD)) ||
      ((cfg->flags & OR_FLOATING) && (cfg->flags & OR_BOLTZMANN))) {
    or_destroy(s);
    return NULL;
  }
  if (cfg->flags & OR_FLOATING) {
    s->phi_vac = (double*)calloc(nn, sizeof(double));
    solve_dirichlet(s, NULL, 1.0, 0.0, s->phi_vac);
    s->C_vac = grain_charge(s, s->phi_vac);
  }
  for (int k = 0; k < cfg->n_species; ++k) {
    s->w[k] = s->V_dom / (double)cfg->sp[k].n_init;
    double gam = sqrt(cfg->sp[k].T / (2.0 * OR_PI * cfg->sp[k].m));
    s->lam[k] = gam * s->A_out * cfg->dt / s->w[k];
  }
  s->bins = (double*)calloc((size_t)cfg->n_species * cfg->n2 * OR_NT, sizeof(double));
  return s;
}

void or_destroy(or_sim* s) {
  if (!s) return;
  for (int k = 0; k < 2; ++k) {
    species_state* p = &s->sp[k];
    free(p->x1); free(p->x2); free(p->vR); free(p->vZ); free(p->vT); free(p->id);
  }
  free(s->rho); free(s->phi); free(s->G1); free(s->G2); free(s->V);
  free(s->band); free(s->piv); free(s->bins); free(s->hist); free(s->phi_vac);
  free(s->tape_st); free(s->tape_nk); free(s->tape_ix);
  free(s);
}

int64_t or_count(const or_sim* s, int sp) { return s->sp[sp].n; }

int or_get_particles(const or_sim* s, int spi, double* st, int64_t* ids) {
  const species_state* p = &s->sp[spi];
  for (int64_t k = 0; k < p->n; ++k) {
    if (st) {
      st[5 * k] = p->x1[k]; st[5 * k + 1] = p->x2[k]; st[5 * k + 2] = p->vR[k];
      st[5 * k + 3] = p->vZ[k]; st[5 * k + 4] = p->vT[k];
    }
    if (ids) ids[k] = p->id[k];
  }
  return 0;
}

void or_get_grid(const or_sim* s, int which, double* out) {
  const double* src = which == 0 ? s->rho : which == 1 ? s->phi : which == 2 ? s->G1 : which == 3 ? s->G2 : s->V;
  memcpy(out, src, sizeof(double) * (size_t)s->N1 * s->N2);
}

void or_get_bins(const or_sim* s, double* out) {
  memcpy(out, s->bins, sizeof(double) * (size_t)s->c.n_species * s->c.n2 * OR_NT);
}

int or_newton_iterations(const or_sim* s) { return s->newton_its; }

int64_t or_get_history(const or_sim* s, double* out) {
  if (out) memcpy(out, s->hist, sizeof(double) * OR_NH * (size_t)s->hist_n);
  return s->hist_n;
}

void or_get_counts(const or_sim* s, int64_t* out) {
  for (int k = 0; k < 2; ++k) {
    const species_state* p = &s->sp[k];
    out[6 * k + 0] = p->loaded;
    out[6 * k + 1] = p->injected;
    out[6 * k + 2] = p->absorbed;
    out[6 * k + 3] = p->escaped;
    out[6 * k + 4] = p->n;
    out[6 * k + 5] = p->draws;
  }
}

void or_get_scalars(const or_sim* s, double* out) {
  out[0] = s->w[0];
  out[1] = s->w[1];
  out[2] = s->V_dom;
  out[3] = s->A_out;
  out[4] = s->A_grain;
  out[5] = s->lam[0];
  out[6] = s->lam[1];
  out[7] = s->Q;
  out[8] = s->FZ;
}

/* ---- decision tape (frozen-decision runs) ----
 * Finite-difference derivatives of a PIC window are only meaningful with the
 * discrete decisions held fixed: a particle absorbed in one run and not in a
 * neighbouring one changes a tally by a whole particle, and a particle that
 * crosses a cell boundary moves onto a different piece of the piecewise
 * bilinear weights.  A run in record mode stores every decision (fates,
 * injection counts, cells, table intervals); runs of perturbed parameters
 * replay them. */
void or_tape_mode(or_sim* s, int mode) {
  s->tape_mode = mode;
  s->tape_pos = 0;
  s->tape_nk_pos = 0;
  s->tape_ix_pos = 0;
  s->tape_short = 0;
  if (mode == OR_TAPE_RECORD) {
    s->tape_n = 0;
    s->tape_nk_n = 0;
    s->tape_ix_n = 0;
  }
}

int64_t or_tape_ix_get(const or_sim* s, int32_t* out) {
  if (out) memcpy(out, s->tape_ix, sizeof(int32_t) * (size_t)s->tape_ix_n);
  return s->tape_ix_n;
}

void or_tape_ix_set(or_sim* s, const int32_t* ix, int64_t n) {
  s->tape_ix = (int32_t*)realloc(s->tape_ix, sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  if (n > 0) memcpy(s->tape_ix, ix, sizeof(int32_t) * (size_t)n);
  s->tape_ix_n = s->tape_ix_cap = n;
  s->tape_ix_pos = 0;
}

int64_t or_tape_get(const or_sim* s, uint8_t* st, int64_t* nk, int64_t* n_nk) {
  if (st) memcpy(st, s->tape_st, (size_t)s->tape_n);
  if (nk) memcpy(nk, s->tape_nk, sizeof(int64_t) * (size_t)s->tape_nk_n);
  if (n_nk) *n_nk = s->tape_nk_n;
  return s->tape_n;
}

void or_tape_set(or_sim* s, const uint8_t* st, int64_t n, const int64_t* nk, int64_t n_nk) {
  s->tape_st = (uint8_t*)realloc(s->tape_st, (size_t)(n > 0 ? n : 1));
  if (n > 0) memcpy(s->tape_st, st, (size_t)n);
  s->tape_n = s->tape_cap = n;
  s->tape_nk = (int64_t*)realloc(s->tape_nk, sizeof(int64_t) * (size_t)(n_nk > 0 ? n_nk : 1));
  if (n_nk > 0) memcpy(s->tape_nk, nk, sizeof(int64_t) * (size_t)n_nk);
  s->tape_nk_n = s->tape_nk_cap = n_nk;
  s->tape_pos = 0;
  s->tape_nk_pos = 0;
}

int or_tape_status(const or_sim* s) { return s->tape_short ? -1 : 0; }
