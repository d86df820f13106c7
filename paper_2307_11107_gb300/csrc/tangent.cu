// Sensitivity window of the APIC step: forward-mode (tangent) derivatives of
// the step (arXiv:2307.11107, Secs. 1-2) with respect to the grain shape
// alpha (Eqs. 2-5, 7), the grain potential phi_g (boundary condition of
// Eq. 6) and the magnetic field B (Eq. 9).
//
// Every particle carries the derivatives of (x1, x2, v_R, v_Z, v_Theta) along
// the three parameters; the particle kernels run the step on dual numbers
// (value + three derivatives), so the value part is the ordinary step and the
// derivative part follows it through the gather of Eq. 10, the Boris push,
// the chord and the rotation back to the meridional plane, Eq. 2, the
// absorption tallies and the surface injection of Eq. 4.  Branch decisions
// (absorbed, escaped, the injection count, the cell of a particle) are taken
// on the values and carry no derivative.  The node-side kernels form the
// right-hand sides of the tangent Poisson problems
//   L(alpha) dphi = -(d rho + dL/dalpha phi),  dphi = d phi_g on the grain,
// and the derivatives of the surface field, charge and electric force.
//
// Compiled once per particle precision (-DAPIC_REAL=double | float); the
// node-side kernels only in the double build (APIC_TANGENT_COMMON).
#include <cuda_runtime.h>

#include <cstdint>

#include "apic_internal.h"
#include "dual.cuh"
#include "geom.cuh"

#ifndef APIC_REAL
#error "compile with -DAPIC_REAL=float or -DAPIC_REAL=double"
#endif

namespace apic {
namespace {

#include "particle_common.cuh"

using D = ad::Dual<Real, kNPar>;
using D1 = ad::Dual<double, 1>;

__device__ __forceinline__ Real* tcomp(const TanPtrs& t, int p, int c) {
  return (Real*)t.ds + (long long)(5 * p + c) * t.stride;
}

__device__ __forceinline__ D load_d(const TanPtrs& t, Real v, int c, long long slot) {
  D x(v);
#pragma unroll
  for (int p = 0; p < kNPar; ++p) x.d[p] = tcomp(t, p, c)[slot];
  return x;
}

__device__ __forceinline__ void store_d(const TanPtrs& t, const D& x, int c, long long slot, void* arr) {
  ((Real*)arr)[slot] = x.v;
#pragma unroll
  for (int p = 0; p < kNPar; ++p) tcomp(t, p, c)[slot] = x.d[p];
}

// Cell of (x1, x2) and the bilinear fractions as duals; a clamped fraction
// (a point outside the grid) has zero derivative.
struct CellD {
  int i, j;
  D f1, f2;
};

__device__ __forceinline__ CellD locate_d(const Inst& I, const D& x1, const D& x2) {
  D u1 = (x1 + Real(1)) / (Real)I.h1;
  D u2 = (x2 + Real(1)) / (Real)I.h2;
  CellD c;
  c.i = (int)floor(u1.v);
  c.j = (int)floor(u2.v);
  c.i = c.i < 0 ? 0 : (c.i > I.n1 - 1 ? I.n1 - 1 : c.i);
  c.j = c.j < 0 ? 0 : (c.j > I.n2 - 1 ? I.n2 - 1 : c.j);
  c.f1 = u1 - (Real)c.i;
  c.f2 = u2 - (Real)c.j;
  if (c.f1.v < Real(0)) c.f1 = D(Real(0));
  if (c.f1.v > Real(1)) c.f1 = D(Real(1));
  if (c.f2.v < Real(0)) c.f2 = D(Real(0));
  if (c.f2.v > Real(1)) c.f2 = D(Real(1));
  return c;
}

// Node value of one gradient component with its three derivatives.
__device__ __forceinline__ D node_d(const TanPtrs& t, long long total_nodes, long long n, int comp, Real v) {
  using Real2 = typename Pair<Real>::T;
  D x(v);
#pragma unroll
  for (int p = 0; p < kNPar; ++p) {
    Real2 g = ((const Real2*)t.dG)[(long long)p * total_nodes + n];
    x.d[p] = comp == 0 ? g.x : g.y;
  }
  return x;
}

// Derivatives of the step tallies that enter the window outputs: charge
// (current), Z momentum (drag) and L_z = m R v_Theta (torque; R of the chord's
// start point, where L_z is that of the whole chord), all times w, whose
// alpha-derivative is w d ln w / d alpha.
__device__ __forceinline__ void tally_d(const TanPtrs& t, const Pop& P, const D& R, const D& vz, const D& vy) {
  double* tt = t.tally + (long long)P.inst * kNOut * kNPar;
  const double q = P.q, m = P.m, w = P.w, dl = t.dlnw[P.inst];
#pragma unroll
  for (int p = 0; p < kNPar; ++p) {
    double a = p == 0 ? dl : 0.0;
    atomicAdd(tt + 0 * kNPar + p, m * w * ((double)vz.d[p] + (double)vz.v * a));
    if (a != 0.0) atomicAdd(tt + 2 * kNPar + p, q * w * a);
    atomicAdd(tt + 3 * kNPar + p, m * w * ((double)R.d[p] * vy.v + (double)R.v * vy.d[p] + (double)R.v * vy.v * a));
  }
}

// Prefix of the populations' slot counts (one thread).
__device__ __forceinline__ void pop_prefix(const DevPtrs& d, long long* pre) {
  if (threadIdx.x == 0) {
    long long a = 0;
    for (int p = 0; p < d.n_pop; ++p) {
      pre[p] = a;
      a += d.ps[p].n;
    }
    pre[d.n_pop] = a;
  }
  __syncthreads();
}

// d rho (before the division by the node volume): sum over live particles of
// q w dW for the four cloud-in-cell corners, per parameter.  Each CTA takes a
// contiguous range of the (row-sorted) particles in chunks and adds into a
// shared-memory window of `rows` node rows of one population ([kNPar][rows]
// [win_n2 + 1] doubles), flushed to global memory when a chunk's first row or
// population leaves it; corners outside the window go to global memory.
constexpr int kTanDepItems = 8;
__global__ void __launch_bounds__(256) k_tan_deposit(DevPtrs d, TanPtrs t, int win_n2, int rows) {
  extern __shared__ double s_tw[];
  __shared__ long long s_pre[kMaxPop + 1];
  __shared__ int s_row0, s_wpop, s_newrow0, s_newpop, s_flush;
  pop_prefix(d, s_pre);
  const int WN = win_n2 + 1, plane = rows * WN;
  for (int k = threadIdx.x; k < kNPar * plane; k += blockDim.x) s_tw[k] = 0.0;
  if (threadIdx.x == 0) s_wpop = -1;
  __syncthreads();
  const long long total = s_pre[d.n_pop];
  const Real* X1 = (const Real*)d.x1;
  const Real* X2 = (const Real*)d.x2;
  const long long CH = (long long)kTanDepItems * blockDim.x;
  const long long nch = (total + CH - 1) / CH;
  const long long per = (nch + gridDim.x - 1) / gridDim.x;
  const long long cb = (long long)blockIdx.x * per, ce = cb + per < nch ? cb + per : nch;
  auto flush = [&](int wp, int row0) {
    const Inst& I = d.inst[d.pop[wp].inst];
    const int nr = I.n2 <= win_n2 ? rows : 0;
    for (int e = threadIdx.x; e < kNPar * nr * I.N2; e += blockDim.x) {
      const int p = e / (nr * I.N2), rem = e - p * nr * I.N2, r = rem / I.N2, j = rem - r * I.N2;
      double* sw = s_tw + p * plane + r * WN + j;
      if (*sw != 0.0 && row0 + r <= I.n1) {
        atomicAdd(t.drho + (long long)p * d.total_nodes + I.node_off + (long long)(row0 + r) * I.N2 + j, *sw);
        *sw = 0.0;
      }
    }
    __syncthreads();
  };
  for (long long ch = cb; ch < ce; ++ch) {
    const long long t0 = ch * CH;
    if (threadIdx.x == 0) {
      int pop = find_pop(s_pre, d.n_pop, t0), row = 0;
      for (long long q = t0; q < t0 + 64 && q < total; ++q) {
        const int pq = find_pop(s_pre, d.n_pop, q);
        const Real xq = X1[d.pop[pq].base + (q - s_pre[pq])];
        if (xq < Real(0)) {
          pop = pq;
          row = (int)floor((double)((xq + Real(1)) / (Real)d.inst[d.pop[pq].inst].h1));
          break;
        }
      }
      const int r0 = row > 0 ? row - 1 : 0;
      const bool keep = s_wpop == pop && r0 >= s_row0 && r0 + 2 < s_row0 + rows;
      s_flush = s_wpop >= 0 && !keep;
      s_newrow0 = keep ? s_row0 : r0;
      s_newpop = pop;
    }
    __syncthreads();
    if (s_flush) flush(s_wpop, s_row0);
    if (threadIdx.x == 0) {
      s_row0 = s_newrow0;
      s_wpop = s_newpop;
    }
    __syncthreads();
    const int wpop = s_wpop, row0 = s_row0;
    for (int it = 0; it < kTanDepItems; ++it) {
      const long long k = t0 + (long long)it * blockDim.x + threadIdx.x;
      if (k >= total) break;
      const int pop = find_pop(s_pre, d.n_pop, k);
      const Pop& P = d.pop[pop];
      const Inst& I = d.inst[P.inst];
      const long long slot = P.base + (k - s_pre[pop]);
      const Real x1v = X1[slot];
      if (!(x1v < Real(0))) continue;
      D x1 = load_d(t, x1v, 0, slot), x2 = load_d(t, X2[slot], 1, slot);
      CellD c = locate_d(I, x1, x2);
      D g1 = Real(1) - c.f1, g2 = Real(1) - c.f2;
      D w00 = g1 * g2, w10 = c.f1 * g2, w01 = g1 * c.f2, w11 = c.f1 * c.f2;
      const double qw = P.q * P.w;
      const int rr = c.i - row0;
      if (pop == wpop && I.n2 <= win_n2 && rr >= 0 && rr + 1 < rows) {
#pragma unroll
        for (int p = 0; p < kNPar; ++p) {
          double* sw = s_tw + p * plane + rr * WN + c.j;
          if (w00.d[p] != Real(0)) atomicAdd(sw, qw * (double)w00.d[p]);
          if (w10.d[p] != Real(0)) atomicAdd(sw + WN, qw * (double)w10.d[p]);
          if (w01.d[p] != Real(0)) atomicAdd(sw + 1, qw * (double)w01.d[p]);
          if (w11.d[p] != Real(0)) atomicAdd(sw + WN + 1, qw * (double)w11.d[p]);
        }
      } else {
        const long long n00 = I.node_off + (long long)c.i * I.N2 + c.j;
#pragma unroll
        for (int p = 0; p < kNPar; ++p) {
          double* r = t.drho + (long long)p * d.total_nodes;
          if (w00.d[p] != Real(0)) atomicAdd(r + n00, qw * (double)w00.d[p]);
          if (w10.d[p] != Real(0)) atomicAdd(r + n00 + I.N2, qw * (double)w10.d[p]);
          if (w01.d[p] != Real(0)) atomicAdd(r + n00 + 1, qw * (double)w01.d[p]);
          if (w11.d[p] != Real(0)) atomicAdd(r + n00 + I.N2 + 1, qw * (double)w11.d[p]);
        }
      }
    }
    __syncthreads();
  }
  if (s_wpop >= 0) flush(s_wpop, s_row0);
}

// One particle over one step on dual numbers: the same sequence as the step's
// push (gather of Eq. 10, Boris push with the field vector -B z-hat, straight
// chord, rotation to the meridional plane, Eq. 2), then absorption / escape
// decided on the values.
__global__ void __launch_bounds__(256) k_tan_push(DevPtrs d, TanPtrs t) {
  using Real2 = typename Pair<Real>::T;
  __shared__ long long s_pre[kMaxPop + 1];
  pop_prefix(d, s_pre);
  const long long total = s_pre[d.n_pop];
  const Real2* G = (const Real2*)d.G;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    int pop = find_pop(s_pre, d.n_pop, k);
    const Pop& P = d.pop[pop];
    const Inst& I = d.inst[P.inst];
    long long kk = k - s_pre[pop];
    long long slot = P.base + kk;
    Real x1v = ((const Real*)d.x1)[slot];
    if (!(x1v < Real(0))) continue;
    D x1 = load_d(t, x1v, 0, slot);
    D x2 = load_d(t, ((const Real*)d.x2)[slot], 1, slot);
    D vR = load_d(t, ((const Real*)d.vR)[slot], 2, slot);
    D vZ = load_d(t, ((const Real*)d.vZ)[slot], 3, slot);
    D vT = load_d(t, ((const Real*)d.vT)[slot], 4, slot);
    const D al = D::seed((Real)I.alpha, 0);
    const D B = D::seed((Real)I.B, 2);
    const Real dt = (Real)I.dt;
    D r = radius(al, x1, x2);
    D sn = sqrt((Real(1) - x2) * (Real(1) + x2));
    D R = r * sn, Z = r * x2;
    // gather: bilinear node gradients (with their derivatives), analytic metric
    CellD c = locate_d(I, x1, x2);
    long long n00 = I.node_off + (long long)c.i * I.N2 + c.j;
    long long n10 = n00 + I.N2, n01 = n00 + 1, n11 = n00 + I.N2 + 1;
    Real2 a00 = G[n00], a10 = G[n10], a01 = G[n01], a11 = G[n11];
    D w00 = (Real(1) - c.f1) * (Real(1) - c.f2), w10 = c.f1 * (Real(1) - c.f2);
    D w01 = (Real(1) - c.f1) * c.f2, w11 = c.f1 * c.f2;
    const long long tn = d.total_nodes;
    D g1 = w00 * node_d(t, tn, n00, 0, a00.x) + w10 * node_d(t, tn, n10, 0, a10.x) +
           w01 * node_d(t, tn, n01, 0, a01.x) + w11 * node_d(t, tn, n11, 0, a11.x);
    D g2 = w00 * node_d(t, tn, n00, 1, a00.y) + w10 * node_d(t, tn, n10, 1, a10.y) +
           w01 * node_d(t, tn, n01, 1, a01.y) + w11 * node_d(t, tn, n11, 1, a11.y);
    Metric<D> m = metric(al, r, x2);
    D ER = -(m.x1R * g1 + m.x2R * g2);
    D EZ = -(m.x1Z * g1 + m.x2Z * g2);
    // Boris in the local frame (R-hat, Theta-hat, Z-hat)
    const Real h = Real(0.5) * (Real)(P.q / P.m) * dt;
    D vx = vR + h * ER, vy = vT, vz = vZ + h * EZ;
    D tz = h * (-B);
    D sz = Real(2) * tz / (Real(1) + tz * tz);
    D px_ = vx + vy * tz, py_ = vy - vx * tz;
    vx = vx + py_ * sz;
    vy = vy - px_ * sz;
    vx = vx + h * ER;
    vz = vz + h * EZ;
    // chord and rotation back to the meridional half plane
    D Xc = R + vx * dt, Yc = vy * dt, Zn = Z + vz * dt;
    D Rn = sqrt(Xc * Xc + Yc * Yc);
    D cr(Real(1)), sr(Real(0));
    if (Rn.v > Real(0)) {
      cr = Xc / Rn;
      sr = Yc / Rn;
    }
    D vRn = cr * vx + sr * vy, vTn = -sr * vx + cr * vy;
    D rn = sqrt(Rn * Rn + Zn * Zn);
    D x2n = Zn / rn;
    if (rn.v < r_grain(al.v, x2n.v)) {
      absorb_tally(d, I, P, R.v, Z.v, vx.v, vz.v, vy.v, dt);
      tally_d(t, P, R, vz, vy);
      atomicAdd((unsigned long long*)&d.ps[pop].absorbed, 1ull);
      ((Real*)d.x1)[slot] = Real(2);
      push_hole(d, P, pop, kk);
      continue;
    }
    D x1n = x1_at(al, rn, x2n);
    if (x1n.v > (Real)I.x1_out) {
      atomicAdd((unsigned long long*)&d.ps[pop].escaped, 1ull);
      ((Real*)d.x1)[slot] = Real(2);
      push_hole(d, P, pop, kk);
      continue;
    }
    store_d(t, x1n, 0, slot, d.x1);
    store_d(t, x2n, 1, slot, d.x2);
    store_d(t, vRn, 2, slot, d.vR);
    store_d(t, vz, 3, slot, d.vZ);
    store_d(t, vTn, 4, slot, d.vT);
  }
}

// Surface injection on dual numbers: x2 from the inverse CDF of Eq. 4 on
// x1_out at the same random number (its alpha-derivative from the derivative
// of the table, d x2 = -(dF/dalpha) / (dF/dx2) of the interpolated table),
// normal / tangential velocity components in the frame of -grad x1, free
// flight, boundary tests; stored particles fill freed slots first.  No
// deposit here: the window deposits every particle at the start of a step.
__global__ void __launch_bounds__(256) k_tan_inject(DevPtrs d, TanPtrs t) {
  int pop = blockIdx.y;
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  PopState& S = d.ps[pop];
  const Pop& P = d.pop[pop];
  const Inst& I = d.inst[P.inst];
  if (k >= S.n_inj) return;
  uint32_t u[8];
  draws8(I, P, S.draws + k, 2u, u);
  const D al = D::seed((Real)I.alpha, 0);
  const Real dt = (Real)I.dt;
  // inverse CDF with its alpha-derivative at fixed u
  const double* cdf = d.tab + I.tab_off + (kTable + 1);
  const double* dcdf = t.dtab + I.tab_off + (kTable + 1);
  Real u0 = unit(u[0]);
  double tq = (double)u0 * cdf[kTable];
  int lo = table_interval(cdf, d.guide + I.tab_off + (kTable + 1), (double)u0, tq);
  double dlt = cdf[lo + 1] - cdf[lo];
  double f = dlt > 0.0 ? (tq - cdf[lo]) / dlt : 0.5;
  double ht = 2.0 / kTable;
  double dtq = (double)u0 * dcdf[kTable];
  double df = dlt > 0.0 ? (dtq - dcdf[lo] - f * (dcdf[lo + 1] - dcdf[lo])) / dlt : 0.0;
  D x2((Real)(-1.0 + lo * ht + f * ht));
  x2.d[0] = (Real)(df * ht);
  const Real vth = (Real)P.vth;
  Real vn = vth * sqrt(Real(-2) * log(unit(u[1])));
  Real ra = sqrt(Real(-2) * log(unit(u[2])));
  Real pa = Real(2 * kPi) * unit(u[3]);
  Real vt = vth * (ra * cos(pa)), vth_ = vth * (ra * sin(pa));
  Real tau = unit(u[4]) * dt;
  D r = radius(al, D((Real)I.x1_out), x2);
  D sn = sqrt((Real(1) - x2) * (Real(1) + x2));
  D R = r * sn, Z = r * x2;
  Metric<D> m = metric(al, r, x2);
  D gn = sqrt(m.x1R * m.x1R + m.x1Z * m.x1Z);
  D nR = -m.x1R / gn, nZ = -m.x1Z / gn;
  D tR = nZ, tZ = -nR;
  D vx = vn * nR + vt * tR, vz = vn * nZ + vt * tZ, vy(vth_);
  D Xc = R + vx * tau, Yc = vy * tau, Zn = Z + vz * tau;
  D Rn = sqrt(Xc * Xc + Yc * Yc);
  D cr(Real(1)), sr(Real(0));
  if (Rn.v > Real(0)) {
    cr = Xc / Rn;
    sr = Yc / Rn;
  }
  D rn = sqrt(Rn * Rn + Zn * Zn);
  D x2n = Zn / rn;
  if (rn.v < r_grain(al.v, x2n.v)) {
    absorb_tally(d, I, P, R.v, Z.v, vx.v, vz.v, vy.v, tau);
    tally_d(t, P, R, vz, vy);
    atomicAdd((unsigned long long*)&S.absorbed, 1ull);
    return;
  }
  D x1n = x1_at(al, rn, x2n);
  if (x1n.v > (Real)I.x1_out) {
    atomicAdd((unsigned long long*)&S.escaped, 1ull);
    return;
  }
  long long sidx = (long long)atomicAdd((unsigned long long*)&S.inj_stored, 1ull);
  long long nh = S.n_holes, n = S.n;
  long long kk = sidx < nh ? d.holes[P.base + nh - 1 - sidx] : n + (sidx - nh);
  if (kk >= P.cap) {
    atomicAdd((unsigned long long*)&S.dropped, 1ull);
    atomicOr(d.err, kErrCapacity);
    return;
  }
  long long slot = P.base + kk;
  store_d(t, x1n, 0, slot, d.x1);
  store_d(t, x2n, 1, slot, d.x2);
  store_d(t, cr * vx + sr * vy, 2, slot, d.vR);
  store_d(t, vz, 3, slot, d.vZ);
  store_d(t, -sr * vx + cr * vy, 4, slot, d.vT);
}

#ifdef APIC_TANGENT_COMMON
__device__ __forceinline__ double x2_node(const Inst& I, int j) { return j == I.n2 ? 1.0 : -1.0 + j * I.h2; }

// Deterministic block sum (fixed tree) of one double per thread; blockDim 256.
__device__ double block_sum(double v, double* sh) {
  int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (t < o) sh[t] += sh[t + o];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

// d rho = (sum q w dW) / V + [alpha] rho (d ln w - dV / V).
__global__ void __launch_bounds__(256) k_tan_rho(DevPtrs d, TanPtrs t) {
  const Inst& I = d.inst[blockIdx.y];
  const double dl = t.dlnw[blockIdx.y];
  for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes;
       nd += (long long)gridDim.x * blockDim.x) {
    long long g = I.node_off + nd;
    double V = d.V[g];
    for (int p = 0; p < kNPar; ++p) {
      double* r = t.drho + (long long)p * d.total_nodes + g;
      double v = *r / V;
      if (p == 0) v += d.rho[g] * (dl - t.dV[g] / V);
      *r = v;
    }
  }
}

// Right-hand side of tangent problem p in the scaled form of the solved
// system, b = -(d rho + [alpha] dL/dalpha phi) rscale + [phi_g] bbc_g, with
// |b|^2 partials for the convergence test; the previous step's solution of
// the same problem is the initial guess.
__global__ void __launch_bounds__(256) k_tan_b(DevPtrs d, TanPtrs t, int p, int direct) {
  __shared__ double sh[256];
  const int inst = blockIdx.y;
  const Inst& I = d.inst[inst];
  const double* phi = t.phi0 + I.node_off;
  const double* st = t.dst + (long long)kSt * I.node_off;
  double part = 0.0;
  for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes;
       nd += (long long)gridDim.x * blockDim.x) {
    int i = (int)(nd / I.N2), j = (int)(nd % I.N2);
    long long g = I.node_off + nd;
    double bv = 0.0;
    if (i > 0 && i < I.n1) {
      double rhs = t.drho[(long long)p * d.total_nodes + g];
      if (p == 0) {
        double a = 0.0;
        for (int di = -1; di <= 1; ++di)
          for (int dj = -1; dj <= 1; ++dj) {
            int jj = j + dj;
            if (jj < 0 || jj > I.n2) continue;
            a += st[(long long)st_slot(di, dj) * I.nodes + nd] * phi[(long long)(i + di) * I.N2 + jj];
          }
        double sp = st[(long long)kStPole * I.nodes + nd];
        if (j == 0) a += sp * phi[(long long)i * I.N2 + 2];
        if (j == I.n2) a += sp * phi[(long long)i * I.N2 + I.n2 - 2];
        rhs += a;
      }
      bv = -rhs * d.rscale[g] + (p == 1 ? t.bbc_g[g] : 0.0);
      if (!direct) d.phi[g] = t.dphi[(long long)p * d.total_nodes + g];
    }
    if (direct) t.bt[(long long)p * d.total_nodes + g] = bv;
    else d.b[g] = bv;
    part += bv * bv;
  }
  double tot = block_sum(part, sh);
  if (threadIdx.x == 0) d.red[((long long)inst * kNRed + (direct ? kTanSlot + p : 0)) * kRedBlocks + blockIdx.x] = tot;
}

// dphi of problem p: the solver's interior values, d phi_g on the grain row,
// zero on the outer row (phi_out is not a parameter); zero without a field.
__global__ void __launch_bounds__(256) k_tan_store(DevPtrs d, TanPtrs t, int p, int direct) {
  const Inst& I = d.inst[blockIdx.y];
  const bool nofield = (I.flags & APIC_NO_FIELD) != 0;
  for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes;
       nd += (long long)gridDim.x * blockDim.x) {
    int i = (int)(nd / I.N2);
    long long g = I.node_off + nd;
    const bool inside = i > 0 && i < I.n1;
    if (direct && inside && !nofield) continue;  // solved in place
    double v = 0.0;
    if (!nofield) {
      if (inside) v = d.phi[g];
      else if (i == 0 && p == 1) v = 1.0;
    }
    t.dphi[(long long)p * d.total_nodes + g] = v;
  }
}

// Derivatives of the grain charge Q = int E_n dA and of the electric force
// F_Z = int (E_n^2 / 2) n_Z dA, E_n = -(dphi/dx1)|grad x1| at x1 = -1
// (trapezoid over the x2 nodes, as the step): through dphi for every
// parameter and through |grad x1|, n_Z and dA of Eq. 4 for alpha.
__global__ void __launch_bounds__(256) k_tan_surface(DevPtrs d, TanPtrs t) {
  __shared__ double sh[256];
  const int inst = blockIdx.x;
  const Inst& I = d.inst[inst];
  const bool nofield = (I.flags & APIC_NO_FIELD) != 0;
  const int N2 = I.N2;
  const double* p0 = d.phi + I.node_off;
  double dq[kNPar] = {0, 0, 0}, dfz[kNPar] = {0, 0, 0};
  for (int j = threadIdx.x; j <= I.n2 && !nofield; j += blockDim.x) {
    double x2 = x2_node(I, j);
    D1 al = D1::seed(I.alpha, 0), X2(x2);
    D1 r = r_grain(al, X2);
    Metric<D1> m = metric(al, r, X2);
    D1 g = sqrt(m.x1R * m.x1R + m.x1Z * m.x1Z);
    D1 nzda = (m.x1Z / g) * area_density(al, D1(-1.0), X2);
    D1 dA = area_density(al, D1(-1.0), X2);
    double G1 = (-3.0 * p0[j] + 4.0 * p0[N2 + j] - p0[2 * N2 + j]) / (2.0 * I.h1);
    double En = -G1 * g.v;
    double tw = (j == 0 || j == I.n2) ? 0.5 * I.h2 : I.h2;
    for (int p = 0; p < kNPar; ++p) {
      const double* q = t.dphi + (long long)p * d.total_nodes + I.node_off;
      double dG1 = (-3.0 * q[j] + 4.0 * q[N2 + j] - q[2 * N2 + j]) / (2.0 * I.h1);
      double dEn = -dG1 * g.v - (p == 0 ? G1 * g.d[0] : 0.0);
      dq[p] += tw * (dEn * dA.v + (p == 0 ? En * dA.d[0] : 0.0));
      dfz[p] += tw * (En * dEn * nzda.v + (p == 0 ? 0.5 * En * En * nzda.d[0] : 0.0));
    }
  }
  double* tt = t.tally + (long long)inst * kNOut * kNPar;
  for (int p = 0; p < kNPar; ++p) {
    double a = block_sum(dfz[p], sh);
    double b = block_sum(dq[p], sh);
    if (threadIdx.x == 0) {
      tt[1 * kNPar + p] = a;
      tt[4 * kNPar + p] = b;
    }
  }
}

// Window sums of the outputs and their derivatives; runs before the step's
// own bookkeeping clears the step tallies.
__global__ void k_tan_step_end(DevPtrs d, TanPtrs t) {
  const int inst = blockIdx.x * blockDim.x + threadIdx.x;
  if (inst >= d.n_inst) return;
  const Inst& I = d.inst[inst];
  const StepState& T = d.stp[inst];
  const double dt = I.dt;
  double tl[5];
  step_tallies(d, inst, tl);
  double* v = t.vals + (long long)inst * kNOut;
  v[0] += tl[1] / dt;
  v[1] += T.FZ;
  v[2] += tl[0] / dt;
  v[3] += tl[2] / dt;
  v[4] += T.Q;
  double* tt = t.tally + (long long)inst * kNOut * kNPar;
  double* J = t.jac + (long long)inst * kNOut * kNPar;
  for (int o = 0; o < kNOut; ++o)
    for (int p = 0; p < kNPar; ++p) {
      double x = tt[o * kNPar + p];
      J[o * kNPar + p] += (o == 1 || o == 4) ? x : x / dt;
      tt[o * kNPar + p] = 0.0;
    }
}
#endif  // APIC_TANGENT_COMMON

unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

template <>
void launch_tan_deposit<Real>(const DevPtrs& d, const TanPtrs& t, int grid, int max_n2, cudaStream_t s) {
  // window: up to 8 node rows of up to 512 cells, within 48 KB of doubles
  const int win_n2 = max_n2 < 512 ? max_n2 : 512;
  int rows = 49152 / (kNPar * (win_n2 + 1) * (int)sizeof(double));
  rows = rows > 8 ? 8 : (rows < 2 ? 2 : rows);
  const int sm = kNPar * rows * (win_n2 + 1) * (int)sizeof(double);
  cudaFuncSetAttribute(k_tan_deposit, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  k_tan_deposit<<<grid, 256, sm, s>>>(d, t, win_n2, rows);
}

template <>
void launch_tan_push<Real>(const DevPtrs& d, const TanPtrs& t, int grid, cudaStream_t s) {
  k_tan_push<<<grid, 256, 0, s>>>(d, t);
}

template <>
void launch_tan_inject<Real>(const DevPtrs& d, const TanPtrs& t, long long max_inj, cudaStream_t s) {
  if (max_inj <= 0) return;
  k_tan_inject<<<dim3(blocks_for(max_inj, 256), d.n_pop), 256, 0, s>>>(d, t);
}

#ifdef APIC_TANGENT_COMMON
void launch_tan_rho(const DevPtrs& d, const TanPtrs& t, cudaStream_t s) {
  k_tan_rho<<<dim3(kRedBlocks, d.n_inst), 256, 0, s>>>(d, t);
}
void launch_tan_b(const DevPtrs& d, const TanPtrs& t, int p, int direct, cudaStream_t s) {
  k_tan_b<<<dim3(kRedBlocks, d.n_inst), 256, 0, s>>>(d, t, p, direct);
}
void launch_tan_store(const DevPtrs& d, const TanPtrs& t, int p, int direct, cudaStream_t s) {
  k_tan_store<<<dim3(kRedBlocks, d.n_inst), 256, 0, s>>>(d, t, p, direct);
}
void launch_tan_surface(const DevPtrs& d, const TanPtrs& t, cudaStream_t s) {
  k_tan_surface<<<d.n_inst, 256, 0, s>>>(d, t);
}
void launch_tan_step_end(const DevPtrs& d, const TanPtrs& t, cudaStream_t s) {
  k_tan_step_end<<<(d.n_inst + 63) / 64, 64, 0, s>>>(d, t);
}
#endif

}  // namespace apic
