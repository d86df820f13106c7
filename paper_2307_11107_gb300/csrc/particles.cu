// Particle kernels of the APIC step (arXiv:2307.11107, Secs. 1-2): volume
// load, surface injection (Eq. 4), field gather (Eq. 10) + Boris push (Eq. 9)
// + absorption tallies + escape, and charge weighing (Eq. 5) into 64-bit
// fixed-point node accumulators.
//
// This file is compiled once per particle precision: -DAPIC_REAL=double (with
// -fmad=false, the parity build) and -DAPIC_REAL=float.
#include <cuda_runtime.h>

#include <cstdint>

#include "apic_internal.h"
#include "geom.cuh"

#ifndef APIC_REAL
#error "compile with -DAPIC_REAL=float or -DAPIC_REAL=double"
#endif

namespace apic {
namespace {

using Real = APIC_REAL;
constexpr bool kF64 = sizeof(Real) == 8;
constexpr int kBisect = kF64 ? 40 : 24;
constexpr unsigned kFull = 0xffffffffu;

template <class T>
struct Pair;
template <>
struct Pair<double> {
  using T = double2;
};
template <>
struct Pair<float> {
  using T = float2;
};
using Real2 = typename Pair<Real>::T;

__device__ __forceinline__ Real rsqrt_(Real x) { return sqrt(x); }

// Uniform in (0, 1) from 32 random bits in the particle precision.
__device__ __forceinline__ Real unit(uint32_t u) {
  if (kF64) return (Real)unit_open(u);
  return ((Real)(u >> 8) + Real(0.5)) * Real(5.9604644775390625e-08);  // 2^-24
}

// Two counter-based blocks of draw g of population p: counter
// (g_lo, g_hi, kind, tag << 16 | species << 8 | block), key = seed.
__device__ __forceinline__ void draws8(const Inst& I, const Pop& P, long long g, uint32_t kind, uint32_t out[8]) {
  uint32_t k0 = (uint32_t)(I.seed & 0xffffffffu), k1 = (uint32_t)(I.seed >> 32);
  uint32_t tagw = ((uint32_t)I.tag << 16) | ((uint32_t)P.species << 8);
  U4 c0 = {(uint32_t)((unsigned long long)g & 0xffffffffu), (uint32_t)((unsigned long long)g >> 32), kind, tagw};
  U4 c1 = c0;
  c1.d = tagw | 1u;
  U4 a = philox10(c0, k0, k1), b = philox10(c1, k0, k1);
  out[0] = a.a; out[1] = a.b; out[2] = a.c; out[3] = a.d;
  out[4] = b.a; out[5] = b.b; out[6] = b.c; out[7] = b.d;
}

// Inverse of a cumulative table over x2 in [-1, 1] with linear interpolation.
__device__ Real sample_x2(const double* cdf, Real u) {
  double t = (double)u * cdf[kTable];
  int lo = 0, hi = kTable;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (cdf[mid] <= t) lo = mid; else hi = mid;
  }
  double dlt = cdf[lo + 1] - cdf[lo];
  double f = dlt > 0.0 ? (t - cdf[lo]) / dlt : 0.5;
  double ht = 2.0 / kTable;
  return (Real)(-1.0 + lo * ht + f * ht);
}

struct Cell {
  int i, j;
  Real f1, f2;
};

// Cell and bilinear fractions of (x1, x2); shared by weighing and gather.
__device__ __forceinline__ Cell locate(const Inst& I, Real x1, Real x2) {
  Real u1 = (x1 + Real(1)) / (Real)I.h1;
  Real u2 = (x2 + Real(1)) / (Real)I.h2;
  Cell c;
  c.i = (int)floor(u1);
  c.j = (int)floor(u2);
  c.i = c.i < 0 ? 0 : (c.i > I.n1 - 1 ? I.n1 - 1 : c.i);
  c.j = c.j < 0 ? 0 : (c.j > I.n2 - 1 ? I.n2 - 1 : c.j);
  c.f1 = u1 - (Real)c.i;
  c.f2 = u2 - (Real)c.j;
  c.f1 = c.f1 < Real(0) ? Real(0) : (c.f1 > Real(1) ? Real(1) : c.f1);
  c.f2 = c.f2 < Real(0) ? Real(0) : (c.f2 > Real(1) ? Real(1) : c.f2);
  return c;
}

struct W4 {
  unsigned long long w00, w10, w01, w11;
};

// Fixed-point cloud-in-cell weights.  FP64: each weight rounded to F bits.
// FP32: fractions quantised to F/2 bits, weights as exact integer products
// (their sum is exactly 2^F: charge is conserved to the last bit).
__device__ __forceinline__ W4 weights(const Cell& c, int F) {
  W4 w;
  if (kF64) {
    double sc = ldexp(1.0, F);
    double g1 = 1.0 - (double)c.f1, g2 = 1.0 - (double)c.f2;
    w.w00 = (unsigned long long)__double2ll_rn(g1 * g2 * sc);
    w.w10 = (unsigned long long)__double2ll_rn((double)c.f1 * g2 * sc);
    w.w01 = (unsigned long long)__double2ll_rn(g1 * (double)c.f2 * sc);
    w.w11 = (unsigned long long)__double2ll_rn((double)c.f1 * (double)c.f2 * sc);
  } else {
    int b = F >> 1;
    unsigned one = 1u << b;
    unsigned q1 = (unsigned)((float)c.f1 * (float)one), q2 = (unsigned)((float)c.f2 * (float)one);
    q1 = q1 > one ? one : q1;
    q2 = q2 > one ? one : q2;
    w.w00 = (unsigned long long)(one - q1) * (one - q2);
    w.w10 = (unsigned long long)q1 * (one - q2);
    w.w01 = (unsigned long long)(one - q1) * q2;
    w.w11 = (unsigned long long)q1 * q2;
  }
  return w;
}

// Warp-cooperative deposit: when all 32 lanes hit the same cell of the same
// population, the four corner weights are summed across the warp first and
// one lane issues the four 64-bit atomics; otherwise each lane adds its own.
// Integer addition makes the result independent of the order.
__device__ __forceinline__ void deposit_warp(unsigned long long* acc, long long key, W4 w, int N2, bool active) {
  long long k0 = __shfl_sync(kFull, key, 0);
  bool uni = __all_sync(kFull, active && key == k0);
  if (uni) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      w.w00 += __shfl_down_sync(kFull, w.w00, o);
      w.w10 += __shfl_down_sync(kFull, w.w10, o);
      w.w01 += __shfl_down_sync(kFull, w.w01, o);
      w.w11 += __shfl_down_sync(kFull, w.w11, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(acc + k0, w.w00);
      atomicAdd(acc + k0 + N2, w.w10);
      atomicAdd(acc + k0 + 1, w.w01);
      atomicAdd(acc + k0 + N2 + 1, w.w11);
    }
  } else if (active) {
    if (w.w00) atomicAdd(acc + key, w.w00);
    if (w.w10) atomicAdd(acc + key + N2, w.w10);
    if (w.w01) atomicAdd(acc + key + 1, w.w01);
    if (w.w11) atomicAdd(acc + key + N2 + 1, w.w11);
  }
}

__device__ __forceinline__ long long dep_key(const Inst& I, const Pop& P, const Cell& c) {
  return P.acc_off + (long long)c.i * I.N2 + c.j;
}

// Absorption event: impact point on the grain by bisection along this step's
// straight chord (local Cartesian frame x = R-hat, y = Theta-hat, z = Z of the
// start point), then the transferred charge, momentum (R at the impact
// azimuth, Z), angular momentum L_z = m R v_Theta and energy are added to the
// surface bin of the impact x2 (Sec. 1).
__device__ void absorb_tally(const DevPtrs& d, const Inst& I, const Pop& P, Real R, Real Z, Real vx, Real vz,
                             Real vy, Real tau) {
  Real al = (Real)I.alpha;
  Real lo = Real(0), hi = Real(1);
  for (int it = 0; it < kBisect; ++it) {
    Real mid = Real(0.5) * (lo + hi);
    Real px = R + vx * tau * mid, py = vy * tau * mid, pz = Z + vz * tau * mid;
    Real rr = sqrt(px * px + py * py + pz * pz);
    if (rr < r_grain(al, pz / rr)) hi = mid; else lo = mid;
  }
  Real sm = Real(0.5) * (lo + hi);
  Real px = R + vx * tau * sm, py = vy * tau * sm, pz = Z + vz * tau * sm;
  Real Ri = sqrt(px * px + py * py);
  Real ri = sqrt(Ri * Ri + pz * pz);
  Real x2i = pz / ri;
  Real c = Real(1), sn = Real(0);
  if (Ri > Real(0)) {
    c = px / Ri;
    sn = py / Ri;
  }
  Real vRi = c * vx + sn * vy;
  int bin = (int)floor((x2i + Real(1)) / (Real)I.h2);
  bin = bin < 0 ? 0 : (bin > I.n2 - 1 ? I.n2 - 1 : bin);
  double q = P.q, m = P.m, w = P.w;
  double ek = 0.5 * m * ((double)vx * vx + (double)vz * vz + (double)vy * vy) * w;
  double eb = q > 0.0 ? I.e_bind * w : 0.0;
  double* b = d.bins + I.bin_off + ((long long)P.species * I.n2 + bin) * kNT;
  atomicAdd(b + 0, 1.0);
  atomicAdd(b + 1, q * w);
  atomicAdd(b + 2, m * (double)vRi * w);
  atomicAdd(b + 3, m * (double)vz * w);
  atomicAdd(b + 4, m * (double)R * (double)vy * w);
  atomicAdd(b + 5, ek);
  atomicAdd(b + 6, ek + eb);
  double* st = d.stp[P.inst].tally;
  atomicAdd(st + 0, q * w);
  atomicAdd(st + 1, m * (double)vz * w);
  atomicAdd(st + 2, m * (double)R * (double)vy * w);
  atomicAdd(st + 3, ek + eb);
  atomicAdd(st + 4, 1.0);
}

__device__ __forceinline__ int find_pop(const long long* pre, int n_pop, long long t) {
  int lo = 0, hi = n_pop;  // pre[lo] <= t < pre[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (pre[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void push_hole(const DevPtrs& d, const Pop& P, int pop, long long k) {
  long long h = atomicAdd((unsigned long long*)&d.ps[pop].n_holes, 1ull);
  d.holes[P.base + h] = (int32_t)k;
}

// One full particle update for slot t of the batch (Sec. 2, Eqs. 8-10, 9).
__global__ void __launch_bounds__(256) k_push(DevPtrs d) {
  __shared__ long long s_pre[kMaxPop + 1];
  if (threadIdx.x == 0) {
    long long a = 0;
    for (int p = 0; p < d.n_pop; ++p) {
      s_pre[p] = a;
      a += d.ps[p].n;
    }
    s_pre[d.n_pop] = a;
  }
  __syncthreads();
  const long long total = s_pre[d.n_pop];
  Real* X1 = (Real*)d.x1;
  Real* X2 = (Real*)d.x2;
  Real* VR = (Real*)d.vR;
  Real* VZ = (Real*)d.vZ;
  Real* VT = (Real*)d.vT;
  const Real2* G = (const Real2*)d.G;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < total; base += stride) {
    long long t = base + (threadIdx.x & 31);
    bool active = t < total;
    int pop = active ? find_pop(s_pre, d.n_pop, t) : 0;
    const Pop& P = d.pop[pop];
    const Inst& I = d.inst[P.inst];
    long long k = active ? t - s_pre[pop] : 0;
    long long slot = P.base + k;
    Real x1 = active ? X1[slot] : Real(2);
    bool alive = active && x1 < Real(0);
    long long key = -1;
    W4 w = {0, 0, 0, 0};
    if (alive) {
      Real x2 = X2[slot], vR = VR[slot], vZ = VZ[slot], vT = VT[slot];
      Real al = (Real)I.alpha, dt = (Real)I.dt;
      Real r = radius(al, x1, x2);
      Real sn = sqrt((Real(1) - x2) * (Real(1) + x2));
      Real R = r * sn, Z = r * x2;
      // gather (Eq. 10): bilinear node gradients, analytic metric at the particle
      Cell c = locate(I, x1, x2);
      long long n00 = I.node_off + (long long)c.i * I.N2 + c.j;
      Real2 a00 = G[n00], a10 = G[n00 + I.N2], a01 = G[n00 + 1], a11 = G[n00 + I.N2 + 1];
      Real w00 = (Real(1) - c.f1) * (Real(1) - c.f2), w10 = c.f1 * (Real(1) - c.f2);
      Real w01 = (Real(1) - c.f1) * c.f2, w11 = c.f1 * c.f2;
      Real g1 = w00 * a00.x + w10 * a10.x + w01 * a01.x + w11 * a11.x;
      Real g2 = w00 * a00.y + w10 * a10.y + w01 * a01.y + w11 * a11.y;
      Metric<Real> m = metric(al, r, x2);
      Real ER = -(m.x1R * g1 + m.x2R * g2);
      Real EZ = -(m.x1Z * g1 + m.x2Z * g2);
      // Boris in the local frame (R-hat, Theta-hat, Z-hat); Eq. 9's Lorentz
      // terms are those of the field vector -B z-hat.
      Real h = Real(0.5) * (Real)(P.q / P.m) * dt;
      Real vx = vR + h * ER, vy = vT, vz = vZ + h * EZ;
      Real tz = h * (-(Real)I.B);
      Real sz = Real(2) * tz / (Real(1) + tz * tz);
      Real px_ = vx + vy * tz, py_ = vy - vx * tz;
      vx = vx + py_ * sz;
      vy = vy - px_ * sz;
      vx = vx + h * ER;
      vz = vz + h * EZ;
      // straight chord, rotation back to the meridional half plane
      Real Xc = R + vx * dt, Yc = vy * dt, Zn = Z + vz * dt;
      Real Rn = sqrt(Xc * Xc + Yc * Yc);
      Real cr = Real(1), sr = Real(0);
      if (Rn > Real(0)) {
        cr = Xc / Rn;
        sr = Yc / Rn;
      }
      Real vRn = cr * vx + sr * vy, vTn = -sr * vx + cr * vy;
      Real rn = sqrt(Rn * Rn + Zn * Zn);
      Real x2n = Zn / rn;
      if (rn < r_grain(al, x2n)) {
        absorb_tally(d, I, P, R, Z, vx, vz, vy, dt);
        atomicAdd((unsigned long long*)&d.ps[pop].absorbed, 1ull);
        X1[slot] = Real(2);
        push_hole(d, P, pop, k);
      } else {
        Real x1n = x1_at(al, rn, x2n);
        if (x1n > (Real)I.x1_out) {
          atomicAdd((unsigned long long*)&d.ps[pop].escaped, 1ull);
          X1[slot] = Real(2);
          push_hole(d, P, pop, k);
        } else {
          X1[slot] = x1n;
          X2[slot] = x2n;
          VR[slot] = vRn;
          VZ[slot] = vz;
          VT[slot] = vTn;
          Cell cn = locate(I, x1n, x2n);
          key = dep_key(I, P, cn);
          w = weights(cn, P.fbits);
        }
      }
    }
    deposit_warp(d.acc, key, w, active ? I.N2 : 1, key >= 0);
  }
}

// Deposit every live particle (after external changes to the particle set).
__global__ void __launch_bounds__(256) k_deposit_all(DevPtrs d) {
  __shared__ long long s_pre[kMaxPop + 1];
  if (threadIdx.x == 0) {
    long long a = 0;
    for (int p = 0; p < d.n_pop; ++p) {
      s_pre[p] = a;
      a += d.ps[p].n;
    }
    s_pre[d.n_pop] = a;
  }
  __syncthreads();
  const long long total = s_pre[d.n_pop];
  const Real* X1 = (const Real*)d.x1;
  const Real* X2 = (const Real*)d.x2;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < total; base += stride) {
    long long t = base + (threadIdx.x & 31);
    bool active = t < total;
    int pop = active ? find_pop(s_pre, d.n_pop, t) : 0;
    const Pop& P = d.pop[pop];
    const Inst& I = d.inst[P.inst];
    long long slot = P.base + (active ? t - s_pre[pop] : 0);
    Real x1 = active ? X1[slot] : Real(2);
    long long key = -1;
    W4 w = {0, 0, 0, 0};
    if (active && x1 < Real(0)) {
      Cell c = locate(I, x1, X2[slot]);
      key = dep_key(I, P, c);
      w = weights(c, P.fbits);
    }
    deposit_warp(d.acc, key, w, active ? I.N2 : 1, key >= 0);
  }
}

// Initial load, uniform in physical volume: x2 from the inverse CDF of
// (r_out^3 - r_g^3)(x2) (Eq. 5 integrated along x1), r by inverting the r^3
// cumulative, velocity Maxwellian at T (three Box-Muller normals).
__global__ void k_load(DevPtrs d, int pop, long long n0, long long count, long long draw0) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  const Pop& P = d.pop[pop];
  const Inst& I = d.inst[P.inst];
  uint32_t u[8];
  draws8(I, P, draw0 + k, 1u, u);
  Real al = (Real)I.alpha;
  Real x2 = sample_x2(d.tab + I.tab_off, unit(u[0]));
  Real rg = r_grain(al, x2), ro = radius(al, (Real)I.x1_out, x2);
  Real r3 = rg * rg * rg + unit(u[1]) * (ro * ro * ro - rg * rg * rg);
  Real r = cbrt(r3);
  Real ra = sqrt(Real(-2) * log(unit(u[2]))), rb = sqrt(Real(-2) * log(unit(u[4])));
  Real pa = Real(2 * kPi) * unit(u[3]), pb = Real(2 * kPi) * unit(u[5]);
  Real vth = (Real)P.vth;
  long long slot = P.base + n0 + k;
  ((Real*)d.x1)[slot] = x1_at(al, r, x2);
  ((Real*)d.x2)[slot] = x2;
  ((Real*)d.vR)[slot] = vth * (ra * cos(pa));
  ((Real*)d.vZ)[slot] = vth * (ra * sin(pa));
  ((Real*)d.vT)[slot] = vth * (rb * cos(pb));
}

__global__ void k_explicit(DevPtrs d, int pop, long long n0, long long count, const double* st) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  long long slot = d.pop[pop].base + n0 + k;
  ((Real*)d.x1)[slot] = (Real)st[5 * k + 0];
  ((Real*)d.x2)[slot] = (Real)st[5 * k + 1];
  ((Real*)d.vR)[slot] = (Real)st[5 * k + 2];
  ((Real*)d.vZ)[slot] = (Real)st[5 * k + 3];
  ((Real*)d.vT)[slot] = (Real)st[5 * k + 4];
}

// Surface injection (Sec. 1, Eq. 4): x2 from the inverse CDF of dA/dx2 on
// x1 = x1_out, flux-weighted half-Maxwellian along the inward normal
// -grad x1 / |grad x1|, Maxwellian along the meridional tangent and Theta,
// free flight for a uniform fraction of dt, then absorption / escape tests.
// Stored particles fill freed slots first, then extend the population.
__global__ void __launch_bounds__(256) k_inject(DevPtrs d) {
  int pop = blockIdx.y;
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  PopState& S = d.ps[pop];
  const Pop& P = d.pop[pop];
  const Inst& I = d.inst[P.inst];
  bool active = k < S.n_inj;
  long long key = -1;
  W4 w = {0, 0, 0, 0};
  if (active) {
    uint32_t u[8];
    draws8(I, P, S.draws + k, 2u, u);
    Real al = (Real)I.alpha, dt = (Real)I.dt;
    Real x2 = sample_x2(d.tab + I.tab_off + (kTable + 1), unit(u[0]));
    Real vth = (Real)P.vth;
    Real vn = vth * sqrt(Real(-2) * log(unit(u[1])));
    Real ra = sqrt(Real(-2) * log(unit(u[2])));
    Real pa = Real(2 * kPi) * unit(u[3]);
    Real vt = vth * (ra * cos(pa)), vth_ = vth * (ra * sin(pa));
    Real tau = unit(u[4]) * dt;
    Real r = radius(al, (Real)I.x1_out, x2);
    Real sn = sqrt((Real(1) - x2) * (Real(1) + x2));
    Real R = r * sn, Z = r * x2;
    Metric<Real> m = metric(al, r, x2);
    Real gn = sqrt(m.x1R * m.x1R + m.x1Z * m.x1Z);
    Real nR = -m.x1R / gn, nZ = -m.x1Z / gn;
    Real tR = nZ, tZ = -nR;
    Real vx = vn * nR + vt * tR, vz = vn * nZ + vt * tZ, vy = vth_;
    Real Xc = R + vx * tau, Yc = vy * tau, Zn = Z + vz * tau;
    Real Rn = sqrt(Xc * Xc + Yc * Yc);
    Real cr = Real(1), sr = Real(0);
    if (Rn > Real(0)) {
      cr = Xc / Rn;
      sr = Yc / Rn;
    }
    Real rn = sqrt(Rn * Rn + Zn * Zn);
    Real x2n = Zn / rn;
    if (rn < r_grain(al, x2n)) {
      absorb_tally(d, I, P, R, Z, vx, vz, vy, tau);
      atomicAdd((unsigned long long*)&S.absorbed, 1ull);
    } else {
      Real x1n = x1_at(al, rn, x2n);
      if (x1n > (Real)I.x1_out) {
        atomicAdd((unsigned long long*)&S.escaped, 1ull);
      } else {
        long long sidx = (long long)atomicAdd((unsigned long long*)&S.inj_stored, 1ull);
        long long nh = S.n_holes, n = S.n;
        long long kk;
        if (sidx < nh) kk = d.holes[P.base + nh - 1 - sidx];
        else kk = n + (sidx - nh);
        if (kk >= P.cap) {
          atomicAdd((unsigned long long*)&S.dropped, 1ull);
          atomicOr(d.err, kErrCapacity);
        } else {
          long long slot = P.base + kk;
          ((Real*)d.x1)[slot] = x1n;
          ((Real*)d.x2)[slot] = x2n;
          ((Real*)d.vR)[slot] = cr * vx + sr * vy;
          ((Real*)d.vZ)[slot] = vz;
          ((Real*)d.vT)[slot] = -sr * vx + cr * vy;
          Cell c = locate(I, x1n, x2n);
          key = dep_key(I, P, c);
          w = weights(c, P.fbits);
        }
      }
    }
  }
  // per-lane atomics: injected particles of a warp rarely share a cell
  if (key >= 0) {
    if (w.w00) atomicAdd(d.acc + key, w.w00);
    if (w.w10) atomicAdd(d.acc + key + I.N2, w.w10);
    if (w.w01) atomicAdd(d.acc + key + 1, w.w01);
    if (w.w11) atomicAdd(d.acc + key + I.N2 + 1, w.w11);
  }
}

// Copy every slot [0, n) of one population to FP64 rows (dead slots keep
// their sentinel x1 > 0; the host drops them).
__global__ void k_copy_out(DevPtrs d, int pop, double* out, long long n) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  long long slot = d.pop[pop].base + k;
  out[5 * k + 0] = (double)((Real*)d.x1)[slot];
  out[5 * k + 1] = (double)((Real*)d.x2)[slot];
  out[5 * k + 2] = (double)((Real*)d.vR)[slot];
  out[5 * k + 3] = (double)((Real*)d.vZ)[slot];
  out[5 * k + 4] = (double)((Real*)d.vT)[slot];
}

unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

template <>
void launch_load<Real>(const DevPtrs& d, int pop, long long n0, long long count, long long draw0, int kind,
                       cudaStream_t s) {
  (void)kind;
  if (count <= 0) return;
  k_load<<<blocks_for(count, 256), 256, 0, s>>>(d, pop, n0, count, draw0);
}

template <>
void launch_explicit<Real>(const DevPtrs& d, int pop, long long n0, long long count, const double* dstate,
                           cudaStream_t s) {
  if (count <= 0) return;
  k_explicit<<<blocks_for(count, 256), 256, 0, s>>>(d, pop, n0, count, dstate);
}

template <>
void launch_deposit_all<Real>(const DevPtrs& d, int max_grid, cudaStream_t s) {
  k_deposit_all<<<max_grid, 256, 0, s>>>(d);
}

template <>
void launch_push<Real>(const DevPtrs& d, int grid, cudaStream_t s) {
  k_push<<<grid, 256, 0, s>>>(d);
}

template <>
void launch_inject<Real>(const DevPtrs& d, long long max_inj, cudaStream_t s) {
  if (max_inj <= 0) return;
  dim3 g(blocks_for(max_inj, 256), d.n_pop);
  k_inject<<<g, 256, 0, s>>>(d);
}

template <>
void launch_gather_particles<Real>(const DevPtrs& d, int pop, double* out, long long* n_out, cudaStream_t s) {
  long long n = *n_out;
  if (n <= 0) return;
  k_copy_out<<<blocks_for(n, 256), 256, 0, s>>>(d, pop, out, n);
}

}  // namespace apic
