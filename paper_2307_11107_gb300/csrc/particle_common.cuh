// Device helpers shared by the particle kernels of the step and of the
// sensitivity window: precision, counter-based draws, inverse-CDF sampling,
// cell location, absorption tallies and the free-slot stack.  Included
// inside namespace apic::{anonymous} by translation units compiled with
// -DAPIC_REAL=float or -DAPIC_REAL=double.
#pragma once

using Real = APIC_REAL;
constexpr bool kF64 = sizeof(Real) == 8;
constexpr int kBisect = kF64 ? 40 : 24;
constexpr int kChordSamples = 8;  // the chord option tests s = k / kChordSamples, k = 1..7

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

// Interval of a cumulative table holding t = u * cdf[kTable]: the largest lo
// with cdf[lo] <= t.  The guide table gives the first candidate (the interval
// of (floor(u * kTable) / kTable) * cdf[kTable] <= t), a short forward scan the
// rest: the same interval as a binary search, in one or two dependent loads.
__device__ __forceinline__ int table_interval(const double* cdf, const int32_t* guide, double u, double t) {
  int lo = guide[(int)(u * kTable)];
  while (lo + 1 < kTable && cdf[lo + 1] <= t) ++lo;
  return lo;
}

// Inverse of a cumulative table over x2 in [-1, 1] with linear interpolation.
__device__ Real sample_x2(const double* cdf, const int32_t* guide, Real u) {
  double t = (double)u * cdf[kTable];
  int lo = table_interval(cdf, guide, (double)u, t);
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


// Absorption event: impact point on the grain by bisection along this step's
// straight chord (local Cartesian frame x = R-hat, y = Theta-hat, z = Z of the
// start point), then the transferred charge, momentum (R at the impact
// azimuth, Z), angular momentum L_z = m R v_Theta and energy are added to the
// surface bin of the impact x2 (Sec. 1).
// Grazing orbits (APIC_CHORD_ABSORB): the step's straight chord P(s) = (R +
// s dx, s dy, Z + s dz), s in [0, 1], in the local Cartesian frame of the
// start point, may pass through the grain although its end point lies
// outside.  Returns the first of the points s = k / kChordSamples that lies
// inside the grain, or 0; chords whose closest approach to the origin stays
// beyond the grain's largest radius (1 + sqrt(1 + 4 |alpha|)) / 2 are not
// sampled.
__device__ __noinline__ Real chord_entry(Real al, Real R, Real Z, Real dx, Real dy, Real dz) {
  const Real dd = dx * dx + dy * dy + dz * dz;
  Real s0 = dd > Real(0) ? -(R * dx + Z * dz) / dd : Real(0);
  s0 = s0 < Real(0) ? Real(0) : (s0 > Real(1) ? Real(1) : s0);
  const Real px = R + s0 * dx, py = s0 * dy, pz = Z + s0 * dz;
  const Real rmax = Real(0.5) * (Real(1) + sqrt(Real(1) + Real(4) * fabs(al)));
  if (px * px + py * py + pz * pz >= rmax * rmax) return Real(0);
  for (int k = 1; k < kChordSamples; ++k) {
    const Real sk = (Real)k / (Real)kChordSamples;
    const Real qx = R + sk * dx, qy = sk * dy, qz = Z + sk * dz;
    const Real rr = sqrt(qx * qx + qy * qy + qz * qz);
    if (rr < r_grain(al, qz / rr)) return sk;
  }
  return Real(0);
}

// One tally component (value already divided by its unit) added to a bin's
// accumulator and, if given, to the step's; out of range sets the status
// word's non-finite bit.
__device__ __forceinline__ void tally_add(const DevPtrs& d, unsigned long long* bin, unsigned long long* step, double x) {
  long long v;
  if (!to_fixed(x, 1.0, &v)) {
    atomicOr(d.err, kErrNonFinite);
    return;
  }
  fixed128_add(bin, v);
  if (step) fixed128_add(step, v);
}

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
  // fixed-point sums (tally_fixed.cuh): hits exactly; momenta and L_z in
  // units of v_th, the kinetic energy in units of v_th^2 (m w applied at
  // read-back, and the binding energy and charge from the hit count)
  const double iu = 1.0 / P.tunit;
  unsigned long long* b = d.tfix + P.tfix_off + (long long)bin * kTallyBinWords;
  unsigned long long* st = d.tfix + P.tfix_off + (long long)I.n2 * kTallyBinWords;
  atomicAdd(b, 1ull);
  atomicAdd(st, 1ull);
  tally_add(d, b + 1, nullptr, (double)vRi * iu);
  tally_add(d, b + 3, st + 1, (double)vz * iu);
  tally_add(d, b + 5, st + 3, (double)R * (double)vy * iu);
  tally_add(d, b + 7, st + 5, 0.5 * ((double)vx * vx + (double)vz * vz + (double)vy * vy) * iu * iu);
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

