// Fixed-point surface tallies (Sec. 1: charge, momentum, angular momentum
// and energy transferred to the grain at the point of impact).
//
// Every absorption event adds its values to 128-bit two's-complement integer
// accumulators (two 64-bit words, low word first): integer addition is
// associative, so the sums do not depend on the order in which the events
// arrive, and a bin or a step's tally is bit-reproducible.  Each value is
// scaled by the population's unit u = v_th (momenta and L_z in m w u, energy
// in m w u^2) and rounded to kTallyBits fraction bits:
//   one event:  |value / unit| < 2^(62 - kTallyBits) = 2^26 (|v| < 11585 v_th
//               for the energy), else the event sets the status word's
//               non-finite bit and is left out;
//   rounding:   at most 2^-(kTallyBits+1) = 7.3e-12 unit per event, so a sum of
//               N events is within 7.3e-12 N unit of the exact sum of the
//               FP64 event values;
//   range:      the 128-bit sums cannot overflow (2^64 events at most).
// Hits are counted exactly; the charge is hits x q w at read-back.
#pragma once
#include <cstdint>

#ifndef __CUDACC__
#ifndef __host__
#define __host__
#endif
#ifndef __device__
#define __device__
#endif
#endif

namespace apic {

constexpr int kTallyBits = 36;
constexpr int kTallyBinWords = 9;   // per (population, bin): hits, then p_R, p_Z, L_z, E_kin as (lo, hi)
constexpr int kTallyStepWords = 7;  // per population and step: hits, then p_Z, L_z, E_kin as (lo, hi)

// Value of a 128-bit accumulator (lo, hi) times 2^-kTallyBits, rounded to FP64.
// A sum that fits in 64 signed bits (hi the sign extension of lo) converts
// with one rounding; larger ones as hi 2^64 + lo, whose relative error is a
// few units of the last place (|sum| >= 2^63 there, no cancellation).
__host__ __device__ inline double fixed128_value(unsigned long long lo, unsigned long long hi) {
  const long long h = (long long)hi, l = (long long)lo;
  const double scale = 1.4551915228366851807e-11;  // 2^-36
  if ((h == 0 && l >= 0) || (h == -1 && l < 0)) return (double)l * scale;
  return ((double)h * 18446744073709551616.0 + (double)lo) * scale;
}

// Adding the signed value v to a 128-bit accumulator whose low word held
// `old`: the low word becomes old + v (mod 2^64), the high word gains the
// sign extension of v plus the carry out of the low word.  Returns that
// high-word increment.
__host__ __device__ inline unsigned long long fixed128_hi_inc(unsigned long long old, long long v) {
  const unsigned long long u = (unsigned long long)v;
  return (v < 0 ? ~0ull : 0ull) + (old + u < old ? 1ull : 0ull);
}

#ifdef __CUDACC__
// Adds the signed fixed-point value v to the accumulator a[0] (low), a[1]
// (high), the carry read from the value the low word's atomic returned.
__device__ __forceinline__ void fixed128_add(unsigned long long* a, long long v) {
  if (!v) return;
  const unsigned long long old = atomicAdd(a, (unsigned long long)v);
  const unsigned long long hi = fixed128_hi_inc(old, v);
  if (hi) atomicAdd(a + 1, hi);
}

// x / unit in fixed point; false (nothing to add) when out of range or not finite.
__device__ __forceinline__ bool to_fixed(double x, double inv_unit, long long* v) {
  const double s = x * inv_unit * 68719476736.0;  // 2^36
  if (!(fabs(s) < 4.611686018427387904e18)) return false;  // 2^62; NaN fails too
  *v = __double2ll_rn(s);
  return true;
}
#endif

}  // namespace apic
