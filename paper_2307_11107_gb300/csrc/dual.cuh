// Forward-mode dual numbers: a value and its derivatives along N independent
// directions (here the parameters alpha, phi_g and B of the sensitivity
// window).  Arithmetic follows the sum, product and quotient rules; sqrt uses
// d sqrt(x) = dx / (2 sqrt(x)).  Comparisons are left to the caller, on .v:
// the derivative of a branch decision is taken as zero (frozen decisions).
#pragma once
#include <cmath>

#ifdef __CUDACC__
#define APIC_DHD __host__ __device__ __forceinline__
#else
#define APIC_DHD inline
#endif

namespace apic {
// Own namespace: its sqrt must not hide the global one for plain numbers
// inside namespace apic (argument-dependent lookup finds it for duals).
namespace ad {

template <class T, int N>
struct Dual {
  T v;
  T d[N];
  APIC_DHD Dual() {}
  APIC_DHD Dual(T x) : v(x) {
#pragma unroll
    for (int k = 0; k < N; ++k) d[k] = T(0);
  }
  APIC_DHD Dual& operator+=(const Dual& b) {
    v = v + b.v;
#pragma unroll
    for (int k = 0; k < N; ++k) d[k] = d[k] + b.d[k];
    return *this;
  }
  APIC_DHD Dual& operator-=(const Dual& b) {
    v = v - b.v;
#pragma unroll
    for (int k = 0; k < N; ++k) d[k] = d[k] - b.d[k];
    return *this;
  }
  // a constant with unit derivative along direction `dir` (a seeded parameter)
  APIC_DHD static Dual seed(T x, int dir) {
    Dual r(x);
    r.d[dir] = T(1);
    return r;
  }
};

template <class T, int N>
APIC_DHD Dual<T, N> operator-(const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = -a.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = -a.d[k];
  return r;
}
template <class T, int N>
APIC_DHD Dual<T, N> operator+(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
template <class T, int N>
APIC_DHD Dual<T, N> operator-(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
template <class T, int N>
APIC_DHD Dual<T, N> operator*(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
template <class T, int N>
APIC_DHD Dual<T, N> operator/(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r;
  r.v = a.v / b.v;
  T ib = T(1) / b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
  return r;
}
template <class T, int N>
APIC_DHD Dual<T, N> sqrt(const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = ::sqrt(a.v);
  T h = r.v > T(0) ? T(0.5) / r.v : T(0);
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * h;
  return r;
}

// mixed forms with a plain scalar of the same type
template <class T, int N>
APIC_DHD Dual<T, N> operator+(const Dual<T, N>& a, T b) { return a + Dual<T, N>(b); }
template <class T, int N>
APIC_DHD Dual<T, N> operator+(T a, const Dual<T, N>& b) { return Dual<T, N>(a) + b; }
template <class T, int N>
APIC_DHD Dual<T, N> operator-(const Dual<T, N>& a, T b) { return a - Dual<T, N>(b); }
template <class T, int N>
APIC_DHD Dual<T, N> operator-(T a, const Dual<T, N>& b) { return Dual<T, N>(a) - b; }
template <class T, int N>
APIC_DHD Dual<T, N> operator*(const Dual<T, N>& a, T b) {
  Dual<T, N> r;
  r.v = a.v * b;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b;
  return r;
}
template <class T, int N>
APIC_DHD Dual<T, N> operator*(T a, const Dual<T, N>& b) { return b * a; }
template <class T, int N>
APIC_DHD Dual<T, N> operator/(const Dual<T, N>& a, T b) { return a / Dual<T, N>(b); }
template <class T, int N>
APIC_DHD Dual<T, N> operator/(T a, const Dual<T, N>& b) { return Dual<T, N>(a) / b; }

// value part of a plain number or a dual number
template <class T>
APIC_DHD T val(T x) { return x; }
template <class T, int N>
APIC_DHD T val(const Dual<T, N>& x) { return x.v; }

}  // namespace ad
}  // namespace apic
