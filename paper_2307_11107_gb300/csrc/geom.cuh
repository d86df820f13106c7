// Geometry of the shape-conforming coordinates (Eqs. 2-5, 7, 8, 10 of
// arXiv:2307.11107) and the counter-based random numbers, for host set-up code
// and device kernels alike.  Lengths in R0.
#pragma once
#include <cmath>
#include <cstdint>

#ifdef __CUDACC__
#define APIC_HD __host__ __device__ __forceinline__
#else
#define APIC_HD inline
#endif

namespace apic {

constexpr double kPi = 3.141592653589793238462643383279502884;

// Eq. 3: radius of the point (x1, x2).
template <class R>
APIC_HD R radius(R alpha, R x1, R x2) {
  return -(R(1) + sqrt(R(1) - R(4) * alpha * x1 * x2)) / (R(2) * x1);
}

// Eq. 2: x1 of the point at radius r and x2 = cos(theta).
template <class R>
APIC_HD R x1_at(R alpha, R r, R x2) {
  return -(R(1) / r) * (R(1) + alpha * x2 / r);
}

// Grain surface x1 = -1 (Eq. 3): r_g(x2).
template <class R>
APIC_HD R r_grain(R alpha, R x2) {
  return (R(1) + sqrt(R(1) + R(4) * alpha * x2)) / R(2);
}

// d(x1, x2)/d(R, Z) at (r, x2): chain rule of Eq. 2 with r^2 = R^2 + Z^2,
// x2 = Z / r (used with the numerical dphi/dx_i in Eq. 10).
template <class R>
struct Metric {
  R x1R, x1Z, x2R, x2Z;
};

template <class R>
APIC_HD Metric<R> metric(R alpha, R r, R x2) {
  R s2 = (R(1) - x2) * (R(1) + x2);
  R s = sqrt(s2);
  R r3 = r * r * r;
  Metric<R> m;
  m.x1R = s * (r + R(3) * alpha * x2) / r3;
  m.x1Z = (r * x2 + alpha * (R(3) * x2 * x2 - R(1))) / r3;
  m.x2R = -x2 * s / r;
  m.x2Z = s2 / r;
  return m;
}

// Eq. 4: dA/dx2 of the surface x1 = const.
template <class R>
APIC_HD R area_density(R alpha, R x1, R x2) {
  R r = radius(alpha, x1, x2);
  R s2 = (R(1) - x2) * (R(1) + x2);
  R k = alpha / (r + R(2) * alpha * x2);
  return R(2.0 * kPi) * r * r * sqrt(R(1) + s2 * k * k);
}

// Eq. 5: dOmega / (dx1 dx2).
template <class R>
APIC_HD R volume_density(R alpha, R x1, R x2) {
  R r = radius(alpha, x1, x2);
  R r2 = r * r;
  return R(2.0 * kPi) * r2 * r2 / (R(1) + R(2) * alpha * x2 / r);
}

// Coefficients of Eq. 7 at (x1, x2): A d2/dx1^2 + C d2/dx2^2 + D d2/dx1dx2 + E d/dx2.
template <class R>
struct LapCoef {
  R A, C, D, E;
};

template <class R>
APIC_HD LapCoef<R> lap_coef(R alpha, R x1, R x2) {
  R r = radius(alpha, x1, x2);
  R s2 = (R(1) - x2) * (R(1) + x2);
  R r2 = r * r;
  R r4 = r2 * r2;
  R q = r + R(2) * alpha * x2;
  LapCoef<R> c;
  c.A = (q * q + alpha * alpha * s2) / (r4 * r2);
  c.C = s2 / r2;
  c.D = R(-2) * alpha * s2 / r4;
  c.E = R(-2) * x2 / r2;
  return c;
}

// Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11): per round the
// two multiplications M0*c0 and M1*c2 feed c' = (hi(M1 c2) ^ c1 ^ k0,
// lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the key advances by the Weyl
// constants after each round.
struct U4 {
  uint32_t a, b, c, d;
};

APIC_HD U4 philox10(U4 x, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int i = 0; i < 10; ++i) {
#ifdef __CUDA_ARCH__
    uint32_t h0 = __umulhi(M0, x.a), l0 = M0 * x.a;
    uint32_t h1 = __umulhi(M1, x.c), l1 = M1 * x.c;
#else
    uint64_t p0 = (uint64_t)M0 * x.a, p1 = (uint64_t)M1 * x.c;
    uint32_t h0 = (uint32_t)(p0 >> 32), l0 = (uint32_t)p0;
    uint32_t h1 = (uint32_t)(p1 >> 32), l1 = (uint32_t)p1;
#endif
    U4 y;
    y.a = h1 ^ x.b ^ k0;
    y.b = l1;
    y.c = h0 ^ x.d ^ k1;
    y.d = l0;
    x = y;
    k0 += W0;
    k1 += W1;
  }
  return x;
}

// Uniform in (0,1) from 32 random bits: (u + 1/2) 2^-32 (exact in FP64).
APIC_HD double unit_open(uint32_t u) { return ((double)u + 0.5) * 2.3283064365386962890625e-10; }

}  // namespace apic
