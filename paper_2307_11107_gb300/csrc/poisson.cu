// GPU solver of the Poisson problem of Eqs. 6-7 (arXiv:2307.11107, Sec. 2).
//
// The paper factorises the finite-difference matrix with LAPACK LU.  On GB300
// a banded LU has a serial dependency chain the length of the grid and the
// FP64 rate is a small fraction of FP32, so the same discrete system is solved
// here by BiCGSTAB with FP64 vectors and an FP64 matrix-vector product (the
// residual of the refinement is always exact to FP64), preconditioned by one
// multigrid V(1,1) cycle in the particle precision (FP32 for the production
// build, FP64 for the parity build):
//   * the rows are scaled by 1/a1 = h1^2 / A (A the d2/dx1^2 coefficient);
//   * coarse operators are Galerkin products R A P (bilinear P, R = P^T / 4),
//     built once on the host;
//   * the smoother is alternating zebra line Gauss-Seidel: x1-lines, then
//     x2-lines (the pole rows' reach to j +- 2 is eliminated in the x2-line
//     system and ordered after the pole line in the x1-line pass);
//   * each line is a tridiagonal system solved by one warp: partitioned
//     Thomas on per-lane chunks, parallel cyclic reduction of the per-lane
//     head unknowns with shuffles;
//   * coarsening stops at the first level with at most kMaxCoarse unknowns;
//     that level is solved with its dense inverse (Gauss-Jordan on the GPU at
//     set-up), the finer levels are smoothed with one CTA per line.
// All dot products are per-CTA partials summed in a fixed order, so results
// do not depend on scheduling.  Every kernel checks the per-instance `done`
// flag, so a fixed launch sequence (CUDA-graph friendly) stops doing work once
// the tolerance is met.
#include <cuda_runtime.h>

#include <cstdint>

#include "apic_internal.h"

namespace apic {
namespace {

#include "solver_common.cuh"

constexpr int kLineThreads = 256;  // threads per CTA (one line) in the multi-CTA line kernels
constexpr int kSolveThreads = 512;

__device__ __forceinline__ double block_sum256(double v, double* sh) {
  int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (t < o) sh[t] += sh[t + o];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ double sum_partials(const DevPtrs& d, int inst, int slot) {
  const double* p = d.red + ((long long)inst * kNRed + slot) * kRedBlocks;
  double s = 0.0;
  for (int k = 0; k < kRedBlocks; ++k) s += p[k];
  return s;
}

// The same fixed-order sum, done once per CTA by warp 0 and broadcast.
__device__ __forceinline__ double cta_partials(const DevPtrs& d, int inst, int slot, double* sh) {
  if (threadIdx.x < 32) {
    const double* p = d.red + ((long long)inst * kNRed + slot) * kRedBlocks;
    double v = p[threadIdx.x] + p[threadIdx.x + 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    if (threadIdx.x == 0) *sh = v;
  }
  __syncthreads();
  double r = *sh;
  __syncthreads();
  return r;
}

__device__ __forceinline__ void put_partial(const DevPtrs& d, int inst, int slot, double v) {
  d.red[((long long)inst * kNRed + slot) * kRedBlocks + blockIdx.x] = v;
}

// ---------------------------------------------------------------------------
// Warp tridiagonal solver.  Row r of the line lives in smem slot
// (r - lane*K) * 32 + lane (lane = r / K): conflict-free per-lane chunks.
// On entry a, b, c, d hold sub-, main-, super-diagonal and right-hand side;
// on exit d holds the solution.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int k_for(int n) { return (n + 31) / 32; }

__device__ __forceinline__ int lslot(int r, int K) {
  int L = r / K;
  return (r - L * K) * 32 + L;
}

template <class Real>
__device__ void warp_tridiag(Real* a, Real* b, Real* c, Real* d, int n, int K) {
  const int lane = threadIdx.x & 31;
  const int r0 = lane * K;
  int m = n - r0;
  m = m < 0 ? 0 : (m > K ? K : m);
  // forward: rows k >= 1 as x_k = d_k - a_k x_head - c_k x_{k+1}
  for (int k = 1; k < m; ++k) {
    int s = k * 32 + lane, sp = (k - 1) * 32 + lane;
    Real ak = a[s], bk = b[s], ck = c[s], dk = d[s];
    Real den, al, ga, de;
    if (k == 1) {
      den = bk;
      al = ak / den;
      ga = ck / den;
      de = dk / den;
    } else {
      den = bk - ak * c[sp];
      al = -ak * a[sp] / den;
      ga = ck / den;
      de = (dk - ak * d[sp]) / den;
    }
    a[s] = al;
    c[s] = ga;
    d[s] = de;
  }
  // backward: rows k >= 1 as x_k = d_k - a_k x_head - c_k x_next_head
  for (int k = m - 2; k >= 1; --k) {
    int s = k * 32 + lane, sn = (k + 1) * 32 + lane;
    Real ga = c[s];
    d[s] = d[s] - ga * d[sn];
    a[s] = a[s] - ga * a[sn];
    c[s] = -ga * c[sn];
  }
  // reduced equation of the head unknown x_{r0}
  Real A = Real(0), B = Real(1), C = Real(0), D = Real(0);
  Real ta = Real(0), tc = Real(0), td = Real(0);  // tail = td - ta*x_head - tc*x_next
  int tail_is_head = 1;
  if (m >= 1) {
    int s0 = lane;
    Real a0 = a[s0], b0 = b[s0], c0 = c[s0], d0 = d[s0];
    if (m >= 2) {
      int s1 = 32 + lane;
      B = b0 - c0 * a[s1];
      C = -c0 * c[s1];
      D = d0 - c0 * d[s1];
      int st = (m - 1) * 32 + lane;
      ta = a[st];
      tc = c[st];
      td = d[st];
      tail_is_head = 0;
    } else {
      B = b0;
      C = c0;
      D = d0;
    }
    A = a0;
  }
  // substitute the previous lane's tail: x_ptail = td' - ta' x_phead - tc' x_head
  Real pta = __shfl_up_sync(kFull, ta, 1), ptc = __shfl_up_sync(kFull, tc, 1), ptd = __shfl_up_sync(kFull, td, 1);
  int pth = __shfl_up_sync(kFull, tail_is_head, 1);
  if (m >= 1 && lane > 0 && !pth) {
    Real a0 = A;
    A = -a0 * pta;
    B = B - a0 * ptc;
    D = D - a0 * ptd;
  }
  if (m < 1) {
    A = Real(0);
    B = Real(1);
    C = Real(0);
    D = Real(0);
  }
  // parallel cyclic reduction over the 32 head unknowns
#pragma unroll
  for (int sft = 1; sft < 32; sft <<= 1) {
    Real Am = __shfl_up_sync(kFull, A, sft), Bm = __shfl_up_sync(kFull, B, sft);
    Real Cm = __shfl_up_sync(kFull, C, sft), Dm = __shfl_up_sync(kFull, D, sft);
    Real Ap = __shfl_down_sync(kFull, A, sft), Bp = __shfl_down_sync(kFull, B, sft);
    Real Cp = __shfl_down_sync(kFull, C, sft), Dp = __shfl_down_sync(kFull, D, sft);
    if (lane < sft) {
      Am = Real(0);
      Bm = Real(1);
      Cm = Real(0);
      Dm = Real(0);
    }
    if (lane + sft >= 32) {
      Ap = Real(0);
      Bp = Real(1);
      Cp = Real(0);
      Dp = Real(0);
    }
    Real k1 = A / Bm, k2 = C / Bp;
    Real nA = -k1 * Am;
    Real nB = B - k1 * Cm - k2 * Ap;
    Real nC = -k2 * Cp;
    Real nD = D - k1 * Dm - k2 * Dp;
    A = nA;
    B = nB;
    C = nC;
    D = nD;
  }
  Real xh = D / B;
  Real xn = __shfl_down_sync(kFull, xh, 1);
  if (lane == 31) xn = Real(0);
  if (m >= 1) {
    d[lane] = xh;
    for (int k = 1; k < m; ++k) {
      int s = k * 32 + lane;
      d[s] = d[s] - a[s] * xh - c[s] * xn;
    }
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// The same partitioned solver split into a matrix-only factorisation (done
// once at set-up: the line matrices are constant in time) and a right-hand-
// side-only solve with no divisions.  Stored per line, in slot layout:
//   rows: a_k, 1/den_k, gamma_k (forward), alpha^_k, gamma^_k   (5 x 32K)
//   lanes: a_0, c_0, PCR factors k1, k2 of the 5 steps, 1/B       (13 x 32)
//   line:  the two pole-elimination factors of x2-lines           (2)
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int fac_stride(int K) { return line_fac_stride(K); }

template <class Real>
__device__ void warp_factor(const Real* a, const Real* b, const Real* c, int n, int K, Real* F) {
  const int lane = threadIdx.x & 31;
  const int r0 = lane * K;
  int m = n - r0;
  m = m < 0 ? 0 : (m > K ? K : m);
  Real* Fa = F;
  Real* Fi = F + 32 * K;
  Real* Fg = F + 64 * K;
  Real* Fah = F + 96 * K;
  Real* Fgh = F + 128 * K;
  Real* L = F + 160 * K;
  Real al_prev = Real(0), ga_prev = Real(0);
  for (int k = 1; k < m; ++k) {
    int s = k * 32 + lane;
    Real ak = a[s], bk = b[s], ck = c[s];
    Real den = k == 1 ? bk : bk - ak * ga_prev;
    Real al = k == 1 ? ak / den : -ak * al_prev / den;
    Real ga = ck / den;
    Fa[s] = ak;
    Fi[s] = Real(1) / den;
    Fg[s] = ga;
    Fah[s] = al;
    Fgh[s] = ga;
    al_prev = al;
    ga_prev = ga;
  }
  for (int k = m - 2; k >= 1; --k) {
    int s = k * 32 + lane, sn = (k + 1) * 32 + lane;
    Real ga = Fg[s];
    Fah[s] = Fah[s] - ga * Fah[sn];
    Fgh[s] = -ga * Fgh[sn];
  }
  Real A = Real(0), B = Real(1), C = Real(0), ta = Real(0), tc = Real(0);
  int tail_is_head = 1;
  Real a0 = Real(0), c0 = Real(0);
  if (m >= 1) {
    a0 = a[lane];
    c0 = c[lane];
    Real b0 = b[lane];
    if (m >= 2) {
      B = b0 - c0 * Fah[32 + lane];
      C = -c0 * Fgh[32 + lane];
      ta = Fah[(m - 1) * 32 + lane];
      tc = Fgh[(m - 1) * 32 + lane];
      tail_is_head = 0;
    } else {
      B = b0;
      C = c0;
    }
    A = a0;
  }
  Real pta = __shfl_up_sync(kFull, ta, 1), ptc = __shfl_up_sync(kFull, tc, 1);
  int pth = __shfl_up_sync(kFull, tail_is_head, 1);
  if (m >= 1 && lane > 0 && !pth) {
    A = -a0 * pta;
    B = B - a0 * ptc;
  }
  if (m < 1) {
    A = Real(0);
    B = Real(1);
    C = Real(0);
  }
  L[0 * 32 + lane] = a0;
  L[1 * 32 + lane] = c0;
  int st = 0;
#pragma unroll
  for (int sft = 1; sft < 32; sft <<= 1, ++st) {
    Real Am = __shfl_up_sync(kFull, A, sft), Bm = __shfl_up_sync(kFull, B, sft), Cm = __shfl_up_sync(kFull, C, sft);
    Real Ap = __shfl_down_sync(kFull, A, sft), Bp = __shfl_down_sync(kFull, B, sft), Cp = __shfl_down_sync(kFull, C, sft);
    if (lane < sft) {
      Am = Real(0);
      Bm = Real(1);
      Cm = Real(0);
    }
    if (lane + sft >= 32) {
      Ap = Real(0);
      Bp = Real(1);
      Cp = Real(0);
    }
    Real k1 = A / Bm, k2 = C / Bp;
    Real nA = -k1 * Am, nB = B - k1 * Cm - k2 * Ap, nC = -k2 * Cp;
    A = nA;
    B = nB;
    C = nC;
    L[(2 + 2 * st) * 32 + lane] = k1;
    L[(3 + 2 * st) * 32 + lane] = k2;
  }
  L[12 * 32 + lane] = Real(1) / B;
}

// Solve with stored factors: d (slot layout, right-hand side) -> solution.
template <class Real>
__device__ __forceinline__ void warp_solve(const Real* __restrict__ F, Real* d, int n, int K) {
  const int lane = threadIdx.x & 31;
  const int r0 = lane * K;
  int m = n - r0;
  m = m < 0 ? 0 : (m > K ? K : m);
  const Real* Fa = F;
  const Real* Fi = F + 32 * K;
  const Real* Fg = F + 64 * K;
  const Real* Fah = F + 96 * K;
  const Real* Fgh = F + 128 * K;
  const Real* L = F + 160 * K;
  Real prev = Real(0);
  for (int k = 1; k < m; ++k) {
    int s = k * 32 + lane;
    Real v = k == 1 ? d[s] * Fi[s] : (d[s] - Fa[s] * prev) * Fi[s];
    d[s] = v;
    prev = v;
  }
  for (int k = m - 2; k >= 1; --k) {
    int s = k * 32 + lane;
    Real v = d[s] - Fg[s] * d[s + 32];
    d[s] = v;
  }
  Real D = Real(0), td = Real(0);
  int tail_is_head = 1;
  if (m >= 1) {
    D = d[lane];
    if (m >= 2) {
      D = D - L[32 + lane] * d[32 + lane];
      td = d[(m - 1) * 32 + lane];
      tail_is_head = 0;
    }
  }
  Real ptd = __shfl_up_sync(kFull, td, 1);
  int pth = __shfl_up_sync(kFull, tail_is_head, 1);
  if (m >= 1 && lane > 0 && !pth) D = D - L[lane] * ptd;
  if (m < 1) D = Real(0);
  int st = 0;
#pragma unroll
  for (int sft = 1; sft < 32; sft <<= 1, ++st) {
    Real Dm = __shfl_up_sync(kFull, D, sft), Dp = __shfl_down_sync(kFull, D, sft);
    if (lane < sft) Dm = Real(0);
    if (lane + sft >= 32) Dp = Real(0);
    D = D - L[(2 + 2 * st) * 32 + lane] * Dm - L[(3 + 2 * st) * 32 + lane] * Dp;
  }
  Real xh = D * L[12 * 32 + lane];
  Real xn = __shfl_down_sync(kFull, xh, 1);
  if (lane == 31) xn = Real(0);
  if (m >= 1) {
    d[lane] = xh;
    for (int k = 1; k < m; ++k) {
      int s = k * 32 + lane;
      d[s] = d[s] - Fah[s] * xh - Fgh[s] * xn;
    }
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Level operations (one line / one node at a time); used by the multi-CTA
// kernels and by the single-CTA tail.
// ---------------------------------------------------------------------------
template <class Real>
struct LevelView {
  const Real* st;
  Real* e;
  const Real* f;
  const Real* fac[2];  // line factorisations (x1-lines by j, x2-lines by i)
  long long nodes;
  int n1, n2, N2, pole;
};

template <class Real>
__device__ __forceinline__ LevelView<Real> view(const DevPtrs& d, const Inst& I, int l) {
  const Level& L = I.lv[l];
  LevelView<Real> v;
  v.st = (const Real*)d.st + L.st;
  v.e = (Real*)d.e + L.off;
  v.f = (const Real*)d.f + L.off;
  v.nodes = (long long)L.N1 * L.N2;
  v.n1 = L.n1;
  v.n2 = L.n2;
  v.N2 = L.N2;
  v.pole = L.pole_extra;
  v.fac[0] = (const Real*)d.fac + L.fac[0];
  v.fac[1] = (const Real*)d.fac + L.fac[1];
  return v;
}

template <class Real>
__device__ __forceinline__ Real resid_at(const LevelView<Real>& v, int i, int j) {
  long long nd = (long long)i * v.N2 + j;
  return v.f[nd] - apply_st<Real, Real>(v.st, v.nodes, v.e, nd, i, j, v.n2, v.N2, v.pole);
}

// Thread groups that assemble a line system: one warp (coarse levels, many
// lines per CTA) or a whole CTA (fine levels, one line per CTA, more loads in
// flight).  In both cases the first warp of the group solves the system.
struct WarpGroup {
  __device__ int tid() const { return threadIdx.x & 31; }
  __device__ int size() const { return 32; }
  __device__ void sync() const { __syncwarp(); }
  __device__ bool solver() const { return true; }
};
struct BlockGroup {
  __device__ int tid() const { return threadIdx.x; }
  __device__ int size() const { return blockDim.x; }
  __device__ void sync() const { __syncthreads(); }
  __device__ bool solver() const { return threadIdx.x < 32; }
};

// Line work buffer: right-hand side (32K) followed by the line's factors,
// copied from global memory in one coalesced pass so that the solver's
// recurrences read shared memory only.
__host__ __device__ constexpr int line_buf(int K) { return 32 * K + fac_stride(K); }

// Bulk copy global -> shared with eight loads in flight per thread before any
// store (a plain load/store loop would pay one memory latency per element).
template <class Real>
__device__ __forceinline__ void copy_batched(Real* dst, const Real* __restrict__ src, long long n, int tid, int stride) {
  for (long long k0 = tid; k0 < n; k0 += 8LL * stride) {
    Real v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      long long k = k0 + (long long)u * stride;
      v[u] = k < n ? src[k] : Real(0);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      long long k = k0 + (long long)u * stride;
      if (k < n) dst[k] = v[u];
    }
  }
}

template <class Real, class Grp>
__device__ __forceinline__ const Real* stage_factors(const Real* F, Real* buf, int K, const Grp& g) {
  Real* S = buf + 32 * K;
  copy_batched(S, F, fac_stride(K), g.tid(), g.size());
  return S;
}

// x1-line j (unknowns i = 1..n1-1) solved exactly for the correction with
// its stored factors F.
template <class Real, class Grp>
__device__ void relax_x1_line(const LevelView<Real>& v, int j, Real* dd, int K, const Real* Fg, const Grp& g) {
  const int n = v.n1 - 1;
  const Real* F = stage_factors(Fg, dd, K, g);
  for (int r = g.tid(); r < n; r += g.size()) dd[lslot(r, K)] = resid_at(v, r + 1, j);
  g.sync();
  if (g.solver()) warp_solve(F, dd, n, K);
  g.sync();
  for (int r = g.tid(); r < n; r += g.size()) v.e[(long long)(r + 1) * v.N2 + j] += dd[lslot(r, K)];
  g.sync();
}

// x2-line i (unknowns j = 0..n2); on the finest level the pole reaches are
// eliminated with the neighbouring row (factors stored with the line).
template <class Real, class Grp>
__device__ void relax_x2_line(const LevelView<Real>& v, int i, Real* dd, int K, const Real* Fg, const Grp& g) {
  const int n = v.n2 + 1;
  long long base = (long long)i * v.N2;
  const Real* F = stage_factors(Fg, dd, K, g);
  for (int r = g.tid(); r < n; r += g.size()) dd[lslot(r, K)] = resid_at(v, i, r);
  g.sync();
  if (v.pole && g.tid() == 0) {
    const Real* P = F + fac_stride(K) - 2;
    dd[lslot(0, K)] -= P[0] * dd[lslot(1, K)];
    dd[lslot(v.n2, K)] -= P[1] * dd[lslot(v.n2 - 1, K)];
  }
  g.sync();
  if (g.solver()) warp_solve(F, dd, n, K);
  g.sync();
  for (int r = g.tid(); r < n; r += g.size()) v.e[base + r] += dd[lslot(r, K)];
  g.sync();
}

// Set-up: the line matrices of level l in direction dir, factorised.
template <class Real>
__device__ void factor_line(const LevelView<Real>& v, int dir, int line, Real* buf, int K, Real* F) {
  const int lane = threadIdx.x & 31;
  const int n = dir == 0 ? v.n1 - 1 : v.n2 + 1;
  Real* a = buf;
  Real* b = buf + 32 * K;
  Real* c = buf + 64 * K;
  for (int r = lane; r < 32 * K; r += 32) {
    a[r] = Real(0);
    b[r] = Real(1);
    c[r] = Real(0);
  }
  __syncwarp();
  for (int r = lane; r < n; r += 32) {
    int s = lslot(r, K);
    if (dir == 0) {
      long long nd = (long long)(r + 1) * v.N2 + line;
      a[s] = v.st[st_slot(-1, 0) * v.nodes + nd];
      b[s] = v.st[st_slot(0, 0) * v.nodes + nd];
      c[s] = v.st[st_slot(1, 0) * v.nodes + nd];
    } else {
      long long nd = (long long)line * v.N2 + r;
      a[s] = r > 0 ? v.st[st_slot(0, -1) * v.nodes + nd] : Real(0);
      b[s] = v.st[st_slot(0, 0) * v.nodes + nd];
      c[s] = r < v.n2 ? v.st[st_slot(0, 1) * v.nodes + nd] : Real(0);
    }
  }
  __syncwarp();
  Real g0 = Real(0), gn = Real(0);
  if (dir == 1 && v.pole && lane == 0) {
    long long base = (long long)line * v.N2;
    int s0 = lslot(0, K), s1 = lslot(1, K);
    g0 = v.st[kStPole * v.nodes + base] / c[s1];
    b[s0] -= g0 * a[s1];
    c[s0] -= g0 * b[s1];
    int sn = lslot(v.n2, K), sm = lslot(v.n2 - 1, K);
    gn = v.st[kStPole * v.nodes + base + v.n2] / a[sm];
    b[sn] -= gn * c[sm];
    a[sn] -= gn * b[sm];
  }
  __syncwarp();
  warp_factor(a, b, c, n, K, F);
  if (lane == 0) {
    F[fac_stride(K) - 2] = g0;
    F[fac_stride(K) - 1] = gn;
  }
  __syncwarp();
}

// Line index of colour class `color` handled by worker w, with the pole
// pairing of the finest level (line 0 then 2, line n2 then n2-2, same worker).
__device__ __forceinline__ int x1_line_of(int w, int color, int n2, int pole, int* second) {
  int j = 2 * w + color;
  *second = -1;
  if (j > n2) return -1;
  if (pole) {
    if (j == 2 || j == n2 - 2) return -2;  // done by the pole worker
    if (j == 0) *second = 2;
    if (j == n2) *second = n2 - 2;
  }
  return j;
}

template <class Real, class Grp>
__device__ void x1_pass(const LevelView<Real>& v, int color, int w, Real* buf, int K, const Grp& g) {
  int second;
  int j = x1_line_of(w, color, v.n2, v.pole, &second);
  if (j < 0) return;
  relax_x1_line(v, j, buf, K, v.fac[0] + (long long)j * fac_stride(K), g);
  if (second >= 0) relax_x1_line(v, second, buf, K, v.fac[0] + (long long)second * fac_stride(K), g);
}

template <class Real, class Grp>
__device__ void x2_pass(const LevelView<Real>& v, int color, int w, Real* buf, int K, const Grp& g) {
  int i = 1 + 2 * w + color;
  if (i > v.n1 - 1) return;
  relax_x2_line(v, i, buf, K, v.fac[1] + (long long)i * fac_stride(K), g);
}

// Set-up kernel: factorise every line of level l in direction dir (one warp per line).
template <class Real>
__global__ void __launch_bounds__(128) k_line_factor(DevPtrs d, int l, int dir, int kmax) {
  extern __shared__ unsigned char smem_raw[];
  const int inst = blockIdx.y;
  const Inst& I = d.inst[inst];
  if (l >= I.n_levels) return;
  LevelView<Real> v = view<Real>(d, I, l);
  const int warp = threadIdx.x >> 5;
  const int line = blockIdx.x * 4 + warp;
  const int K = dir == 0 ? k_for(v.n1 - 1) : k_for(v.n2 + 1);
  if (dir == 0 ? line > v.n2 : (line < 1 || line > v.n1 - 1)) return;
  Real* buf = (Real*)smem_raw + (long long)warp * 96 * kmax;
  factor_line(v, dir, line, buf, K, (Real*)v.fac[dir] + (long long)line * fac_stride(K));
}

// Coarse right-hand side f_c = R (f - A e) with R = P^T / 4, and e_c = 0.
template <class Real>
__device__ void restrict_node(const LevelView<Real>& F, const LevelView<Real>& Cc, long long ndc) {
  int I = (int)(ndc / Cc.N2), J = (int)(ndc % Cc.N2);
  Real acc = Real(0);
  if (I > 0 && I < Cc.n1) {
    for (int di = -1; di <= 1; ++di) {
      int i = 2 * I + di;
      if (i < 1 || i > F.n1 - 1) continue;
      Real wi = di == 0 ? Real(1) : Real(0.5);
      for (int dj = -1; dj <= 1; ++dj) {
        int j = 2 * J + dj;
        if (j < 0 || j > F.n2) continue;
        Real wj = dj == 0 ? Real(1) : Real(0.5);
        acc += Real(0.25) * wi * wj * resid_at(F, i, j);
      }
    }
  }
  ((Real*)Cc.f)[ndc] = acc;
  Cc.e[ndc] = Real(0);
}

// e_f += P e_c (bilinear; coarse Dirichlet rows carry zero).
template <class Real>
__device__ void prolong_node(const LevelView<Real>& F, const LevelView<Real>& Cc, long long nd) {
  int i = (int)(nd / F.N2), j = (int)(nd % F.N2);
  if (i < 1 || i > F.n1 - 1) return;
  int I0 = i >> 1, I1 = (i + 1) >> 1, J0 = j >> 1, J1 = (j + 1) >> 1;
  const Real* ec = Cc.e;
  Real v = Real(0.25) * (ec[(long long)I0 * Cc.N2 + J0] + ec[(long long)I1 * Cc.N2 + J0] +
                         ec[(long long)I0 * Cc.N2 + J1] + ec[(long long)I1 * Cc.N2 + J1]);
  F.e[nd] += v;
}


// ---------------------------------------------------------------------------
// Kernels.
// ---------------------------------------------------------------------------
// One CTA per line of colour `color` (dir 0: x1-lines, dir 1: x2-lines).
template <class Real>
__global__ void __launch_bounds__(kLineThreads) k_xlines(DevPtrs d, int l, int color, int dir) {
  extern __shared__ unsigned char smem_raw[];
  const int inst = blockIdx.y;
  const Inst& I = d.inst[inst];
  if (d.sol[inst].done || l >= I.tail_level) return;
  LevelView<Real> v = view<Real>(d, I, l);
  int K = dir == 0 ? k_for(v.n1 - 1) : k_for(v.n2 + 1);
  Real* buf = (Real*)smem_raw;
  BlockGroup g;
  if (dir == 0) x1_pass(v, color, (int)blockIdx.x, buf, K, g);
  else x2_pass(v, color, (int)blockIdx.x, buf, K, g);
}

template <class Real>
__global__ void __launch_bounds__(256) k_restrict(DevPtrs d, int l) {
  const int inst = blockIdx.y;
  const Inst& I = d.inst[inst];
  if (d.sol[inst].done || l >= I.tail_level) return;
  LevelView<Real> F = view<Real>(d, I, l), Cc = view<Real>(d, I, l + 1);
  for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < Cc.nodes;
       nd += (long long)gridDim.x * blockDim.x)
    restrict_node(F, Cc, nd);
}

template <class Real>
__global__ void __launch_bounds__(256) k_prolong(DevPtrs d, int l) {
  const int inst = blockIdx.y;
  const Inst& I = d.inst[inst];
  if (d.sol[inst].done || l >= I.tail_level) return;
  LevelView<Real> F = view<Real>(d, I, l), Cc = view<Real>(d, I, l + 1);
  for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < F.nodes;
       nd += (long long)gridDim.x * blockDim.x)
    prolong_node(F, Cc, nd);
}

// Coarsest level: e = Cinv f over its unknowns (rows 1..n1-1, all j), one
// warp per row of the dense inverse (coalesced, eight partial sums).
template <class Real>
__device__ __forceinline__ void coarse_rows(const DevPtrs& d, const Inst& I, long long warp0, long long nwarps) {
  const int lane = threadIdx.x & 31;
  LevelView<Real> C = view<Real>(d, I, I.n_levels - 1);
  const Real* cinv = (const Real*)d.cinv + I.cinv_off;
  const Real* f = C.f + C.N2;
  const int nu = I.coarse_n;
  for (long long u = warp0; u < nu; u += nwarps) {
    const Real* row = cinv + u * nu;
    Real acc = Real(0);
    for (int k = lane; k < nu; k += 32) acc += row[k] * f[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kFull, acc, o);
    if (lane == 0) C.e[C.N2 + u] = acc;
  }
}

template <class Real>
__global__ void __launch_bounds__(256) k_coarse(DevPtrs d) {
  const int inst = blockIdx.y;
  const Inst& I = d.inst[inst];
  if (d.sol[inst].done) return;
  long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  coarse_rows<Real>(d, I, (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), warps);
}

// Set-up: Gauss-Jordan with partial pivoting on an n x 2n FP64 matrix [A | I]
// in one cooperative launch.  Per column c: CTA 0 picks the pivot, swaps it
// into row c, scales row c and records the elimination factors fb; after a
// grid barrier every warp updates its rows; a second barrier ends the column.
// The barrier counts on *cnt (zeroed before the launch), each wait bounded by
// wait_ns of global time (then kErrTimeout in *err and every CTA returns).
__device__ bool gj_sync(unsigned long long* cnt, unsigned nb, int32_t* err, unsigned long long wait_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long old = atom_add_release_u64(cnt, 1ull);
    const unsigned long long target = (old / nb + 1ull) * nb;
    int ok = 1;
    unsigned long long t0 = 0;
    for (long long spins = 0; ld_acquire_u64(cnt) < target; ++spins) {
      if ((spins & 255) == 255) {
        if ((*(volatile int*)err) & kErrTimeout) {
          ok = 0;
          break;
        }
        const unsigned long long now = global_ns();
        if (t0 == 0) t0 = now;
        else if (now - t0 > wait_ns) {
          atomicOr(err, kErrTimeout);
          ok = 0;
          break;
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__global__ void __launch_bounds__(1024) k_gj(double* M, double* fb, int n, unsigned long long* cnt, int32_t* err,
                                             unsigned long long wait_ns) {
  __shared__ double sv[1024];
  __shared__ int si[1024];
  const long long w = 2LL * n;
  const unsigned nb = gridDim.x;
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  for (int c = 0; c < n; ++c) {
    if (blockIdx.x == 0) {
      double best = -1.0;
      int arg = c;
      for (int r = c + threadIdx.x; r < n; r += blockDim.x) {
        const double v = fabs(M[(long long)r * w + c]);
        if (v > best) {
          best = v;
          arg = r;
        }
      }
      sv[threadIdx.x] = best;
      si[threadIdx.x] = arg;
      __syncthreads();
      for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
          const double x = sv[threadIdx.x], y = sv[threadIdx.x + o];
          const int ix = si[threadIdx.x], iy = si[threadIdx.x + o];
          if (y > x || (y == x && iy < ix)) {
            sv[threadIdx.x] = y;
            si[threadIdx.x] = iy;
          }
        }
        __syncthreads();
      }
      const int p = si[0];
      if (p != c)
        for (long long k = threadIdx.x; k < w; k += blockDim.x) {
          const double t = M[(long long)c * w + k];
          M[(long long)c * w + k] = M[(long long)p * w + k];
          M[(long long)p * w + k] = t;
        }
      __syncthreads();
      const double inv = 1.0 / M[(long long)c * w + c];
      __syncthreads();
      for (long long k = threadIdx.x; k < w; k += blockDim.x) M[(long long)c * w + k] *= inv;
      for (int r = threadIdx.x; r < n; r += blockDim.x) fb[r] = r == c ? 0.0 : M[(long long)r * w + c];
    }
    if (!gj_sync(cnt, nb, err, wait_ns)) return;
    for (long long r = gw; r < n; r += warps) {
      const double f = fb[r];
      if (f == 0.0) continue;
      for (long long k = c + lane; k < w; k += 32) M[r * w + k] -= f * M[(long long)c * w + k];
    }
    if (!gj_sync(cnt, nb, err, wait_ns)) return;
  }
}

template <class Real>
__global__ void k_gj_store(const double* M, int n, Real* out) {
  const long long w = 2LL * n;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < (long long)n * n;
       k += (long long)gridDim.x * blockDim.x)
    out[k] = (Real)M[(k / n) * w + n + (k % n)];
}

// ---- BiCGSTAB (FP64 vectors) ----
// r = b - A x, rh = r, p = v = 0; partials (rh, r), |r|^2.
template <class Real>
__global__ void __launch_bounds__(256) k_bicg_init(DevPtrs d) {
  __shared__ double sh[256];
  const int inst = blockIdx.y;
  const Inst& I = d.inst[inst];
  const bool nofield = (I.flags & APIC_NO_FIELD) != 0;
  const double* st = d.st64 + (long long)kSt * I.node_off;
  const double* x = d.phi + I.node_off;
  double pr = 0.0;
  for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes;
       nd += (long long)gridDim.x * blockDim.x) {
    int i = (int)(nd / I.N2), j = (int)(nd % I.N2);
    long long g = I.node_off + nd;
    double r = 0.0;
    if (i > 0 && i < I.n1 && !nofield)
      r = d.b[g] - apply_st<double, double>(st, I.nodes, x, nd, i, j, I.n2, I.N2, 1);
    d.r[g] = r;
    d.rh[g] = r;
    d.p[g] = 0.0;
    d.v[g] = 0.0;
    pr += r * r;
  }
  double t = block_sum256(pr, sh);
  if (threadIdx.x == 0) {
    put_partial(d, inst, 1, t);
    put_partial(d, inst, 2, t);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    SolverState& S = d.sol[inst];
    S.rho_old = 1.0;
    S.alpha = 1.0;
    S.omega = 1.0;
    S.iters = 0;
    S.done = nofield ? 1 : 0;
    S.res = 0.0;
  }
}

// Convergence test; p = r + beta (p - omega v); f0 = p, e0 = 0.
template <class Real>
__global__ void __launch_bounds__(256) k_bicg_p(DevPtrs d, int final_check) {
  const int inst = blockIdx.y;
  const Inst& I = d.inst[inst];
  SolverState& S = d.sol[inst];
  if (S.done) return;
  __shared__ double shp;
  double bn = cta_partials(d, inst, 0, &shp), rho = cta_partials(d, inst, 1, &shp), rn = cta_partials(d, inst, 2, &shp);
  double tol2 = I.tol * I.tol;
  const double rn0 = S.iters == 0 ? rn : S.rn0;
  bool conv = rn <= fmax(tol2 * bn, S.eta2 * rn0) || !(rn == rn);
  bool last = final_check || S.iters >= I.max_iter;
  if (conv || last) {
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      S.done = 1;
      S.res = bn > 0.0 ? sqrt(rn / bn) : 0.0;
      if (!conv) atomicOr(d.err, kErrNotConverged);
      if (!(rn == rn)) atomicOr(d.err, kErrNonFinite);
    }
    return;
  }
  double beta = (S.omega != 0.0 && S.rho_old != 0.0) ? (rho / S.rho_old) * (S.alpha / S.omega) : 0.0;
  double om = S.omega;
  const Level& L0 = I.lv[0];
  Real* f0 = (Real*)d.f + L0.off;
  Real* e0 = (Real*)d.e + L0.off;
  for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes;
       nd += (long long)gridDim.x * blockDim.x) {
    long long g = I.node_off + nd;
    double p = d.r[g] + beta * (d.p[g] - om * d.v[g]);
    d.p[g] = p;
    f0[nd] = (Real)p;
    e0[nd] = Real(0);
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S.rho = rho;
    if (S.iters == 0) S.rn0 = rn;
  }
}

// ph = M^-1 p (from e0), v = A ph; partial (rh, v).  Same kernel for the
// second half (sh = M^-1 s, t = A sh; partials (t, s), (t, t)).
template <class Real>
__global__ void __launch_bounds__(256) k_bicg_apply(DevPtrs d, int second) {
  __shared__ double sh[256];
  const int inst = blockIdx.y;
  const Inst& I = d.inst[inst];
  if (d.sol[inst].done) return;
  const Level& L0 = I.lv[0];
  const Real* e0 = (const Real*)d.e + L0.off;
  const double* st = d.st64 + (long long)kSt * I.node_off;
  double* out_pre = second ? d.sh : d.ph;
  double* out = second ? d.t : d.v;
  double q1 = 0.0, q2 = 0.0;
  for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes;
       nd += (long long)gridDim.x * blockDim.x) {
    int i = (int)(nd / I.N2), j = (int)(nd % I.N2);
    long long g = I.node_off + nd;
    double y = 0.0, z = 0.0;
    if (i > 0 && i < I.n1) {
      z = (double)e0[nd];
      y = apply_st<double, Real>(st, I.nodes, e0, nd, i, j, I.n2, I.N2, 1);
    }
    out_pre[g] = z;
    out[g] = y;
    if (second) {
      q1 += y * d.s[g];
      q2 += y * y;
    } else {
      q1 += d.rh[g] * y;
    }
  }
  double a = block_sum256(q1, sh);
  double b = second ? block_sum256(q2, sh) : 0.0;
  if (threadIdx.x == 0) {
    if (second) {
      put_partial(d, inst, 4, a);
      put_partial(d, inst, 5, b);
    } else {
      put_partial(d, inst, 3, a);
    }
  }
}

// alpha = rho / (rh, v); s = r - alpha v; f0 = s, e0 = 0.
template <class Real>
__global__ void __launch_bounds__(256) k_bicg_s(DevPtrs d) {
  const int inst = blockIdx.y;
  const Inst& I = d.inst[inst];
  SolverState& S = d.sol[inst];
  if (S.done) return;
  __shared__ double shp;
  double den = cta_partials(d, inst, 3, &shp);
  double alpha = den != 0.0 ? S.rho / den : 0.0;
  const Level& L0 = I.lv[0];
  Real* f0 = (Real*)d.f + L0.off;
  Real* e0 = (Real*)d.e + L0.off;
  for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes;
       nd += (long long)gridDim.x * blockDim.x) {
    long long g = I.node_off + nd;
    double s = d.r[g] - alpha * d.v[g];
    d.s[g] = s;
    f0[nd] = (Real)s;
    e0[nd] = Real(0);
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S.alpha = alpha;
    S.rho_old = S.rho;
  }
}

// omega = (t, s) / (t, t); x += alpha ph + omega sh; r = s - omega t;
// partials (rh, r), |r|^2 for the next test.
template <class Real>
__global__ void __launch_bounds__(256) k_bicg_x(DevPtrs d) {
  __shared__ double sh[256];
  const int inst = blockIdx.y;
  const Inst& I = d.inst[inst];
  SolverState& S = d.sol[inst];
  if (S.done) return;
  __shared__ double shp;
  double ts = cta_partials(d, inst, 4, &shp), tt = cta_partials(d, inst, 5, &shp);
  double om = tt != 0.0 ? ts / tt : 0.0;
  double al = S.alpha;
  double q1 = 0.0, q2 = 0.0;
  for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes;
       nd += (long long)gridDim.x * blockDim.x) {
    int i = (int)(nd / I.N2);
    long long g = I.node_off + nd;
    if (i > 0 && i < I.n1) d.phi[g] += al * d.ph[g] + om * d.sh[g];
    double r = d.s[g] - om * d.t[g];
    d.r[g] = r;
    q1 += d.rh[g] * r;
    q2 += r * r;
  }
  double a = block_sum256(q1, sh);
  double b = block_sum256(q2, sh);
  if (threadIdx.x == 0) {
    put_partial(d, inst, 1, a);
    put_partial(d, inst, 2, b);
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S.omega = om;
    S.iters += 1;
  }
}

// End-of-iteration test for every instance: converged (or out of
// iterations) instances are marked done; the graph's while-condition is set
// to "some instance still iterating".
__global__ void k_bicg_check(DevPtrs d, cudaGraphConditionalHandle h, int use_handle) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int inst = threadIdx.x; inst < d.n_inst; inst += blockDim.x) {
    SolverState& S = d.sol[inst];
    const Inst& I = d.inst[inst];
    if (S.done) continue;
    double bn = sum_partials(d, inst, 0), rn = sum_partials(d, inst, 2);
    bool conv = rn <= fmax(I.tol * I.tol * bn, S.eta2 * S.rn0);
    bool bad = !(rn == rn);
    if (conv || bad || S.iters >= I.max_iter) {
      S.done = 1;
      S.res = bn > 0.0 ? sqrt(rn / bn) : 0.0;
      if (!conv) atomicOr(d.err, bad ? kErrNonFinite : kErrNotConverged);
    } else {
      S.res = bn > 0.0 ? sqrt(rn / bn) : 0.0;
      atomicOr(&any, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    d.cnt[0] += 1;
    if (use_handle) cudaGraphSetConditional(h, any ? 1u : 0u);
  }
}

template <class Real>
void vcycle(const DevPtrs& d, const SolvePlan& pl, cudaStream_t s) {
  const size_t R = sizeof(Real);
  auto smooth = [&](int l, int which) {
    for (int dir = 0; dir < 2; ++dir)
      for (int color = 0; color < 2; ++color) {
        if (pl.smooth_split && dir != which) continue;
        int nb = dir == 0 ? pl.x1_blocks[l] : pl.x2_blocks[l];
        int k = dir == 0 ? pl.x1_k[l] : pl.x2_k[l];
        size_t sm = (size_t)line_buf(k) * R;
        k_xlines<Real><<<dim3(nb, d.n_inst), kLineThreads, sm, s>>>(d, l, color, dir);
      }
  };
  for (int l = 0; l < pl.max_tail; ++l) {
    smooth(l, 0);
    k_restrict<Real><<<dim3(pl.node_blocks[l + 1], d.n_inst), 256, 0, s>>>(d, l);
  }
  k_coarse<Real><<<dim3(64, d.n_inst), 256, 0, s>>>(d);
  for (int l = pl.max_tail - 1; l >= 0; --l) {
    k_prolong<Real><<<dim3(pl.node_blocks[l], d.n_inst), 256, 0, s>>>(d, l);
    smooth(l, 1);
  }
}

// ---------------------------------------------------------------------------
// The whole solve in one cooperative launch: the BiCGSTAB loop with every
// multigrid phase separated by a grid barrier instead of a kernel boundary.
// Every CTA computes the same per-instance scalars from the same partial sums
// (fixed order), so all CTAs take the same branches.
// ---------------------------------------------------------------------------

template <class Real>
__device__ bool coop_vcycle(const DevPtrs& d, const SolvePlan& pl, int nb, const int* done, unsigned char* smem) {
  Real* buf = (Real*)smem;
  BlockGroup g;
  auto smooth = [&](int l, int which) -> bool {
    for (int dir = 0; dir < 2; ++dir)
      for (int color = 0; color < 2; ++color) {
        if (pl.smooth_split && dir != which) continue;
        for (int inst = 0; inst < d.n_inst; ++inst) {
          const Inst& I = d.inst[inst];
          if (done[inst] || l >= I.tail_level) continue;
          LevelView<Real> v = view<Real>(d, I, l);
          int lines = dir == 0 ? v.n2 / 2 + 1 : v.n1 / 2;
          int K = dir == 0 ? k_for(v.n1 - 1) : k_for(v.n2 + 1);
          for (int w = blockIdx.x; w < lines; w += nb) {
            if (dir == 0) x1_pass(v, color, w, buf, K, g);
            else x2_pass(v, color, w, buf, K, g);
          }
        }
        if (!grid_sync(d, nb)) return false;
      }
    return true;
  };
  for (int l = 0; l < pl.max_tail; ++l) {
    if (!smooth(l, 0)) return false;
    for (int inst = 0; inst < d.n_inst; ++inst) {
      const Inst& I = d.inst[inst];
      if (done[inst] || l >= I.tail_level) continue;
      LevelView<Real> F = view<Real>(d, I, l), Cc = view<Real>(d, I, l + 1);
      for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < Cc.nodes;
           nd += (long long)nb * blockDim.x)
        restrict_node(F, Cc, nd);
    }
    if (!grid_sync(d, nb)) return false;
  }
  for (int inst = 0; inst < d.n_inst; ++inst)
    if (!done[inst])
      coarse_rows<Real>(d, d.inst[inst], (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5),
                        (long long)nb * (blockDim.x >> 5));
  if (!grid_sync(d, nb)) return false;
  for (int l = pl.max_tail - 1; l >= 0; --l) {
    for (int inst = 0; inst < d.n_inst; ++inst) {
      const Inst& I = d.inst[inst];
      if (done[inst] || l >= I.tail_level) continue;
      LevelView<Real> F = view<Real>(d, I, l), Cc = view<Real>(d, I, l + 1);
      for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < F.nodes;
           nd += (long long)nb * blockDim.x)
        prolong_node(F, Cc, nd);
    }
    if (!grid_sync(d, nb)) return false;
    if (!smooth(l, 1)) return false;
  }
  return true;
}

template <class Real>
__global__ void __launch_bounds__(kSolveThreads, 1) k_solve(DevPtrs d, SolvePlan pl) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ double sh[40];
  __shared__ int done[kCoopMaxInst];
  __shared__ double s_rho[kCoopMaxInst], s_rho_old[kCoopMaxInst], s_alpha[kCoopMaxInst], s_omega[kCoopMaxInst];
  __shared__ double s_bn[kCoopMaxInst];
  __shared__ double s_eta2[kCoopMaxInst], s_rn0[kCoopMaxInst];
  __shared__ int s_iters[kCoopMaxInst];
  const int nb = gridDim.x;
  const long long stride = (long long)nb * blockDim.x;
  auto put = [&](int inst, int slot, double v) {
    double t = block_sum_any(v, sh);
    if (threadIdx.x == 0) d.cred[((long long)inst * kNRed + slot) * kCoopMaxBlocks + blockIdx.x] = t;
  };
  // init: r = b - A x, rh = r, p = v = 0
  for (int inst = 0; inst < d.n_inst; ++inst) {
    const Inst& I = d.inst[inst];
    const bool nofield = (I.flags & APIC_NO_FIELD) != 0;
    if (threadIdx.x == 0) {
      done[inst] = nofield ? 1 : 0;
      if (nofield && blockIdx.x == 0) {
        d.sol[inst].res = 0.0;
        d.sol[inst].iters = 0;
        d.sol[inst].done = 1;
      }
      s_rho_old[inst] = 1.0;
      s_alpha[inst] = 1.0;
      s_omega[inst] = 1.0;
      s_iters[inst] = 0;
      s_eta2[inst] = d.sol[inst].eta2;
    }
    const double* st = d.st64 + (long long)kSt * I.node_off;
    const double* x = d.phi + I.node_off;
    double pr = 0.0;
    for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes; nd += stride) {
      int i = (int)(nd / I.N2), j = (int)(nd % I.N2);
      long long gi = I.node_off + nd;
      double r = 0.0;
      if (i > 0 && i < I.n1 && !nofield) r = d.b[gi] - apply_st<double, double>(st, I.nodes, x, nd, i, j, I.n2, I.N2, 1);
      d.r[gi] = r;
      d.rh[gi] = r;
      d.p[gi] = 0.0;
      d.v[gi] = 0.0;
      pr += r * r;
    }
    double t = block_sum_any(pr, sh);
    if (threadIdx.x == 0) {
      d.cred[((long long)inst * kNRed + 1) * kCoopMaxBlocks + blockIdx.x] = t;
      d.cred[((long long)inst * kNRed + 2) * kCoopMaxBlocks + blockIdx.x] = t;
    }
    // |b|^2 from the deposit kernel's partials (fixed order)
    if (threadIdx.x == 0) {
      const double* pb = d.red + ((long long)inst * kNRed + 0) * kRedBlocks;
      double bn = 0.0;
      for (int k = 0; k < kRedBlocks; ++k) bn += pb[k];
      s_bn[inst] = bn;
    }
  }
  if (!grid_sync(d, nb)) return;
  bool ok = true;
  for (int it = 0;; ++it) {
    // convergence test and p update
    int remaining = 0;
    for (int inst = 0; inst < d.n_inst; ++inst) {
      const Inst& I = d.inst[inst];
      if (done[inst]) continue;
      double rho = coop_sum(d, inst, 1, nb, sh), rn = coop_sum(d, inst, 2, nb, sh);
      double bn = s_bn[inst];
      if (it == 0 && threadIdx.x == 0) s_rn0[inst] = rn;
      __syncthreads();
      bool conv = rn <= fmax(I.tol * I.tol * bn, s_eta2[inst] * s_rn0[inst]);
      bool bad = !(rn == rn);
      __syncthreads();
      if (threadIdx.x == 0) {
        if (conv || bad || s_iters[inst] >= I.max_iter) {
          done[inst] = 1;
          if (blockIdx.x == 0) {
            d.sol[inst].res = bn > 0.0 ? sqrt(rn / bn) : 0.0;
            d.sol[inst].iters = s_iters[inst];
            d.sol[inst].done = 1;
            if (!conv) atomicOr(d.err, bad ? kErrNonFinite : kErrNotConverged);
          }
        }
        s_rho[inst] = rho;
      }
      __syncthreads();
      if (done[inst]) continue;
      ++remaining;
      double beta = (s_omega[inst] != 0.0 && s_rho_old[inst] != 0.0)
                        ? (rho / s_rho_old[inst]) * (s_alpha[inst] / s_omega[inst]) : 0.0;
      double om = s_omega[inst];
      const Level& L0 = I.lv[0];
      Real* f0 = (Real*)d.f + L0.off;
      Real* e0 = (Real*)d.e + L0.off;
      for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes; nd += stride) {
        long long gi = I.node_off + nd;
        double p = d.r[gi] + beta * (d.p[gi] - om * d.v[gi]);
        d.p[gi] = p;
        f0[nd] = (Real)p;
        e0[nd] = Real(0);
      }
    }
    if (remaining == 0) break;
    if (!(ok = grid_sync(d, nb))) break;
    for (int half = 0; half < 2 && ok; ++half) {
      if (!(ok = coop_vcycle<Real>(d, pl, nb, done, smem_raw))) break;
      // apply: z = M^-1 (.) from e0, y = A z
      for (int inst = 0; inst < d.n_inst; ++inst) {
        const Inst& I = d.inst[inst];
        if (done[inst]) continue;
        const Real* e0 = (const Real*)d.e + I.lv[0].off;
        const double* st = d.st64 + (long long)kSt * I.node_off;
        double* outz = half ? d.sh : d.ph;
        double* outy = half ? d.t : d.v;
        double q1 = 0.0, q2 = 0.0;
        for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes; nd += stride) {
          int i = (int)(nd / I.N2), j = (int)(nd % I.N2);
          long long gi = I.node_off + nd;
          double y = 0.0, z = 0.0;
          if (i > 0 && i < I.n1) {
            z = (double)e0[nd];
            y = apply_st<double, Real>(st, I.nodes, e0, nd, i, j, I.n2, I.N2, 1);
          }
          outz[gi] = z;
          outy[gi] = y;
          if (half) {
            q1 += y * d.s[gi];
            q2 += y * y;
          } else {
            q1 += d.rh[gi] * y;
          }
        }
        if (half) {
          put(inst, 4, q1);
          put(inst, 5, q2);
        } else {
          put(inst, 3, q1);
        }
      }
      if (!(ok = grid_sync(d, nb))) break;
      if (half == 0) {
        // alpha = rho / (rh, v); s = r - alpha v; f0 = s, e0 = 0
        for (int inst = 0; inst < d.n_inst; ++inst) {
          const Inst& I = d.inst[inst];
          if (done[inst]) continue;
          double den = coop_sum(d, inst, 3, nb, sh);
          double alpha = den != 0.0 ? s_rho[inst] / den : 0.0;
          if (threadIdx.x == 0) s_alpha[inst] = alpha;
          Real* f0 = (Real*)d.f + I.lv[0].off;
          Real* e0 = (Real*)d.e + I.lv[0].off;
          for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes; nd += stride) {
            long long gi = I.node_off + nd;
            double sv = d.r[gi] - alpha * d.v[gi];
            d.s[gi] = sv;
            f0[nd] = (Real)sv;
            e0[nd] = Real(0);
          }
        }
        if (!(ok = grid_sync(d, nb))) break;
      }
    }
    if (!ok) break;
    // omega = (t, s)/(t, t); x += alpha ph + omega sh; r = s - omega t
    for (int inst = 0; inst < d.n_inst; ++inst) {
      const Inst& I = d.inst[inst];
      if (done[inst]) continue;
      double ts = coop_sum(d, inst, 4, nb, sh), tt = coop_sum(d, inst, 5, nb, sh);
      double om = tt != 0.0 ? ts / tt : 0.0;
      double al = s_alpha[inst];
      double q1 = 0.0, q2 = 0.0;
      for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes; nd += stride) {
        int i = (int)(nd / I.N2);
        long long gi = I.node_off + nd;
        if (i > 0 && i < I.n1) d.phi[gi] += al * d.ph[gi] + om * d.sh[gi];
        double r = d.s[gi] - om * d.t[gi];
        d.r[gi] = r;
        q1 += d.rh[gi] * r;
        q2 += r * r;
      }
      put(inst, 1, q1);
      put(inst, 2, q2);
      if (threadIdx.x == 0) {
        s_omega[inst] = om;
        s_rho_old[inst] = s_rho[inst];
        s_iters[inst] += 1;
      }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) d.cnt[0] += 1;
    if (!(ok = grid_sync(d, nb))) break;
  }
}

}  // namespace

template <>
void launch_bicg_init<APIC_POISSON_REAL>(const DevPtrs& d, cudaStream_t s) {
  k_bicg_init<APIC_POISSON_REAL><<<dim3(kRedBlocks, d.n_inst), 256, 0, s>>>(d);
}

template <>
void launch_bicg_iter<APIC_POISSON_REAL>(const DevPtrs& d, const SolvePlan& pl, cudaStream_t s) {
  using Real = APIC_POISSON_REAL;
  dim3 g(kRedBlocks, d.n_inst);
  k_bicg_p<Real><<<g, 256, 0, s>>>(d, 0);
  vcycle<Real>(d, pl, s);
  k_bicg_apply<Real><<<g, 256, 0, s>>>(d, 0);
  k_bicg_s<Real><<<g, 256, 0, s>>>(d);
  vcycle<Real>(d, pl, s);
  k_bicg_apply<Real><<<g, 256, 0, s>>>(d, 1);
  k_bicg_x<Real><<<g, 256, 0, s>>>(d);
}

template <>
cudaError_t set_poisson_smem<APIC_POISSON_REAL>(const SolvePlan& pl) {
  using Real = APIC_POISSON_REAL;
  int most = 0;
  for (int l = 0; l < pl.max_tail; ++l) {
    int k = pl.x1_k[l] > pl.x2_k[l] ? pl.x1_k[l] : pl.x2_k[l];
    int b = line_buf(k) * (int)sizeof(Real);
    most = b > most ? b : most;
  }
  return cudaFuncSetAttribute(k_xlines<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, most > 0 ? most : 1024);
}

template <>
void launch_line_factor<APIC_POISSON_REAL>(const DevPtrs& d, int level, int dir, int lines, int kmax, cudaStream_t s) {
  using Real = APIC_POISSON_REAL;
  size_t sm = (size_t)4 * 96 * kmax * sizeof(Real);
  cudaFuncSetAttribute(k_line_factor<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_line_factor<Real><<<dim3((lines + 3) / 4, d.n_inst), 128, sm, s>>>(d, level, dir, kmax);
}

template <>
int coop_blocks<APIC_POISSON_REAL>(const SolvePlan& pl, int sms) {
  using Real = APIC_POISSON_REAL;
  int smem = pl.tail_bytes;
  int line = 0;
  for (int l = 0; l < pl.max_tail; ++l) {
    int k = pl.x1_k[l] > pl.x2_k[l] ? pl.x1_k[l] : pl.x2_k[l];
    line = line_buf(k) * (int)sizeof(Real) > line ? line_buf(k) * (int)sizeof(Real) : line;
  }
  smem = smem > line ? smem : line;
  if (cudaFuncSetAttribute(k_solve<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve<Real>, kSolveThreads, smem) != cudaSuccess) return 0;
  long long nb = (long long)per_sm * sms;
  return (int)(nb > kCoopMaxBlocks ? kCoopMaxBlocks : nb);
}

template <>
cudaError_t launch_solve_coop<APIC_POISSON_REAL>(const DevPtrs& d, const SolvePlan& pl, int blocks, cudaStream_t s) {
  using Real = APIC_POISSON_REAL;
  int smem = pl.tail_bytes;
  for (int l = 0; l < pl.max_tail; ++l) {
    int k = pl.x1_k[l] > pl.x2_k[l] ? pl.x1_k[l] : pl.x2_k[l];
    smem = line_buf(k) * (int)sizeof(Real) > smem ? line_buf(k) * (int)sizeof(Real) : smem;
  }
  DevPtrs dd = d;
  SolvePlan pp = pl;
  void* args[] = {&dd, &pp};
  return cudaLaunchCooperativeKernel((const void*)k_solve<Real>, dim3(blocks), dim3(kSolveThreads), args, (size_t)smem, s);
}

template <>
cudaError_t launch_dense_inverse<APIC_POISSON_REAL>(double* work, double* fbuf, int n, APIC_POISSON_REAL* out,
                                                    unsigned long long* cnt, int32_t* err,
                                                    unsigned long long wait_ns, cudaStream_t s) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_gj, 1024, 0);
  if (e != cudaSuccess) return e;
  if (per < 1) return cudaErrorCooperativeLaunchTooLarge;
  e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  void* args[] = {&work, &fbuf, &n, &cnt, &err, &wait_ns};
  e = cudaLaunchCooperativeKernel((const void*)k_gj, dim3(sms), dim3(1024), args, 0, s);
  if (e != cudaSuccess) return e;
  k_gj_store<APIC_POISSON_REAL><<<256, 256, 0, s>>>(work, n, out);
  return cudaGetLastError();
}

#if APIC_POISSON_COMMON
void launch_bicg_check(const DevPtrs& d, cudaGraphConditionalHandle h, int use_handle, cudaStream_t s) {
  k_bicg_check<<<1, 128, 0, s>>>(d, h, use_handle);
}
#endif

}  // namespace apic
