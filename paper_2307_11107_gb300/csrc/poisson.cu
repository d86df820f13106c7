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
//   * the coarse levels (<= kTailNodes nodes) run in one CTA per instance, the
//     coarsest level is a dense inverse.
// All dot products are per-CTA partials summed in a fixed order, so results
// do not depend on scheduling.  Every kernel checks the per-instance `done`
// flag, so a fixed launch sequence (CUDA-graph friendly) stops doing work once
// the tolerance is met.
#include <cuda_runtime.h>

#include <cstdint>

#include "apic_internal.h"

namespace apic {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kLineWarps = 4;   // warps (lines) per CTA in the multi-CTA line kernels
constexpr int kTailThreads = 512;

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

__device__ __forceinline__ void put_partial(const DevPtrs& d, int inst, int slot, double v) {
  d.red[((long long)inst * kNRed + slot) * kRedBlocks + blockIdx.x] = v;
}

// y = A x at node (i, j) of a level with stencil `st` (kSt arrays of `nodes`).
// Entries towards Dirichlet rows are stored as zero.
template <class S, class V>
__device__ __forceinline__ S apply_st(const S* st, long long nodes, const V* x, long long nd, int i, int j, int n2,
                                      int N2, int pole) {
  S acc = S(0);
#pragma unroll
  for (int di = -1; di <= 1; ++di) {
#pragma unroll
    for (int dj = -1; dj <= 1; ++dj) {
      if ((dj < 0 && j == 0) || (dj > 0 && j == n2)) continue;
      S c = st[st_slot(di, dj) * nodes + nd];
      acc += c * (S)x[nd + (long long)di * N2 + dj];
    }
  }
  if (pole) {
    if (j == 0) acc += st[kStPole * nodes + nd] * (S)x[nd + 2];
    else if (j == n2) acc += st[kStPole * nodes + nd] * (S)x[nd - 2];
  }
  (void)i;
  return acc;
}

// ---------------------------------------------------------------------------
// Warp tridiagonal solver.  Row r of the line lives in smem slot
// (r - lane*K) * 32 + lane (lane = r / K): conflict-free per-lane chunks.
// On entry a, b, c, d hold sub-, main-, super-diagonal and right-hand side;
// on exit d holds the solution.
// ---------------------------------------------------------------------------
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
// Level operations (one line / one node at a time); used by the multi-CTA
// kernels and by the single-CTA tail.
// ---------------------------------------------------------------------------
template <class Real>
struct LevelView {
  const Real* st;
  Real* e;
  const Real* f;
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
  return v;
}

template <class Real>
__device__ __forceinline__ Real resid_at(const LevelView<Real>& v, int i, int j) {
  long long nd = (long long)i * v.N2 + j;
  return v.f[nd] - apply_st<Real, Real>(v.st, v.nodes, v.e, nd, i, j, v.n2, v.N2, v.pole);
}

// x1-line j (unknowns i = 1..n1-1) solved exactly for the correction, by one warp.
template <class Real>
__device__ void relax_x1_line(const LevelView<Real>& v, int j, Real* buf, int K) {
  const int lane = threadIdx.x & 31;
  const int n = v.n1 - 1;
  Real* a = buf;
  Real* b = buf + 32 * K;
  Real* c = buf + 64 * K;
  Real* dd = buf + 96 * K;
  for (int r = lane; r < n; r += 32) {
    int i = r + 1;
    long long nd = (long long)i * v.N2 + j;
    int s = lslot(r, K);
    a[s] = v.st[st_slot(-1, 0) * v.nodes + nd];
    b[s] = v.st[st_slot(0, 0) * v.nodes + nd];
    c[s] = v.st[st_slot(1, 0) * v.nodes + nd];
    dd[s] = resid_at(v, i, j);
  }
  __syncwarp();
  warp_tridiag(a, b, c, dd, n, K);
  for (int r = lane; r < n; r += 32) {
    long long nd = (long long)(r + 1) * v.N2 + j;
    v.e[nd] += dd[lslot(r, K)];
  }
  __syncwarp();
}

// x2-line i (unknowns j = 0..n2), pole reaches eliminated with the neighbour row.
template <class Real>
__device__ void relax_x2_line(const LevelView<Real>& v, int i, Real* buf, int K) {
  const int lane = threadIdx.x & 31;
  const int n = v.n2 + 1;
  Real* a = buf;
  Real* b = buf + 32 * K;
  Real* c = buf + 64 * K;
  Real* dd = buf + 96 * K;
  long long base = (long long)i * v.N2;
  for (int r = lane; r < n; r += 32) {
    long long nd = base + r;
    int s = lslot(r, K);
    a[s] = r > 0 ? v.st[st_slot(0, -1) * v.nodes + nd] : Real(0);
    b[s] = v.st[st_slot(0, 0) * v.nodes + nd];
    c[s] = r < v.n2 ? v.st[st_slot(0, 1) * v.nodes + nd] : Real(0);
    dd[s] = resid_at(v, i, r);
  }
  __syncwarp();
  if (v.pole && lane == 0) {
    int s0 = lslot(0, K), s1 = lslot(1, K);
    Real e0 = v.st[kStPole * v.nodes + base];
    Real g = e0 / c[s1];
    b[s0] -= g * a[s1];
    c[s0] -= g * b[s1];
    dd[s0] -= g * dd[s1];
    int sn = lslot(v.n2, K), sm = lslot(v.n2 - 1, K);
    Real en = v.st[kStPole * v.nodes + base + v.n2];
    Real h = en / a[sm];
    b[sn] -= h * c[sm];
    a[sn] -= h * b[sm];
    dd[sn] -= h * dd[sm];
  }
  __syncwarp();
  warp_tridiag(a, b, c, dd, n, K);
  for (int r = lane; r < n; r += 32) v.e[base + r] += dd[lslot(r, K)];
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

template <class Real>
__device__ void x1_pass(const LevelView<Real>& v, int color, int w, Real* buf, int K) {
  int second;
  int j = x1_line_of(w, color, v.n2, v.pole, &second);
  if (j < 0) return;
  relax_x1_line(v, j, buf, K);
  if (second >= 0) relax_x1_line(v, second, buf, K);
}

template <class Real>
__device__ void x2_pass(const LevelView<Real>& v, int color, int w, Real* buf, int K) {
  int i = 1 + 2 * w + color;
  if (i > v.n1 - 1) return;
  relax_x2_line(v, i, buf, K);
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

__device__ __forceinline__ int k_for(int n) { return (n + 31) / 32; }

// ---------------------------------------------------------------------------
// Kernels.
// ---------------------------------------------------------------------------
template <class Real>
__global__ void __launch_bounds__(kLineWarps * 32) k_xlines(DevPtrs d, int l, int color, int dir) {
  extern __shared__ unsigned char smem_raw[];
  const int inst = blockIdx.y;
  const Inst& I = d.inst[inst];
  if (d.sol[inst].done || l >= I.tail_level) return;
  LevelView<Real> v = view<Real>(d, I, l);
  int K = dir == 0 ? k_for(v.n1 - 1) : k_for(v.n2 + 1);
  int warp = threadIdx.x >> 5;
  Real* buf = (Real*)smem_raw + (long long)warp * 128 * K;
  int w = blockIdx.x * kLineWarps + warp;
  if (dir == 0) x1_pass(v, color, w, buf, K);
  else x2_pass(v, color, w, buf, K);
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

// Coarse levels l >= tail_level of one instance, entirely inside one CTA.
template <class Real>
__global__ void __launch_bounds__(kTailThreads) k_tail(DevPtrs d) {
  extern __shared__ unsigned char smem_raw[];
  const int inst = blockIdx.x;
  const Inst& I = d.inst[inst];
  if (d.sol[inst].done) return;
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5;
  const int L0 = I.tail_level, Lc = I.n_levels - 1;
  int Kmax = 1;
  for (int l = L0; l <= Lc; ++l) {
    int k1 = k_for(I.lv[l].n1 - 1), k2 = k_for(I.lv[l].n2 + 1);
    Kmax = k1 > Kmax ? k1 : Kmax;
    Kmax = k2 > Kmax ? k2 : Kmax;
  }
  Real* buf = (Real*)smem_raw + (long long)warp * 128 * Kmax;
  auto smooth = [&](const LevelView<Real>& v) {
    int K1 = k_for(v.n1 - 1), K2 = k_for(v.n2 + 1);
    for (int color = 0; color < 2; ++color) {
      for (int w = warp; 2 * w + color <= v.n2; w += nw) x1_pass(v, color, w, buf, K1);
      __syncthreads();
    }
    for (int color = 0; color < 2; ++color) {
      for (int w = warp; 1 + 2 * w + color <= v.n1 - 1; w += nw) x2_pass(v, color, w, buf, K2);
      __syncthreads();
    }
  };
  for (int l = L0; l < Lc; ++l) {
    LevelView<Real> F = view<Real>(d, I, l), Cc = view<Real>(d, I, l + 1);
    smooth(F);
    for (long long nd = threadIdx.x; nd < Cc.nodes; nd += blockDim.x) restrict_node(F, Cc, nd);
    __syncthreads();
  }
  {
    // coarsest: e = Cinv f over the unknowns (rows 1..n1-1, all j)
    LevelView<Real> C = view<Real>(d, I, Lc);
    const Real* cinv = (const Real*)d.cinv + I.cinv_off;
    int nu = I.coarse_n;
    for (int u = threadIdx.x; u < nu; u += blockDim.x) {
      Real acc = Real(0);
      for (int k = 0; k < nu; ++k) acc += cinv[(long long)u * nu + k] * C.f[C.N2 + k];
      C.e[C.N2 + u] = acc;
    }
    __syncthreads();
  }
  for (int l = Lc - 1; l >= L0; --l) {
    LevelView<Real> F = view<Real>(d, I, l), Cc = view<Real>(d, I, l + 1);
    for (long long nd = threadIdx.x; nd < F.nodes; nd += blockDim.x) prolong_node(F, Cc, nd);
    __syncthreads();
    smooth(F);
  }
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
  double bn = sum_partials(d, inst, 0), rho = sum_partials(d, inst, 1), rn = sum_partials(d, inst, 2);
  double tol2 = I.tol * I.tol;
  bool conv = rn <= tol2 * bn || !(rn == rn);
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
  if (blockIdx.x == 0 && threadIdx.x == 0) S.rho = rho;
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
  double den = sum_partials(d, inst, 3);
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
  double ts = sum_partials(d, inst, 4), tt = sum_partials(d, inst, 5);
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
    bool conv = rn <= I.tol * I.tol * bn;
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
  auto smooth = [&](int l) {
    for (int dir = 0; dir < 2; ++dir)
      for (int color = 0; color < 2; ++color) {
        int nb = dir == 0 ? pl.x1_blocks[l] : pl.x2_blocks[l];
        int k = dir == 0 ? pl.x1_k[l] : pl.x2_k[l];
        size_t sm = (size_t)kLineWarps * 128 * k * R;
        k_xlines<Real><<<dim3(nb, d.n_inst), kLineWarps * 32, sm, s>>>(d, l, color, dir);
      }
  };
  for (int l = 0; l < pl.max_tail; ++l) {
    smooth(l);
    k_restrict<Real><<<dim3(pl.node_blocks[l + 1], d.n_inst), 256, 0, s>>>(d, l);
  }
  k_tail<Real><<<d.n_inst, pl.tail_threads, (size_t)(pl.tail_threads / 32) * 128 * pl.tail_k * R, s>>>(d);
  for (int l = pl.max_tail - 1; l >= 0; --l) {
    k_prolong<Real><<<dim3(pl.node_blocks[l], d.n_inst), 256, 0, s>>>(d, l);
    smooth(l);
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
    int b = kLineWarps * 128 * k * (int)sizeof(Real);
    most = b > most ? b : most;
  }
  cudaError_t e = cudaFuncSetAttribute(k_xlines<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, most > 0 ? most : 1024);
  if (e != cudaSuccess) return e;
  int tb = (pl.tail_threads / 32) * 128 * pl.tail_k * (int)sizeof(Real);
  return cudaFuncSetAttribute(k_tail<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, tb > 0 ? tb : 1024);
}

#if APIC_POISSON_COMMON
void launch_bicg_check(const DevPtrs& d, cudaGraphConditionalHandle h, int use_handle, cudaStream_t s) {
  k_bicg_check<<<1, 128, 0, s>>>(d, h, use_handle);
}
#endif

}  // namespace apic
