// Direct FP32 solver of the Poisson problem of Eqs. 6-7 (Sec. 2) inside an
// FP64 iterative refinement, for every instance of a batch in one
// cooperative launch.
//
// The finite-difference system of an instance is block tridiagonal in x1:
// row i of N2 unknowns couples to rows i - 1 and i + 1 through the blocks A_i
// and C_i and to itself through B_i.  Block cyclic reduction eliminates the
// odd rows, then the odd rows of what is left, and so on; the blocks of every
// level are formed once at set-up (FP64 on the host) and stored in FP32, and
// the few rows left after Lt levels are solved with a dense inverse.  Rows
// beyond n1 - 1 carry a zero correction, so any n1 works.  A solve is then a
// fixed sequence of phases of dense matrix-vector products whose tasks (one
// row of one instance each) are spread over the CTAs, one grid barrier per
// phase, instead of the dozens of line-relaxation phases per multigrid cycle.
// The refinement loop of each instance
//   r = b - A x (FP64),  e = (FP32 reduction) r,  x += e
// stops when |r| <= tol |b|; the FP32 reduction leaves about 1e-5 of the
// residual, so two passes reach 1e-10.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>

#include "apic_internal.h"

namespace apic {
namespace {

#include "solver_common.cuh"
#include "fields_common.cuh"

constexpr int kBcrThreads = 512;
constexpr int kBcrWarps = kBcrThreads / 32;
constexpr int kTailChunk = 16;      // tail rows per task at most (one per warp)
constexpr int kUpdRows = kBcrUpdRows;
constexpr int kRangesPerPass = kBcrThreads / kBcrSub;  // partial-sum ranges a CTA covers at once
static_assert(kRangesPerPass * kBcrSub == kBcrThreads, "whole ranges per pass");

// ---- bulk asynchronous copies (global -> shared, completion on an mbarrier) ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}


__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of the copy barrier (every thread).  On
// time-out the error word gets kErrTimeout, the copies still in flight are
// waited for (again bounded) and false is returned by every thread.
__device__ bool mbar_wait(uint64_t* bar, unsigned parity, int32_t* err) {
  bool ok = false;
  for (long long k = 0; k < (1ll << 22); ++k) {
    if (mbar_try_wait(bar, parity)) {
      ok = true;
      break;
    }
    if ((k & 1023) == 1023 && ((*(volatile int32_t*)err) & kErrTimeout)) break;
    __nanosleep(32);
  }
  if (!ok) {
    atomicOr(err, kErrTimeout);
    for (long long k = 0; k < (1ll << 22); ++k) {
      if (mbar_try_wait(bar, parity)) break;
      __nanosleep(64);
    }
  }
  return __syncthreads_and(ok) != 0;
}

// res = sum_t M_t v_t for NT column-major blocks (column stride Np) and
// vectors v_t in shared memory, by the whole CTA: warp w takes the columns
// w, w + kBcrWarps, ..., lane l the rows l + 32 m; the per-warp partial sums
// are added in warp order (the result does not depend on scheduling).
// kMC outputs per lane: blocks of up to 32 kMC unknowns.
template <int NT, bool kShared, int kMC>
__device__ __forceinline__ void task_mv(const float* const* Mt, const float* const* vt, int N, int Np, float* red,
                                        float* res) {
  // U columns per warp and block are loaded before their products, so that
  // U * NT * kMC loads per lane are in flight when the blocks stream from
  // global memory (about 64 values per lane: U = 8 / 4 / 2 for NT = 1 / 2 / 3
  // with 8 outputs per lane)
  constexpr int Ug = 64 / (NT * kMC) > 8 ? 8 : (64 / (NT * kMC) < 1 ? 1 : 64 / (NT * kMC));
  constexpr int U = kShared ? (Ug < 2 ? Ug : 2) : Ug;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float acc[kMC];
#pragma unroll
  for (int m = 0; m < kMC; ++m) acc[m] = 0.0f;
  for (int c0 = warp; c0 < N; c0 += U * kBcrWarps) {
    float v[U][NT][kMC], xs[U][NT];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int c = c0 + u * kBcrWarps;
      const bool ok = c < N;
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const float* col = Mt[t] + (long long)(ok ? c : 0) * Np;
        xs[u][t] = ok ? vt[t][c] : 0.0f;
#pragma unroll
        for (int m = 0; m < kMC; ++m) {
          const int j = lane + 32 * m;
          v[u][t][m] = ok && j < N ? (kShared ? col[j] : __ldg(col + j)) : 0.0f;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int t = 0; t < NT; ++t)
#pragma unroll
        for (int m = 0; m < kMC; ++m) acc[m] = fmaf(v[u][t][m], xs[u][t], acc[m]);
  }
#pragma unroll
  for (int m = 0; m < kMC; ++m) {
    const int j = lane + 32 * m;
    if (j < N) red[warp * N + j] = acc[m];
  }
  __syncthreads();
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    float s = 0.0f;
    for (int w = 0; w < kBcrWarps; ++w) s += red[w * N + j];
    res[j] = s;
  }
  __syncthreads();
}

struct Ctx {
  float* sbuf;  // dynamic shared memory: staged blocks or a tail chunk and its right-hand side
  uint64_t* bar;
  unsigned parity;
  float* red;
  float* sres;
  int32_t* err;
};

// res = sum_t src_t v_t: the blocks are staged in shared memory by one bulk
// copy each when the instance's blocks fit, else read from global memory.
// False on a copy time-out (every thread).
template <int NT, int kMC>
__device__ bool run_task(Ctx& c, const BcrInst& B, const float* const* src, const float* const* vt) {
  if (B.smem) {
    const unsigned bytes = (unsigned)(B.blk * sizeof(float));
    if (threadIdx.x == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(c.bar, bytes * NT);
#pragma unroll
      for (int t = 0; t < NT; ++t) bulk_g2s(c.sbuf + t * B.blk, src[t], bytes, c.bar);
    }
    if (!mbar_wait(c.bar, c.parity, c.err)) return false;
    c.parity ^= 1u;
    const float* Ms[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) Ms[t] = c.sbuf + t * B.blk;
    task_mv<NT, true, kMC>(Ms, vt, B.N, B.Np, c.red, c.sres);
  } else {
    task_mv<NT, false, kMC>(src, vt, B.N, B.Np, c.red, c.sres);
  }
  return true;
}

// Instance of task t of a phase: pre[k] <= t < pre[k + 1] (prefix in shared memory).
__device__ __forceinline__ int task_inst_s(const int* pre, int ni, int t) {
  int lo = 0, hi = ni - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Blocks (or tail rows) read by task q of kind `kind` at level l of instance
// B: up to three ranges (pointer, bytes); returns their count.
__device__ int task_ranges(const DevPtrs& d, const BcrInst& B, int kind, int l, int q, const float** p,
                           unsigned* bytes) {
  const float* blk = d.bcr + B.base;
  const unsigned bb = (unsigned)(B.blk * sizeof(float));
  switch (kind) {
    case kBcrFwd1:
    case kBcrBack1:
      p[0] = blk + (B.Binv[1] + q) * B.blk;
      bytes[0] = bb;
      return 1;
    case kBcrFwd:
      p[0] = blk + (B.P[l] + q) * B.blk;
      p[1] = blk + (B.Q[l] + q) * B.blk;
      bytes[0] = bytes[1] = bb;
      return 2;
    case kBcrBack:
      p[0] = blk + (B.Binv[l] + q) * B.blk;
      p[1] = blk + (B.G[l] + q) * B.blk;
      p[2] = blk + (B.H[l] + q) * B.blk;
      bytes[0] = bytes[1] = bytes[2] = bb;
      return 3;
    case kBcrTail: {
      const int r0 = q * B.tail_rows, r1 = min(B.tail_n, r0 + B.tail_rows);
      p[0] = d.bcr + B.tail + (long long)r0 * B.tail_np;
      bytes[0] = (unsigned)((r1 - r0) * B.tail_np * sizeof(float));
      return 1;
    }
    default: return 0;
  }
}

// Task q of kind `kind` at level l of instance k (the whole CTA).  Row r of
// the reduced right-hand side f and of the correction e is at (r - 1) N.
template <int MAXN>
__device__ bool run_stage(const DevPtrs& d, Ctx& c, const BcrInst& B, int kind, int l, int q, float (*sv)[MAXN],
                          float* fb, float* eb, double* xb) {
  constexpr int kMC = MAXN / 32;
  const int N = B.N, M = B.M;
  float* f = fb + B.foff;
  float* e = eb + B.foff;
  double* x = xb + B.node_off;
  const float* rp[3];
  unsigned rb[3];
  task_ranges(d, B, kind, l, q, rp, rb);
  switch (kind) {
    case kBcrFwd1: {  // y_k = B_k^-1 f_k, kept in e until the back substitution
      const int kr = 2 * q + 1;
      for (int j = threadIdx.x; j < N; j += blockDim.x) sv[0][j] = f[(long long)(kr - 1) * N + j];
      __syncthreads();
      const float* vt[1] = {sv[0]};
      if (!run_task<1, kMC>(c, B, rp, vt)) return false;
      for (int j = threadIdx.x; j < N; j += blockDim.x) e[(long long)(kr - 1) * N + j] = c.sres[j];
      __syncthreads();
      return true;
    }
    case kBcrUpd1: {  // f_i -= A_i y_{i-1} + C_i y_{i+1} (tridiagonal in j) on kUpdRows kept rows
      const float* st = (const float*)d.st + B.st_off;
      const long long nodes = B.nodes;
      const int nk = M / 2, q0 = q * kUpdRows, nq = min(kUpdRows, nk - q0);
      for (int o = threadIdx.x; o < nq * N; o += blockDim.x) {
        const int qq = o / N, j = o - qq * N, i = 2 * (q0 + qq + 1);
        const bool right = i + 1 <= M;
        const long long nd = (long long)i * N + j;
        float a = 0.0f;
#pragma unroll
        for (int dj = -1; dj <= 1; ++dj) {
          const int jj = j + dj;
          if (jj < 0 || jj >= N) continue;
          a = fmaf(st[st_slot(-1, dj) * nodes + nd], e[(long long)(i - 2) * N + jj], a);
          if (right) a = fmaf(st[st_slot(1, dj) * nodes + nd], e[(long long)i * N + jj], a);
        }
        f[(long long)(i - 1) * N + j] -= a;
      }
      return true;
    }
    case kBcrFwd: {  // f_i -= P f_{i-h} + Q f_{i+h}
      const int h = 1 << (l - 1), i = 2 * h * (q + 1);
      const bool right = i + h <= M;
      for (int j = threadIdx.x; j < N; j += blockDim.x) {
        sv[0][j] = f[(long long)(i - h - 1) * N + j];
        sv[1][j] = right ? f[(long long)(i + h - 1) * N + j] : 0.0f;
      }
      __syncthreads();
      const float* vt[2] = {sv[0], sv[1]};
      if (!run_task<2, kMC>(c, B, rp, vt)) return false;
      for (int j = threadIdx.x; j < N; j += blockDim.x) f[(long long)(i - 1) * N + j] -= c.sres[j];
      __syncthreads();
      return true;
    }
    case kBcrTail: {  // e = T^-1 f on rows r0..r1 of the tail: one row per warp, lanes over the columns
      const int tn = B.tail_n, tnp = B.tail_np, hs = 1 << B.Lt;
      const int r0 = q * B.tail_rows, r1 = min(tn, r0 + B.tail_rows);
      float* rows = c.sbuf;
      float* fs = c.sbuf + (long long)B.tail_rows * tnp;
      if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(c.bar, rb[0]);
        bulk_g2s(rows, rp[0], rb[0], c.bar);
      }
      for (int o = threadIdx.x; o < tn; o += blockDim.x) {
        const int qq = o / N, j = o - qq * N;
        fs[o] = f[(long long)(hs * (qq + 1) - 1) * N + j];
      }
      if (!mbar_wait(c.bar, c.parity, c.err)) return false;
      c.parity ^= 1u;
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      for (int o = r0 + warp; o < r1; o += kBcrWarps) {
        const float* row = rows + (long long)(o - r0) * tnp;
        float a = 0.0f;
#pragma unroll 4
        for (int cc = lane; cc < tn; cc += 32) a = fmaf(row[cc], fs[cc], a);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(kFull, a, off);
        if (lane == 0) {
          const int qq = o / N, j = o - qq * N, i = hs * (qq + 1);
          e[(long long)(i - 1) * N + j] = a;
          x[(long long)i * N + j] += (double)a;
        }
      }
      __syncthreads();
      return true;
    }
    case kBcrBack: {  // e_k = B_k^-1 f_k - G e_{k-h} - H e_{k+h}; x += e
      const int h = 1 << (l - 1), kr = h * (2 * q + 1);
      for (int j = threadIdx.x; j < N; j += blockDim.x) {
        sv[0][j] = f[(long long)(kr - 1) * N + j];
        sv[1][j] = kr - h >= 1 ? -e[(long long)(kr - h - 1) * N + j] : 0.0f;
        sv[2][j] = kr + h <= M ? -e[(long long)(kr + h - 1) * N + j] : 0.0f;
      }
      __syncthreads();
      const float* vt[3] = {sv[0], sv[1], sv[2]};
      if (!run_task<3, kMC>(c, B, rp, vt)) return false;
      for (int j = threadIdx.x; j < N; j += blockDim.x) {
        e[(long long)(kr - 1) * N + j] = c.sres[j];
        x[(long long)kr * N + j] += (double)c.sres[j];
      }
      __syncthreads();
      return true;
    }
    case kBcrBack1: {  // e_k = B_k^-1 (f_k - A_k e_{k-1} - C_k e_{k+1}); x += e
      const int kr = 2 * q + 1;
      const float* st = (const float*)d.st + B.st_off;
      const long long nodes = B.nodes;
      const bool left = kr - 1 >= 1, right = kr + 1 <= M;
      for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const long long nd = (long long)kr * N + j;
        float a = f[(long long)(kr - 1) * N + j];
#pragma unroll
        for (int dj = -1; dj <= 1; ++dj) {
          const int jj = j + dj;
          if (jj < 0 || jj >= N) continue;
          if (left) a = fmaf(-st[st_slot(-1, dj) * nodes + nd], e[(long long)(kr - 2) * N + jj], a);
          if (right) a = fmaf(-st[st_slot(1, dj) * nodes + nd], e[(long long)kr * N + jj], a);
        }
        sv[0][j] = a;
      }
      __syncthreads();
      const float* vt[1] = {sv[0]};
      if (!run_task<1, kMC>(c, B, rp, vt)) return false;
      for (int j = threadIdx.x; j < N; j += blockDim.x) {
        e[(long long)(kr - 1) * N + j] = c.sres[j];
        x[(long long)kr * N + j] += (double)c.sres[j];
      }
      __syncthreads();
      return true;
    }
  }
  return true;
}

// ---- nested dissection (BcrInst::nd) ----
// Dot products of matrix rows (row-major, 16-byte aligned rows of n4 float4)
// with a vector in shared memory: G lanes per row, 32 / G rows per warp at a
// time, partial sums added in a fixed butterfly (the result does not depend
// on the CTA or the batch).  fn(row, value) is called by the first lane of
// each row's group.
template <int G, class Fn>
__device__ __forceinline__ void rows_dot(const float* mat, int stride4, int row0, int row1, const float4* v, int n4,
                                         int lane, int first, int step, Fn fn) {
  const int gl = lane & (G - 1), gr = lane / G;
  for (int a0 = row0 + first * (32 / G); a0 < row1; a0 += step * (32 / G)) {
    const int a = a0 + gr;
    float acc = 0.0f;
    if (a < row1) {
      const float4* r = (const float4*)mat + (long long)a * stride4;
      for (int t = gl; t < n4; t += G) {
        const float4 m = __ldg(r + t), x = v[t];
        acc = fmaf(m.x, x.x, fmaf(m.y, x.y, fmaf(m.z, x.z, fmaf(m.w, x.w, acc))));
      }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if (a < row1 && gl == 0) fn(a, acc);
  }
}

template <class Fn>
__device__ __forceinline__ void rows_dot_any(int n4, const float* mat, int stride4, int row0, int row1, const float4* v,
                                             int lane, int first, int step, Fn fn) {
  if (n4 >= 32) rows_dot<32>(mat, stride4, row0, row1, v, n4, lane, first, step, fn);
  else if (n4 > 8) rows_dot<16>(mat, stride4, row0, row1, v, n4, lane, first, step, fn);
  else if (n4 > 4) rows_dot<8>(mat, stride4, row0, row1, v, n4, lane, first, step, fn);
  else if (n4 > 2) rows_dot<4>(mat, stride4, row0, row1, v, n4, lane, first, step, fn);
  else if (n4 > 1) rows_dot<2>(mat, stride4, row0, row1, v, n4, lane, first, step, fn);
  else rows_dot<1>(mat, stride4, row0, row1, v, n4, lane, first, step, fn);
}

// Rows of a tiny front by the 8-lane group that holds it (four fronts per
// warp): G lanes per row (G <= 8), 8 / G rows at a time, butterflies inside
// the group.  Every lane of the warp runs the same trip count (the largest
// row count of the warp's fronts, nrows_max) so the shuffles stay converged.
template <int G, class Fn>
__device__ __forceinline__ void rows_dot_grp(const float* mat, int stride4, int nrows, int nrows_max, const float4* v,
                                             int n4, int gl, Fn fn) {
  const int sl = gl & (G - 1), sr = gl / G;
  for (int a0 = 0; a0 < nrows_max; a0 += 8 / G) {
    const int a = a0 + sr;
    float acc = 0.0f;
    if (a < nrows) {
      const float4* r = (const float4*)mat + (long long)a * stride4;
      for (int t = sl; t < n4; t += G) {
        const float4 m = __ldg(r + t), x = v[t];
        acc = fmaf(m.x, x.x, fmaf(m.y, x.y, fmaf(m.z, x.z, fmaf(m.w, x.w, acc))));
      }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if (a < nrows && sl == 0) fn(a, acc);
  }
}

template <class Fn>
__device__ __forceinline__ void rows_dot_grp_any(int Gw, const float* mat, int stride4, int nrows, int nrows_max,
                                                 const float4* v, int n4, int gl, Fn fn) {
  if (Gw >= 8) rows_dot_grp<8>(mat, stride4, nrows, nrows_max, v, n4, gl, fn);
  else if (Gw >= 4) rows_dot_grp<4>(mat, stride4, nrows, nrows_max, v, n4, gl, fn);
  else if (Gw >= 2) rows_dot_grp<2>(mat, stride4, nrows, nrows_max, v, n4, gl, fn);
  else rows_dot_grp<1>(mat, stride4, nrows, nrows_max, v, n4, gl, fn);
}

__device__ __forceinline__ int warp_max(int x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(kFull, x, o));
  return x;
}

// Entry p of front F's assembled right-hand side: the residual at its node
// (separator positions only) plus what its children's update vectors hold
// for it, in the order child 0, child 1.
__device__ __forceinline__ float nd_rhs(const DevPtrs& d, const NdFront& F, int p, const float* f, const float* w) {
  const int2 g = *(const int2*)(d.nd_gather + F.G + 2 * p);  // absolute offsets into w (-1: none)
  float v = p < F.s ? f[d.nd_idx[F.S + p]] : 0.0f;
  if (g.x >= 0) v += w[g.x];
  if (g.y >= 0) v += w[g.y];
  return v;
}

// Forward rows [r0, r1) of front F with its v_S in vs (sp floats, zero
// padded): rows below s give z_S into e, the others W = v_U - M v_S.
__device__ __forceinline__ void nd_fwd_rows(const DevPtrs& d, const NdFront& F, int r0, int r1, const float* vs,
                                            const float* f, float* e, float* w, int lane, int first, int step) {
  rows_dot_any(F.sp >> 2, (const float*)d.bcr + F.FM, F.sp >> 2, r0, r1, (const float4*)vs, lane, first, step,
               [&](int a, float acc) {
                 if (a < F.s) e[d.nd_idx[F.S + a]] = acc;
                 else w[F.W + a - F.s] = nd_rhs(d, F, a, f, w) - acc;
               });
}

// Backward rows [r0, r1) of front F with x_U in xu (up floats, zero padded):
// x_S = z_S - N x_U into e, and x += e at the node.
__device__ __forceinline__ void nd_back_rows(const DevPtrs& d, const NdFront& F, int r0, int r1, const float* xu,
                                             float* e, double* x, int N, int lane, int first, int step) {
  auto put = [&](int a, float acc) {
    const int u = d.nd_idx[F.S + a];
    const float val = e[u] - acc;
    e[u] = val;
    x[(long long)u + N] += (double)val;
  };
  if (F.u == 0) {
    for (int a = r0 + first * 32 + lane; a < r1; a += step * 32) put(a, 0.0f);
    return;
  }
  rows_dot_any(F.up >> 2, (const float*)d.bcr + F.NB, F.up >> 2, r0, r1, (const float4*)xu, lane, first, step, put);
}

// One task of a nested-dissection phase of instance B: either rows
// [T.y, T.y + T.z) of the large front T.x (the whole CTA), or the T.z small
// fronts from T.x (one warp each, per-warp vectors in red).
__device__ bool run_nd(const DevPtrs& d, Ctx& c, const BcrInst& B, int kind, int l, int q, float* fb, float* eb,
                       double* xb, float* wb) {
  const float* f = fb + B.foff;
  float* e = eb + B.foff;
  double* x = xb + B.node_off;
  const int4 T = d.nd_task[(kind == kNdFwd ? B.nd_ft[l] : B.nd_bt[l]) + q];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (T.w == 0) {
    const NdFront F = d.nd_front[T.x];
    float* v = c.red;
    if (kind == kNdFwd) {
      for (int p = threadIdx.x; p < F.sp; p += blockDim.x) v[p] = p < F.s ? nd_rhs(d, F, p, f, wb) : 0.0f;
      __syncthreads();
      nd_fwd_rows(d, F, T.y, T.y + T.z, v, f, e, wb, lane, warp, kBcrWarps);
    } else {
      for (int p = threadIdx.x; p < F.up; p += blockDim.x) v[p] = p < F.u ? e[d.nd_idx[F.U + p]] : 0.0f;
      __syncthreads();
      nd_back_rows(d, F, T.y, T.y + T.z, v, e, x, B.N, lane, warp, kBcrWarps);
    }
    __syncthreads();
    return true;
  }
  if (T.w == 2) {
    // tiny fronts, four per warp: group g = lane / 8 takes front
    // T.x + 4 (warp + kBcrWarps i) + g, its vector at kNdTinyU floats of the
    // warp's area
    const int g = lane >> 3, gl = lane & 7;
    float* vg = c.red + warp * (kNdWarpMaxS + kNdWarpMaxU) + g * kNdTinyU;
    for (int k0 = 4 * warp; k0 < T.z; k0 += 4 * kBcrWarps) {
      const int k = k0 + g;
      const bool has = k < T.z;
      NdFront F;
      if (has) F = d.nd_front[T.x + k];
      const int len = !has ? 0 : (kind == kNdFwd ? F.sp : F.up);
      for (int p = gl; p < len; p += 8) {
        if (kind == kNdFwd) vg[p] = p < F.s ? nd_rhs(d, F, p, f, wb) : 0.0f;
        else vg[p] = p < F.u ? e[d.nd_idx[F.U + p]] : 0.0f;
      }
      __syncwarp();
      const int n4 = len >> 2;
      const int Gf = n4 <= 1 ? 1 : (n4 <= 2 ? 2 : (n4 <= 4 ? 4 : 8));
      const int Gw = warp_max(has ? Gf : 1);
      if (kind == kNdFwd) {
        const int nrows = has ? F.s + F.u : 0;
        rows_dot_grp_any(Gw, has ? (const float*)d.bcr + F.FM : (const float*)d.bcr, n4, nrows, warp_max(nrows),
                         (const float4*)vg, n4, gl, [&](int a, float acc) {
                           if (a < F.s) e[d.nd_idx[F.S + a]] = acc;
                           else wb[F.W + a - F.s] = nd_rhs(d, F, a, f, wb) - acc;
                         });
      } else {
        const int nrows = has ? F.s : 0;
        if (warp_max(has && F.u > 0 ? 1 : 0)) {
          rows_dot_grp_any(Gw, has ? (const float*)d.bcr + F.NB : (const float*)d.bcr, n4, nrows, warp_max(nrows),
                           (const float4*)vg, n4, gl, [&](int a, float acc) {
                             const int u = d.nd_idx[F.S + a];
                             const float val = e[u] - (F.u > 0 ? acc : 0.0f);
                             e[u] = val;
                             x[(long long)u + B.N] += (double)val;
                           });
        } else {
          for (int a = gl; a < nrows; a += 8) {
            const int u = d.nd_idx[F.S + a];
            x[(long long)u + B.N] += (double)e[u];
          }
        }
      }
      __syncwarp();
    }
    __syncthreads();
    return true;
  }
  // small fronts, one per warp (per-warp vector of kNdWarpMaxS + kNdWarpMaxU floats)
  float* v = c.red + warp * (kNdWarpMaxS + kNdWarpMaxU);
  for (int k = warp; k < T.z; k += kBcrWarps) {
    const NdFront F = d.nd_front[T.x + k];
    if (kind == kNdFwd) {
      for (int p = lane; p < F.sp; p += 32) v[p] = p < F.s ? nd_rhs(d, F, p, f, wb) : 0.0f;
      __syncwarp();
      nd_fwd_rows(d, F, 0, F.s + F.u, v, f, e, wb, lane, 0, 1);
    } else {
      for (int p = lane; p < F.up; p += 32) v[p] = p < F.u ? e[d.nd_idx[F.U + p]] : 0.0f;
      __syncwarp();
      nd_back_rows(d, F, 0, F.s, v, e, x, B.N, lane, 0, 1);
    }
    __syncwarp();
  }
  // the next task may be a large front's, whose vector overwrites the
  // per-warp areas: every warp finishes here first
  __syncthreads();
  return true;
}

// Fixed-order sum of part[r chunks + npre[k] .. r chunks + npre[k+1]) for
// every system v = r ni + k (right-hand side r < nrhs, instance k) with
// sel[v] (all when sel is null), one warp per system; out[v] in shared
// memory, the same in every CTA.
__device__ void inst_sums(const double* part, const int* npre, int ni, int nrhs, long long chunks, const int* sel,
                          double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int v = warp; v < nrhs * ni; v += kBcrWarps) {
    if (sel && !sel[v]) continue;
    const int r = v / ni, k = v - r * ni;
    const double* pr = part + (long long)r * chunks;
    double x = 0.0;
    for (int c = npre[k] + lane; c < npre[k + 1]; c += 32) x += pr[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(kFull, x, o);
    if (lane == 0) out[v] = x;
  }
  __syncthreads();
}

// Node tasks over the ranges of kBcrSub nodes of every instance (range c of
// instance k: nodes c kBcrSub .. (c + 1) kBcrSub - 1).  A task covers tsub
// consecutive ranges of one instance, kRangesPerPass per pass of the CTA; the tasks of
// all instances (and right-hand sides r < nrhs) are spread over the CTAs.
// body(r, k, I, nd) returns the node's contribution to its range's sum,
// which goes to part[r chunks + npre[k] + c] (when part
// is not null) as a warp-shuffle tree per warp and the range's warps in order: the
// sums do not depend on the task size, the CTA or the other instances of a
// batch.  ws: kBcrMaxTaskSub / kRangesPerPass * kBcrWarps doubles of shared memory.
template <class F>
__device__ void node_tasks(const DevPtrs& d, const int* npre, const int* tpre, int tsub, int nrhs, long long chunks,
                           const int* sel, double* part, double* ws, F body) {
  constexpr int kPasses = kBcrMaxTaskSub / kRangesPerPass;
  const int ni = d.n_inst, nb = gridDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int half = threadIdx.x / kBcrSub, r = threadIdx.x % kBcrSub;  // range within the pass, node within it
  const int per_rhs = tpre[ni], total = nrhs * per_rhs;
  for (int t = blockIdx.x; t < total; t += nb) {
    const int rh = t / per_rhs, tt = t - rh * per_rhs;
    const int k = task_inst_s(tpre, ni, tt);
    if (sel && !sel[rh * ni + k]) continue;
    const Inst& I = d.inst[k];
    const int s0 = (tt - tpre[k]) * tsub, s1 = min(npre[k + 1] - npre[k], s0 + tsub);
    double v[kPasses];
#pragma unroll
    for (int u = 0; u < kPasses; ++u) {
      const int sc = s0 + kRangesPerPass * u + half;
      const long long nd = (long long)sc * kBcrSub + r;
      v[u] = sc < s1 && nd < I.nodes ? body(rh, k, I, nd) : 0.0;
    }
    if (!part) continue;
#pragma unroll
    for (int u = 0; u < kPasses; ++u) {
      if (s0 + kRangesPerPass * u >= s1) break;
      double x = v[u];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(kFull, x, o);
      if (lane == 0) ws[u * kBcrWarps + warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < s1 - s0) {
      const int i = threadIdx.x, u = i / kRangesPerPass, w0 = (i % kRangesPerPass) * (kBcrSub / 32);
      double sum = 0.0;
      for (int w = w0; w < w0 + kBcrSub / 32; ++w) sum += ws[u * kBcrWarps + w];
      part[(long long)rh * chunks + npre[k] + s0 + i] = sum;
    }
    __syncthreads();
  }
}

// mode: kBcrRho = the step's density, initial guess and right-hand side are
// formed here (else b and its |b|^2 partials come from the caller);
// kBcrFields = node gradients and surface quantities after the solve.
// only >= 0: that instance alone is solved (the others keep their phi).
// rhs: the right-hand sides solved together (one for a step's solve: x = phi,
// b = DevPtrs::b).  An instance computes the same values alone or in a batch.
// MAXN: the largest block size of the batch this instantiation handles (256
// or 544 = 17 x 32, for grids up to 543 cells in x2).
template <int MAXN>
__global__ void __launch_bounds__(kBcrThreads, 1) k_solve_bcr(DevPtrs d, BcrPlan pl, int mode, int only, BcrRhs rhs) {
  extern __shared__ __align__(128) float s_dyn[];
  __shared__ double sh[40];
  __shared__ float sv[3][MAXN];
  __shared__ float sres[MAXN];
  __shared__ __align__(16) float red[kBcrWarps * MAXN];
  __shared__ double s_bn[kCoopMaxInst];
  __shared__ double s_rn[kCoopMaxInst];
  __shared__ int s_act[kCoopMaxInst];
  __shared__ int s_npre[kCoopMaxInst + 1];
  __shared__ int s_tpre[kCoopMaxInst + 1];
  __shared__ double s_ws[kBcrMaxTaskSub / kRangesPerPass * kBcrWarps];
  __shared__ int s_pre[kCoopMaxInst + 1];
  __shared__ int s_kind[kCoopMaxInst];
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ __align__(16) BcrInst s_b0;  // instance 0's table (one load per kernel instead of one per task)
  const int nb = gridDim.x, ni = d.n_inst, R = rhs.n, nv = R * ni;
  static_assert(kBcrMaxRhs == 3, "selections below");
  // selections instead of dynamic indexing (which would put the parameter
  // arrays in local memory)
  auto x_of = [&](int r) { return r == 0 ? rhs.x[0] : (r == 1 ? rhs.x[1] : rhs.x[2]); };
  auto b_of = [&](int r) { return r == 0 ? rhs.b[0] : (r == 1 ? rhs.b[1] : rhs.b[2]); };
  Ctx c{s_dyn, &s_bar, 0u, red, sres, d.err};
  double* part_b = d.bcr_part;                           // |b|^2 per range
  double* part_r = d.bcr_part + pl.chunks;  // |r|^2 per range and right-hand side ([kBcrMaxRhs][chunks])
  for (int k = threadIdx.x; k <= ni; k += blockDim.x) {
    s_npre[k] = d.bcr_npre[k];
    s_tpre[k] = d.bcr_tpre[k];
  }
  const int tsub = pl.task_sub;
  for (int v = threadIdx.x; v < nv; v += blockDim.x) s_act[v] = only < 0 || v % ni == only;
  if (threadIdx.x == 0) mbar_init(&s_bar, 1);
  for (int w = threadIdx.x; w < (int)(sizeof(BcrInst) / 4); w += blockDim.x)
    ((int*)&s_b0)[w] = ((const int*)d.bcr_inst)[w];
  // this thread's entries of the next phase's task tables, loaded before a
  // barrier and stored after it
  int r_pre = 0, r_kind = 0;
  auto load_tab = [&](int p) {
    if (threadIdx.x <= ni) {
      r_pre = __ldg(d.bcr_pre + (long long)p * (ni + 1) + threadIdx.x);
      r_kind = threadIdx.x < ni ? __ldg(d.bcr_kind + (long long)p * ni + threadIdx.x) : 0;
    }
  };
  auto store_tab = [&]() {
    if (threadIdx.x <= ni) {
      s_pre[threadIdx.x] = r_pre;
      if (threadIdx.x < ni) s_kind[threadIdx.x] = r_kind;
    }
  };
  __syncthreads();
  if (mode & kBcrRho) {
    // rho, the initial guess and b at every node; |b|^2 per instance
    node_tasks(d, s_npre, s_tpre, tsub, 1, pl.chunks, nullptr, part_b, s_ws,
               [&](int, int k, const Inst& I, long long nd) {
                 const double bv = rho_node(d, I, k, nd);
                 return bv * bv;
               });
    if (!grid_sync(d, nb)) return;
    inst_sums(part_b, s_npre, ni, 1, pl.chunks, nullptr, s_bn);
  } else {
    // |b|^2 from the right-hand-side kernels' partials (fixed order)
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
      const int r = v / ni, k = v - r * ni;
      const int slot = r == 0 ? rhs.slot[0] : (r == 1 ? rhs.slot[1] : rhs.slot[2]);
      const double* pr = d.red + ((long long)k * kNRed + slot) * kRedBlocks;
      double s0 = 0.0;
      for (int q = 0; q < kRedBlocks; ++q) s0 += pr[q];
      s_bn[v] = s0;
    }
    __syncthreads();
  }
  for (int it = 0;; ++it) {
    // FP64 residual of every instance still iterating, stored as the FP32
    // right-hand side of its reduction
    node_tasks(d, s_npre, s_tpre, tsub, R, pl.chunks, s_act, part_r, s_ws,
               [&](int rh, int k, const Inst& I, long long nd) {
                 const int N = I.N2;
                 const int i = (int)(nd / N), j = (int)(nd % N);
                 double rr = 0.0;
                 if (i > 0 && i < I.n1) {
                   const double r = b_of(rh)[I.node_off + nd] -
                                    apply_st<double, double>(d.st64 + (long long)kSt * I.node_off, I.nodes,
                                                             x_of(rh) + I.node_off, nd, i, j, I.n2, N, 1);
                   d.bcr_f[rh * pl.rows + d.bcr_inst[k].foff + (long long)(i - 1) * N + j] = (float)r;
                   rr = r * r;
                 }
                 return rr;
               });
    load_tab(0);
    if (!grid_sync(d, nb)) return;
    store_tab();  // read after the synchronisation that ends inst_sums
    inst_sums(part_r, s_npre, ni, R, pl.chunks, s_act, s_rn);
    int more = 0;
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
      if (!s_act[v]) continue;
      const int k = v % ni;
      const Inst& I = d.inst[k];
      const double rn = s_rn[v], bn = s_bn[v];
      const bool conv = rn <= I.tol * I.tol * bn, bad = !(rn == rn);
      if (conv || bad || it >= I.max_iter) {
        if (blockIdx.x == 0) {
          if (v < ni) {  // the first right-hand side reports the solver state
            SolverState& S = d.sol[k];
            S.res = bn > 0.0 ? sqrt(rn / bn) : 0.0;
            S.iters = it;
            S.done = 1;
          }
          if (!conv) atomicOr(d.err, bad ? kErrNonFinite : kErrNotConverged);
        }
        s_act[v] = 0;
      } else {
        more = 1;
      }
    }
    if (!__syncthreads_or(more)) break;
    // the reduction passes: phase p runs the p-th stage of every instance
    for (int p = 0; p < pl.phases; ++p) {
      if (p > 0) {  // the phase's task tables (loaded before the last barrier)
        store_tab();
        __syncthreads();
      }
      const int per_rhs = s_pre[ni], total = R * per_rhs;
      for (int t = blockIdx.x; t < total; t += nb) {
        const int rh = t / per_rhs, tt = t - rh * per_rhs;
        const int k = task_inst_s(s_pre, ni, tt);
        if (!s_act[rh * ni + k]) continue;
        const BcrInst& B = k == 0 ? s_b0 : d.bcr_inst[k];
        const int kind = s_kind[k] >> 8;
        if (kind == kNdFwd || kind == kNdBack) {
          if (!run_nd(d, c, B, kind, s_kind[k] & 255, tt - s_pre[k], d.bcr_f + rh * pl.rows, d.bcr_e + rh * pl.rows,
                      x_of(rh), d.nd_w + rh * pl.nd_wrows))
            return;
        } else if (!run_stage<MAXN>(d, c, B, kind, s_kind[k] & 255, tt - s_pre[k], sv, d.bcr_f + rh * pl.rows,
                                    d.bcr_e + rh * pl.rows, x_of(rh))) {
          return;
        }
      }
      if (p + 1 < pl.phases) load_tab(p + 1);
      if (!grid_sync(d, nb)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) d.cnt[0] += 1;
  }
  if (mode & kBcrFields) {
    // phi is final everywhere (the last pass ended at a grid barrier)
    node_tasks(d, s_npre, s_tpre, tsub, 1, pl.chunks, nullptr, nullptr, s_ws,
               [&](int, int, const Inst& I, long long nd) {
                 grad_node<float, float2>(d, I, nd);
                 return 0.0;
               });
    for (int k = nb - 1 - (int)blockIdx.x; k < ni; k += nb) surface_block(d, k, sh);
  }
}

constexpr int static_smem(int maxn) {
  return 40 * 8 + 3 * maxn * 4 + maxn * 4 + kBcrWarps * maxn * 4 + kCoopMaxInst * 36 + 12 +
         kBcrMaxTaskSub / kRangesPerPass * kBcrWarps * 8 + (int)sizeof(BcrInst) + 16 + 64;
}

const void* kernel_for(const BcrPlan& b) {
  return b.wide ? (const void*)k_solve_bcr<kBcrMaxNWide> : (const void*)k_solve_bcr<kBcrMaxN>;
}

// Check of the bounded grid-barrier wait: the CTAs wait at a barrier that
// expects one arrival more than there are CTAs, so no wait can complete; each
// gives up after d.wait_ns, sets the status word's time-out bit and returns.
__global__ void k_wait_check(DevPtrs d) { grid_sync(d, gridDim.x + 1u); }

}  // namespace

const void* bcr_kernel(const SolvePlan& pl) { return kernel_for(pl.bcr); }

void launch_wait_check(const DevPtrs& d, int blocks, cudaStream_t s) { k_wait_check<<<blocks, 32, 0, s>>>(d); }

int bcr_configure(SolvePlan& pl, BcrInst* bi, int ni, int sms) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int nb = sms < kCoopMaxBlocks ? sms : kCoopMaxBlocks;
  int widest = 0;
  for (int k = 0; k < ni; ++k)
    if (!bi[k].nd) widest = bi[k].N > widest ? bi[k].N : widest;
  // nested dissection uses the reduction buffer (kBcrWarps x MAXN floats) for
  // a large front's vector
  pl.bcr.wide = widest > kBcrMaxN || pl.bcr.nd_floats > kBcrWarps * kBcrMaxN ? 1 : 0;
  if (pl.bcr.nd_floats > kBcrWarps * kBcrMaxNWide) return 0;
  const long long budget = (long long)optin - static_smem(pl.bcr.wide ? kBcrMaxNWide : kBcrMaxN);
  const void* kern = kernel_for(pl.bcr);
  // tail chunks: about one per CTA when the tails are few, else one row per warp
  long long tail_total = 0;
  for (int k = 0; k < ni; ++k) tail_total += bi[k].tail_n;
  int rows = (int)((tail_total + nb - 1) / nb);
  rows = rows < 1 ? 1 : (rows > kTailChunk ? kTailChunk : rows);
  bool stage_ok = true;
  if (const char* e = std::getenv("APIC_BCR_STAGE")) stage_ok = std::atoi(e) != 0;
  long long dyn = 0;
  int any = 0;
  for (int k = 0; k < ni; ++k) {
    BcrInst& B = bi[k];
    B.tail_rows = rows;
    while (B.tail_rows > 1 && (long long)(B.tail_rows + 1) * B.tail_np * 4 > budget) --B.tail_rows;
    const long long tail = (long long)(B.tail_rows + 1) * B.tail_np * 4;  // rows + right-hand side
    if (tail > budget) return 0;
    dyn = tail > dyn ? tail : dyn;
    const long long staged = 3ll * B.blk * (long long)sizeof(float);
    // staging pays when the blocks come from L2; streamed from DRAM the
    // direct loads keep more bytes in flight
    B.smem = stage_ok && pl.bcr.resident && staged <= budget ? 1 : 0;
    if (B.smem) {
      any = 1;
      dyn = staged > dyn ? staged : dyn;
    }
  }
  pl.bcr.smem = any;
  pl.bcr.dyn = (int)dyn;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBcrThreads, (size_t)dyn) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (per_sm < 1) return 0;
  return nb;
}

static cudaError_t launch_bcr(const DevPtrs& d, const SolvePlan& pl, int blocks, int mode, int only, const BcrRhs& rhs,
                              cudaStream_t s) {
  DevPtrs dd = d;
  BcrPlan pp = pl.bcr;
  BcrRhs rr = rhs;
  int mm = mode, oo = only;
  void* args[] = {&dd, &pp, &mm, &oo, &rr};
  return cudaLaunchCooperativeKernel(kernel_for(pl.bcr), dim3(blocks), dim3(kBcrThreads), args,
                                     (size_t)pl.bcr.dyn, s);
}

cudaError_t launch_solve_bcr(const DevPtrs& d, const SolvePlan& pl, int blocks, int mode, int only, cudaStream_t s) {
  BcrRhs one{};
  one.n = 1;
  one.slot[0] = 0;
  one.x[0] = d.phi;
  one.b[0] = d.b;
  return launch_bcr(d, pl, blocks, mode, only, one, s);
}

cudaError_t launch_solve_bcr_rhs(const DevPtrs& d, const SolvePlan& pl, int blocks, const BcrRhs& rhs, cudaStream_t s) {
  if (rhs.n < 1 || rhs.n > kBcrMaxRhs || rhs.n * d.n_inst > kCoopMaxInst) return cudaErrorInvalidValue;
  return launch_bcr(d, pl, blocks, 0, -1, rhs, s);
}

}  // namespace apic
