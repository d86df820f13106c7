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
#include "bulk_copy.cuh"

constexpr int kBcrThreads = 512;
constexpr int kBcrWarps = kBcrThreads / 32;
constexpr int kTailChunk = 16;      // tail rows per task at most (one per warp)
constexpr int kUpdRows = kBcrUpdRows;
constexpr int kRangesPerPass = kBcrThreads / kBcrSub;  // partial-sum ranges a CTA covers at once
// shared memory of the nested-dissection tasks (the wide kernel's reduction
// buffer, kBcrWarps x kBcrMaxNWide floats): a large front's vector
// (kNdVecCap floats) and its task's rows after it; a small front's v_S, z_S
// and U rows (kNdWarpArea floats per warp); a tiny front's (kNdTinyArea per
// 8-lane group, four groups per warp)
constexpr int kNdVecCap = kBcrWarps * kBcrMaxNWide - kNdTaskRows;
static_assert(kNdStageFloats == kBcrWarps * kNdWarpStage && kNdTaskFronts * kNdUnits == kBcrWarps, "one front per warp");
// per-warp area, forward: v_S, z_S, the U rows, the separator's node indices;
// backward: x_U, N x_U, the separator's node indices, z_S, x (doubles)
constexpr int kNdWarpArea = 8 * kNdWarpMaxS;   // 512 floats
constexpr int kNdTinyArea = 8 * kNdTinyS;      // 128 floats, four groups per warp
static_assert(kNdWarpMaxU == 3 * kNdWarpMaxS && kNdTinyU == 3 * kNdTinyS, "area layout");
static_assert(kNdWarpArea <= kBcrMaxNWide && 4 * kNdTinyArea <= kNdWarpArea && kNdTinyArea % 4 == 0, "areas");
static_assert(kRangesPerPass * kBcrSub == kBcrThreads, "whole ranges per pass");

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
// Every task runs in three stages, each a round of independent loads: (1) the
// vectors (v_S and the U rows' right-hand sides forward, x_U backward) into
// shared memory; (2) the matrix rows' dot products into shared memory; (3)
// the results scattered to their nodes.  No load waits on another except the
// index-then-value pairs of the gathers, which are issued in batches.

// Dot products of matrix rows staged in shared memory (row-major, 16-byte
// aligned rows of n4 float4; row a at mat + (a - base) stride4 float4) with a
// vector in shared memory: G lanes per row, 32 / G rows per warp pass and U
// passes in flight, partial sums added in a fixed butterfly (the result does
// not depend on the CTA or the batch).  Rows past row1 load the last row
// (branch-free loads) and are not reported.  fn(row, value) is called by the
// first lane of each row's group.
template <int G, class Fn>
__device__ __forceinline__ void rows_dot(const float* mat, int stride4, int row0, int row1, int base, const float4* v,
                                         int n4, int lane, int first, int step, Fn fn) {
  constexpr int R = 32 / G, U = G >= 16 ? 2 : 4;
  const int gl = lane & (G - 1), gr = lane / G;
  const int pass = step * R;
  const float4* m4 = (const float4*)mat;
  for (int a0 = row0 + first * R; a0 < row1; a0 += U * pass) {
    float acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] = 0.0f;
    for (int t = gl; t < n4; t += G) {
      const float4 x = v[t];
      float4 m[U];
#pragma unroll
      for (int u = 0; u < U; ++u) m[u] = m4[(long long)(min(a0 + u * pass + gr, row1 - 1) - base) * stride4 + t];
#pragma unroll
      for (int u = 0; u < U; ++u)
        acc[u] = fmaf(m[u].x, x.x, fmaf(m[u].y, x.y, fmaf(m[u].z, x.z, fmaf(m[u].w, x.w, acc[u]))));
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) acc[u] += __shfl_xor_sync(kFull, acc[u], o);
      const int a = a0 + u * pass + gr;
      if (a < row1 && gl == 0) fn(a, acc[u]);
    }
  }
}

template <class Fn>
__device__ __forceinline__ void rows_dot_any(int n4, const float* mat, int stride4, int row0, int row1, int base,
                                             const float4* v, int lane, int first, int step, Fn fn) {
  if (n4 > 16) rows_dot<32>(mat, stride4, row0, row1, base, v, n4, lane, first, step, fn);
  else if (n4 > 8) rows_dot<16>(mat, stride4, row0, row1, base, v, n4, lane, first, step, fn);
  else if (n4 > 4) rows_dot<8>(mat, stride4, row0, row1, base, v, n4, lane, first, step, fn);
  else rows_dot<4>(mat, stride4, row0, row1, base, v, n4, lane, first, step, fn);
}

// Rows of a tiny front by the 8-lane group that holds it (four fronts per
// warp): G lanes per row (G <= 8), 8 / G rows per group pass, four passes in
// flight, butterflies inside the group.  Every lane of the warp runs the same
// trip count (the largest row count of the warp's fronts, nrows_max) so the
// shuffles stay converged; a group without rows (nrows = 0) loads nothing.
template <int G, class Fn>
__device__ __forceinline__ void rows_dot_grp(const float* mat, int stride4, int nrows, int nrows_max, const float4* v,
                                             int n4, int gl, Fn fn) {
  constexpr int R = 8 / G, U = 4;
  const int sl = gl & (G - 1), sr = gl / G;
  const float4* m4 = (const float4*)mat;
  const int n4g = nrows > 0 ? n4 : 0;
  for (int a0 = 0; a0 < nrows_max; a0 += U * R) {
    float acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] = 0.0f;
    for (int t = sl; t < n4g; t += G) {
      const float4 x = v[t];
      float4 m[U];
#pragma unroll
      for (int u = 0; u < U; ++u) m[u] = m4[(long long)min(a0 + u * R + sr, nrows - 1) * stride4 + t];
#pragma unroll
      for (int u = 0; u < U; ++u)
        acc[u] = fmaf(m[u].x, x.x, fmaf(m[u].y, x.y, fmaf(m[u].z, x.z, fmaf(m[u].w, x.w, acc[u]))));
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) acc[u] += __shfl_xor_sync(kFull, acc[u], o);
      const int a = a0 + u * R + sr;
      if (a < nrows && sl == 0) fn(a, acc[u]);
    }
  }
}

__device__ __forceinline__ int warp_max(int x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(kFull, x, o));
  return x;
}

// out[k] = entry p0 + k of front F's assembled right-hand side for k < n
// (pad: zeros up to n_pad), by the threads `lane` + multiples of `stride`:
// the residual at its node (separator positions p < s only) plus what its
// children's update vectors hold for it, child 0 then child 1.  Four
// entries per thread in flight: their table entries first, then the values.
__device__ __forceinline__ void nd_rhs_into(const DevPtrs& d, const NdFront& F, int p0, int n, int n_pad, float* out,
                                            const float* f, const float* w, int lane, int stride,
                                            int* sidx = nullptr) {
  constexpr int U = 4;
  for (int b = lane; b < n_pad; b += U * stride) {
    int2 g[U];
    int ix[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = b + u * stride, p = p0 + k;
      g[u] = k < n ? *(const int2*)(d.nd_gather + F.G + 2 * p) : make_int2(-1, -1);  // absolute offsets into w
      ix[u] = k < n && p < F.s ? d.nd_idx[F.S + p] : -1;
    }
    float val[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      float x = ix[u] >= 0 ? f[ix[u]] : 0.0f;
      if (g[u].x >= 0) x += w[g[u].x];
      if (g[u].y >= 0) x += w[g[u].y];
      val[u] = x;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (b + u * stride < n_pad) out[b + u * stride] = val[u];
      if (sidx && ix[u] >= 0) sidx[b + u * stride] = ix[u];  // the separator's node (p0 = 0)
    }
  }
}

// The separator's node indices, z_S (e) and x there, for F's backward rows
// (all loads of a thread in flight at once).
__device__ __forceinline__ void nd_sx_into(const DevPtrs& d, const NdFront& F, int* sidx, float* sz, double* sx,
                                           const float* e, const double* x, int N, int lane, int stride) {
  constexpr int U = 4;
  for (int b = lane; b < F.s; b += U * stride) {
    int ix[U];
#pragma unroll
    for (int u = 0; u < U; ++u) ix[u] = b + u * stride < F.s ? d.nd_idx[F.S + b + u * stride] : -1;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (ix[u] < 0) continue;
      sidx[b + u * stride] = ix[u];
      sz[b + u * stride] = e[ix[u]];
      sx[b + u * stride] = x[(long long)ix[u] + N];
    }
  }
}

// out[k] = e at update-set node k of F (k < u; zeros up to n_pad).
__device__ __forceinline__ void nd_xu_into(const DevPtrs& d, const NdFront& F, int n_pad, float* out, const float* e,
                                           int lane, int stride) {
  constexpr int U = 4;
  for (int b = lane; b < n_pad; b += U * stride) {
    int ix[U];
#pragma unroll
    for (int u = 0; u < U; ++u) ix[u] = b + u * stride < F.u ? d.nd_idx[F.U + b + u * stride] : -1;
    float val[U];
#pragma unroll
    for (int u = 0; u < U; ++u) val[u] = ix[u] >= 0 ? e[ix[u]] : 0.0f;
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (b + u * stride < n_pad) out[b + u * stride] = val[u];
  }
}

// Forward results of F's rows [r0, r1) held in res (row a at res[a - r0]):
// z_S into e at the separator's nodes, W = v_U - M v_S into F's update vector.
__device__ __forceinline__ void nd_fwd_store(const DevPtrs& d, const NdFront& F, int r0, int r1, const float* res,
                                             float* e, float* w, int lane, int stride) {
  constexpr int U = 4;
  for (int b = r0 + lane; b < r1; b += U * stride) {
    int ix[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int a = b + u * stride;
      ix[u] = a < r1 && a < F.s ? d.nd_idx[F.S + a] : -1;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int a = b + u * stride;
      if (ix[u] >= 0) e[ix[u]] = res[a - r0];
      else if (a < r1) w[F.W + a - F.s] = res[a - r0];
    }
  }
}

// Backward results for F's separator rows [r0, r1), res[a - r0] = (N x_U)_a
// (null when u = 0): x_S = z_S - N x_U into e, and x += x_S at the node.
__device__ __forceinline__ void nd_back_store(const DevPtrs& d, const NdFront& F, int r0, int r1, const float* res,
                                              float* e, double* x, int N, int lane, int stride) {
  constexpr int U = 4;
  for (int b = r0 + lane; b < r1; b += U * stride) {
    int ix[U];
    float z[U];
    double xo[U];
#pragma unroll
    for (int u = 0; u < U; ++u) ix[u] = b + u * stride < r1 ? d.nd_idx[F.S + b + u * stride] : -1;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      z[u] = ix[u] >= 0 ? e[ix[u]] : 0.0f;
      xo[u] = ix[u] >= 0 ? x[(long long)ix[u] + N] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (ix[u] < 0) continue;
      const float val = z[u] - (res ? res[b + u * stride - r0] : 0.0f);
      e[ix[u]] = val;
      x[(long long)ix[u] + N] = xo[u] + (double)val;
    }
  }
}

// One task of a nested-dissection phase of instance B: rows [T.y, T.y + T.z)
// of the large front T.x (T.w = 0, the whole CTA), the T.z <= kBcrWarps small
// fronts from T.x (T.w = 1, one per warp) or the T.z <= 4 kBcrWarps tiny
// fronts from T.x (T.w = 2, one per 8-lane group).  A task's matrix rows are
// one contiguous range (the fronts' matrices are stored level by level in
// task order, within kNdStageFloats), staged into the dynamic shared memory
// by one bulk copy issued before the vectors are gathered; the vectors live in the wide kernel's
// reduction buffer (a large front's at [0, kNdVecCap) and its task rows'
// values after it; kNdWarpArea floats per warp, kNdTinyArea per 8-lane group).
// A nested-dissection worker: the whole CTA (barrier 0), or one half of it
// (named barriers 1 and 2, 256 threads each) in the dataflow sweeps, so that
// an SM has two tasks in flight.  Its vectors, stage and copy barrier are its
// own.
struct NdUnit {
  int t, n, nw;   // thread within the unit, threads, warps
  int id;         // named barrier (0: __syncthreads)
  float* red;     // the unit's vector areas
  float* sbuf;    // the unit's matrix stage
  uint64_t* bar;  // the unit's copy barrier
  int vcap;       // floats of a large front's vector; its task rows' values follow
  __device__ __forceinline__ void sync() const {
    if (id == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
  }
  __device__ __forceinline__ bool sync_and(bool p) const {
    if (id == 0) return __syncthreads_and(p) != 0;
    unsigned r;
    asm volatile(
        "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n bar.red.and.pred po, %2, %3, pi;\n"
        " selp.u32 %0, 1, 0, po;\n}\n"
        : "=r"(r)
        : "r"((unsigned)p), "r"(id), "r"(n)
        : "memory");
    return r != 0;
  }
};

// mbar_wait for a unit's copies (every thread of the unit).
__device__ bool nd_mbar_wait(const NdUnit& U, uint64_t* bar, unsigned parity, int32_t* err) {
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
  return U.sync_and(ok);
}

// Issue the bulk copy of task `tr`'s matrix rows into the unit's stage (its
// thread 0; after the unit's earlier reads of the stage).
__device__ __forceinline__ void nd_issue(const DevPtrs& d, const NdUnit& U, const longlong2 tr) {
  if (U.t == 0 && tr.y > tr.x && tr.y - tr.x <= kNdUnitStage) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(U.bar, (unsigned)(tr.y - tr.x) * 4u);
    bulk_g2s(U.sbuf, (const float*)d.bcr + tr.x, (unsigned)(tr.y - tr.x) * 4u, U.bar);
  }
}

// issued: the task's copy was issued before (nd_issue), e.g. while its
// dependencies were awaited.
__device__ bool run_nd_task(const DevPtrs& d, Ctx& c, const NdUnit& U, const BcrInst& B, int kind, const int4 T,
                            const longlong2 tr, bool issued, float* fb, float* eb, double* xb, float* wb) {
  const float* f = fb + B.foff;
  float* e = eb + B.foff;
  double* x = xb + B.node_off;
  const int lane = U.t & 31, warp = U.t >> 5;
  const bool fwd = kind == kNdFwd;
  const float* mat = (const float*)d.bcr;
  // the task's matrix range [m0, m1) (the layout keeps it within a worker's
  // stage, kNdUnitStage: a larger one is a table fault, reported as a
  // capacity error and not computed)
  const long long m0 = tr.x, m1 = tr.y;
  if (m1 - m0 > kNdUnitStage) {
    if (U.t == 0) atomicOr(c.err, kErrCapacity);
    return true;
  }
  const bool staged = m1 > m0;
  if (!issued) nd_issue(d, U, tr);
  // matrix float o of the buffer in the stage
  auto at = [&](long long o) { return U.sbuf + (o - m0); };
  auto wait = [&]() {
    if (!staged) return true;
    if (!nd_mbar_wait(U, U.bar, c.parity, c.err)) return false;
    c.parity ^= 1u;
    return true;
  };
  if (T.w == 0) {
    const NdFront F = d.nd_front[T.x];
    float* v = U.red;
    float* res = U.red + U.vcap;
    const int r0 = T.y, r1 = T.y + T.z;
    if (fwd) {
      nd_rhs_into(d, F, 0, F.s, F.sp, v, f, wb, U.t, U.n);
      const int u0 = max(r0, F.s);  // the task's U rows start with their right-hand sides
      if (u0 < r1) nd_rhs_into(d, F, u0, r1 - u0, r1 - u0, res + (u0 - r0), f, wb, U.t, U.n);
      U.sync();
      if (!wait()) return false;
      const int fs = F.s;
      rows_dot_any(F.sp >> 2, at(m0), F.sp >> 2, r0, r1, r0, (const float4*)v, lane, warp, U.nw,
                  [=](int a, float acc) { res[a - r0] = a < fs ? acc : res[a - r0] - acc; });
      U.sync();
      nd_fwd_store(d, F, r0, r1, res, e, wb, U.t, U.n);
    } else {
      nd_xu_into(d, F, F.up, v, e, U.t, U.n);
      U.sync();
      if (!wait()) return false;
      if (F.u > 0)
        rows_dot_any(F.up >> 2, at(m0), F.up >> 2, r0, r1, r0, (const float4*)v, lane, warp, U.nw,
                    [=](int a, float acc) { res[a - r0] = acc; });
      U.sync();
      nd_back_store(d, F, r0, r1, F.u > 0 ? res : nullptr, e, x, B.N, U.t, U.n);
    }
    U.sync();
    return true;
  }
  if (T.w == 2) {
    // tiny fronts: group g = lane / 8 of warp w takes front T.x + 4 w + g.
    // Its rows go G = 4 lanes to a row forward (sp <= kNdTinyS = 16: at most
    // four float4), 8 backward (up <= kNdTinyU = 48): the sums do not depend
    // on the other fronts of the warp
    const int g = lane >> 3, gl = lane & 7;
    float* a0 = U.red + warp * kNdWarpArea + g * kNdTinyArea;
    const int k = 4 * warp + g;
    const bool has = k < T.z;
    NdFront F;
    if (has) F = d.nd_front[T.x + k];
    const int n4 = has ? (fwd ? F.sp : F.up) >> 2 : 0;
    const int nrows = !has ? 0 : (fwd ? F.s + F.u : (F.u > 0 ? F.s : 0));
    const int nmax = warp_max(nrows);
    if (fwd) {
      float* vs = a0;                    // v_S, kNdTinyS floats
      float* rs = a0 + kNdTinyS;         // z_S
      float* ru = a0 + 2 * kNdTinyS;     // the U rows' right-hand sides, then W
      int* si = (int*)(a0 + 5 * kNdTinyS);  // the separator's nodes
      if (has) {
        nd_rhs_into(d, F, 0, F.s, F.sp, vs, f, wb, gl, 8, si);
        nd_rhs_into(d, F, F.s, F.u, F.u, ru, f, wb, gl, 8);
      }
      U.sync();
      if (!wait()) return false;
      if (nmax > 0) {
        const float* m = has ? at(F.FM) : U.sbuf;
        const int fs = has ? F.s : 0;
        auto put = [=](int a, float acc) {
          if (a < fs) rs[a] = acc;
          else ru[a - fs] -= acc;
        };
        rows_dot_grp<4>(m, n4, nrows, nmax, (const float4*)vs, n4, gl, put);
      }
      __syncwarp();
      if (has) {
        for (int a = gl; a < F.s; a += 8) e[si[a]] = rs[a];
        for (int a = gl; a < F.u; a += 8) wb[F.W + a] = ru[a];
      }
    } else {
      float* vu = a0;                    // x_U, kNdTinyU floats
      float* rs = a0 + kNdTinyU;         // N x_U
      int* si = (int*)(a0 + 4 * kNdTinyS);
      float* sz = a0 + 5 * kNdTinyS;
      double* sx = (double*)(a0 + 6 * kNdTinyS);
      if (has) {
        nd_xu_into(d, F, F.up, vu, e, gl, 8);
        nd_sx_into(d, F, si, sz, sx, e, x, B.N, gl, 8);
      }
      U.sync();
      if (!wait()) return false;
      if (nmax > 0) {
        const float* m = has ? at(F.NB) : U.sbuf;
        auto put = [=](int a, float acc) { rs[a] = acc; };
        rows_dot_grp<8>(m, n4, nrows, nmax, (const float4*)vu, n4, gl, put);
      }
      __syncwarp();
      if (has)
        for (int a = gl; a < F.s; a += 8) {
          const float val = sz[a] - (F.u > 0 ? rs[a] : 0.0f);
          e[si[a]] = val;
          x[(long long)si[a] + B.N] = sx[a] + (double)val;
        }
    }
    U.sync();
    return true;
  }
  // small fronts, one per warp
  float* a0 = U.red + warp * kNdWarpArea;
  const bool has = warp < T.z;
  NdFront F;
  if (has) F = d.nd_front[T.x + warp];
  if (fwd) {
    float* vs = a0;                      // v_S, kNdWarpMaxS floats
    float* rs = a0 + kNdWarpMaxS;        // z_S
    float* ru = a0 + 2 * kNdWarpMaxS;    // the U rows' right-hand sides, then W
    int* si = (int*)(a0 + 5 * kNdWarpMaxS);  // the separator's nodes
    if (has) {
      nd_rhs_into(d, F, 0, F.s, F.sp, vs, f, wb, lane, 32, si);
      nd_rhs_into(d, F, F.s, F.u, F.u, ru, f, wb, lane, 32);
    }
    U.sync();
    if (!wait()) return false;
    if (has) {
      const int fs = F.s;
      rows_dot_any(F.sp >> 2, at(F.FM), F.sp >> 2, 0, F.s + F.u, 0, (const float4*)vs, lane, 0, 1,
                   [=](int a, float acc) {
                     if (a < fs) rs[a] = acc;
                     else ru[a - fs] -= acc;
                   });
      __syncwarp();
      for (int a = lane; a < F.s; a += 32) e[si[a]] = rs[a];
      for (int a = lane; a < F.u; a += 32) wb[F.W + a] = ru[a];
    }
  } else {
    float* vu = a0;                      // x_U, kNdWarpMaxU floats
    float* rs = a0 + kNdWarpMaxU;        // N x_U
    int* si = (int*)(a0 + 4 * kNdWarpMaxS);
    float* sz = a0 + 5 * kNdWarpMaxS;
    double* sx = (double*)(a0 + 6 * kNdWarpMaxS);
    if (has) {
      nd_xu_into(d, F, F.up, vu, e, lane, 32);
      nd_sx_into(d, F, si, sz, sx, e, x, B.N, lane, 32);
    }
    U.sync();
    if (!wait()) return false;
    if (has) {
      if (F.u > 0)
        rows_dot_any(F.up >> 2, at(F.NB), F.up >> 2, 0, F.s, 0, (const float4*)vu, lane, 0, 1,
                     [=](int a, float acc) { rs[a] = acc; });
      __syncwarp();
      for (int a = lane; a < F.s; a += 32) {
        const float val = sz[a] - (F.u > 0 ? rs[a] : 0.0f);
        e[si[a]] = val;
        x[(long long)si[a] + B.N] = sx[a] + (double)val;
      }
    }
  }
  // the next task's copy overwrites the staged rows and its vectors the
  // per-warp areas: every warp finishes here first
  U.sync();
  return true;
}

// Task q of level l of instance B's sweep `kind`.
__device__ __forceinline__ bool run_nd(const DevPtrs& d, Ctx& c, const BcrInst& B, int kind, int l, int q, float* fb,
                                       float* eb, double* xb, float* wb) {
  const int t = (kind == kNdFwd ? B.nd_ft[l] : B.nd_bt[l]) + q;
  const NdUnit U{(int)threadIdx.x, (int)blockDim.x, kBcrWarps, 0, c.red, c.sbuf, c.bar, kNdVecCap};
  return run_nd_task(d, c, U, B, kind, d.nd_task[t], d.nd_trange[t], false, fb, eb, xb, wb);
}

// ---- dataflow sweeps (BcrPlan::nd_flow) ----
// CTA b takes the sweep's tasks b, b + nb, ... of the task order (right-hand
// side by right-hand side).  Before a task runs, thread f of the CTA
// waits until front f of the task has what it reads: forward, both children
// have finished all their tasks; backward, the parent has.  After the task,
// each of its fronts counts one finished task (release; the waits acquire).
// The order puts every task after those it waits for, every CTA runs its
// tasks in order and every CTA is resident (cooperative launch), so the
// earliest unfinished task always runs.  A wait gives up after d.wait_ns (kErrTimeout): false.
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ bool nd_wait_deps(const DevPtrs& d, const BcrPlan& pl, const NdUnit& U, int kind, int rh, const int4 T) {
  const int nfr = T.w == 0 ? 1 : T.z;
  const int sw = kind == kNdFwd ? 0 : 1;
  const unsigned* done = d.nd_done + ((long long)sw * kBcrMaxRhs + rh) * pl.nd_fronts;
  const int32_t* need = d.nd_need + (long long)sw * pl.nd_fronts;
  bool ok = true;
  if (U.t < nfr) {
    const NdFront& F = d.nd_front[T.x + U.t];
    int dep[2] = {-1, -1};
    if (kind == kNdFwd) {
      dep[0] = F.child[0];
      dep[1] = F.child[1];
    } else {
      dep[0] = F.parent;
    }
    unsigned long long t0 = 0;
    for (int q = 0; q < 2 && ok; ++q) {
      if (dep[q] < 0) continue;
      const unsigned want = (unsigned)need[dep[q]];
      for (long long spins = 0; ld_acquire_u32(done + dep[q]) < want; ++spins) {
        if ((spins & 63) == 63) {
          if ((*(volatile int*)d.err) & kErrTimeout) {
            ok = false;
            break;
          }
          const unsigned long long now = global_ns();
          if (t0 == 0) t0 = now;
          else if (now - t0 > d.wait_ns) {
            atomicOr(d.err, kErrTimeout);
            ok = false;
            break;
          }
        }
        __nanosleep(64);
      }
    }
  }
  return U.sync_and(ok);
}

// After a task (its last unit barrier behind it): each front counts one.
__device__ __forceinline__ void nd_signal(const DevPtrs& d, const BcrPlan& pl, const NdUnit& U, int kind, int rh,
                                          const int4 T) {
  const int nfr = T.w == 0 ? 1 : T.z;
  const int sw = kind == kNdFwd ? 0 : 1;
  if (U.t < nfr) {
    unsigned* p = d.nd_done + ((long long)sw * kBcrMaxRhs + rh) * pl.nd_fronts + T.x + U.t;
    __threadfence();
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(p) : "memory");
  }
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
// kParts: 1 = reduction stages, 2 = nested-dissection tasks, 3 = both (a
// batch of both kinds); each instantiation compiles only what it runs, so
// the registers of one path do not spill the other's.
template <int MAXN, int kParts>
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
  __shared__ __align__(8) uint64_t s_ubar[kNdUnits];  // the workers' copy barriers (dataflow sweeps)
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
  if (threadIdx.x < kNdUnits) mbar_init(&s_ubar[threadIdx.x], 1);
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
    if constexpr ((kParts & 2) != 0) {
      if (pl.nd_flow) {  // the dataflow sweeps' counters, for this pass
        const long long nz = 2ll * kBcrMaxRhs * pl.nd_fronts;
        for (long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x; z < nz; z += (long long)nb * blockDim.x)
          d.nd_done[z] = 0u;
      }
    }
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
    if constexpr (kParts == 2) {
      if (pl.nd_flow) {  // nested dissection of every instance: one dataflow phase per sweep
        for (int sw = 0; sw < 2; ++sw) {
          const int kind = sw == 0 ? kNdFwd : kNdBack;
          const int n = sw == 0 ? pl.nd_nf : pl.nd_nb;
          const int2* list = d.nd_flow + (sw == 0 ? 0 : pl.nd_nf);
          const long long total = (long long)R * n;
          // unit u (two per CTA) takes tasks u, u + 2 nb, ... (each after
          // the tasks it waits for); the next task's entry is loaded while
          // this one runs
          constexpr int UT = kBcrThreads / kNdUnits, UW = kBcrWarps / kNdUnits;
          const int h = (int)threadIdx.x / UT;
          const NdUnit U{(int)threadIdx.x - h * UT, UT, UW, kNdUnits == 1 ? 0 : 1 + h, red + h * UW * MAXN,
                         s_dyn + h * kNdUnitStage, s_ubar + h, UW * MAXN - kNdTaskRows};
          const long long u0 = (long long)kNdUnits * blockIdx.x + h, nu = (long long)kNdUnits * nb;
          auto entry = [&](long long t) { return list[t - (t / n) * n]; };
          int2 en = u0 < total ? entry(u0) : make_int2(0, 0);
          int4 T = u0 < total ? d.nd_task[en.x] : make_int4(0, 0, 0, 0);
          bool good = true;
          for (long long t = u0; t < total && good; t += nu) {
            const int rh = (int)(t / n);
            const long long tn = t + nu;
            const int2 en_n = tn < total ? entry(tn) : en;
            if (s_act[rh * ni + en.y]) {
              // the matrix rows are static: their copy runs while the
              // dependencies are awaited
              const longlong2 tr = d.nd_trange[en.x];
              nd_issue(d, U, tr);
              good = nd_wait_deps(d, pl, U, kind, rh, T);
              const BcrInst& B = en.y == 0 ? s_b0 : d.bcr_inst[en.y];
              if (good)
                good = run_nd_task(d, c, U, B, kind, T, tr, true, d.bcr_f + rh * pl.rows, d.bcr_e + rh * pl.rows,
                                   x_of(rh), d.nd_w + rh * pl.nd_wrows);
              if (good) nd_signal(d, pl, U, kind, rh, T);
            }
            en = en_n;
            if (tn < total) T = d.nd_task[en.x];
          }
          // (a unit that gave up goes on to the grid barrier, which sees the
          // time-out bit and ends the kernel)
          if (!grid_sync(d, nb)) return;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) d.cnt[0] += 1;
        continue;
      }
    }
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
          if constexpr ((kParts & 2) != 0) {
            if (!run_nd(d, c, B, kind, s_kind[k] & 255, tt - s_pre[k], d.bcr_f + rh * pl.rows,
                        d.bcr_e + rh * pl.rows, x_of(rh), d.nd_w + rh * pl.nd_wrows))
              return;
          }
        } else if constexpr ((kParts & 1) != 0) {
          if (!run_stage<MAXN>(d, c, B, kind, s_kind[k] & 255, tt - s_pre[k], sv, d.bcr_f + rh * pl.rows,
                               d.bcr_e + rh * pl.rows, x_of(rh)))
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
  // wide: 0 the narrow reduction, 1 the wide reduction (and nested
  // dissection, if some instance uses it), 2 nested dissection alone
  return b.wide == 2   ? (const void*)k_solve_bcr<kBcrMaxNWide, 2>
         : b.wide == 1 ? (const void*)k_solve_bcr<kBcrMaxNWide, 3>
                       : (const void*)k_solve_bcr<kBcrMaxN, 1>;
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
  // nested dissection keeps its vectors in the wide kernel's reduction
  // buffer (kBcrWarps x kBcrMaxNWide floats)
  int any_nd = 0;
  for (int k = 0; k < ni; ++k) any_nd |= bi[k].nd;
  int any_bcr = 0;
  for (int k = 0; k < ni; ++k) any_bcr |= !bi[k].nd;
  pl.bcr.wide = !any_bcr ? 2 : (widest > kBcrMaxN || any_nd ? 1 : 0);
  if (pl.bcr.nd_floats > (kBcrWarps / kNdUnits) * kBcrMaxNWide - kNdTaskRows) return 0;  // a worker's vector area
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
  if (any_nd) {  // the nested-dissection tasks stage their matrix rows
    const long long nd_stage_bytes = (long long)kNdStageFloats * (long long)sizeof(float);
    if (nd_stage_bytes > budget) return 0;
    dyn = nd_stage_bytes > dyn ? nd_stage_bytes : dyn;
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
