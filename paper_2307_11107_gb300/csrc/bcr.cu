// Direct FP32 solver of the Poisson problem of Eqs. 6-7 (Sec. 2) inside an
// FP64 iterative refinement, for one instance whose grid has n1 = 2^K cells
// in x1.
//
// The finite-difference system is block tridiagonal in x1: row i of N2
// unknowns couples to rows i - 1 and i + 1 through the blocks A_i and C_i and
// to itself through B_i.  Block cyclic reduction eliminates the odd rows, then
// the odd rows of what is left, and so on, until one row remains; the blocks
// of every level are formed once at set-up (FP64 on the host) and stored in
// FP32.  A solve is then 2K - 1 phases of dense matrix-vector products whose
// tasks (one row each) are spread over the CTAs, instead of the dozens of
// line-relaxation phases per multigrid cycle.  The refinement loop
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
constexpr int kMC = kBcrMaxN / 32;  // outputs per lane

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

__device__ __forceinline__ void prefetch_l2(const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
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
template <int NT, bool kShared>
__device__ __forceinline__ void task_mv(const float* const* Mt, const float* const* vt, int N, int Np, float* red,
                                        float* res) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float acc[kMC];
#pragma unroll
  for (int m = 0; m < kMC; ++m) acc[m] = 0.0f;
#pragma unroll 2
  for (int c = warp; c < N; c += kBcrWarps) {
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const float* col = Mt[t] + (long long)c * Np;
      const float x = vt[t][c];
#pragma unroll
      for (int m = 0; m < kMC; ++m) {
        const int j = lane + 32 * m;
        if (j < N) acc[m] = fmaf(kShared ? col[j] : __ldg(col + j), x, acc[m]);
      }
    }
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
  const BcrPlan* B;
  const float* blk;
  float* sbuf;      // NT staged blocks (shared memory mode)
  uint64_t* bar;
  unsigned parity;
  float* red;
  float* sres;
  int32_t* err;
};

// res = sum_t src_t v_t: the blocks are staged in shared memory by one bulk
// copy each (when they fit), else read from global memory.  False on a copy
// time-out (every thread).
template <int NT>
__device__ bool run_task(Ctx& c, const float* const* src, const float* const* vt) {
  const int N = c.B->N, Np = c.B->Np;
  if (c.B->smem) {
    const unsigned bytes = (unsigned)(c.B->blk * sizeof(float));
    if (threadIdx.x == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(c.bar, bytes * NT);
#pragma unroll
      for (int t = 0; t < NT; ++t) bulk_g2s(c.sbuf + t * c.B->blk, src[t], bytes, c.bar);
    }
    if (!mbar_wait(c.bar, c.parity, c.err)) return false;
    c.parity ^= 1u;
    const float* Ms[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) Ms[t] = c.sbuf + t * c.B->blk;
    task_mv<NT, true>(Ms, vt, N, Np, c.red, c.sres);
  } else {
    task_mv<NT, false>(src, vt, N, Np, c.red, c.sres);
  }
  return true;
}

// mode: kBcrRho = the step's density, initial guess and right-hand side are
// formed here (else b and its |b|^2 partials come from the caller);
// kBcrFields = node gradients and surface quantities after the solve.
__global__ void __launch_bounds__(kBcrThreads, 1) k_solve_bcr(DevPtrs d, SolvePlan pl, int mode) {
  extern __shared__ __align__(128) float s_blocks[];
  __shared__ double sh[40];
  __shared__ float sv[3][kBcrMaxN];
  __shared__ float sres[kBcrMaxN];
  __shared__ float red[kBcrWarps * kBcrMaxN];
  __shared__ __align__(8) uint64_t s_bar;
  const BcrPlan& B = pl.bcr;
  const int nb = gridDim.x;
  const Inst& I = d.inst[0];
  const int N = I.N2, K = B.K, M = (1 << K) - 1;
  const long long stride = (long long)nb * blockDim.x;
  const float* blk = d.bcr;
  float* f = d.bcr_f;
  float* e = d.bcr_e;
  double* x = d.phi;
  Ctx c{&B, blk, s_blocks, &s_bar, 0u, red, sres, d.err};
  if (threadIdx.x == 0) {
    mbar_init(&s_bar, 1);
    // bring this CTA's blocks of the whole reduction (and its share of the
    // tail inverse) into L2 while the first residual is formed
    const unsigned bytes = (unsigned)(B.blk * sizeof(float));
    for (int l = 1; l <= B.Lt; ++l) {
      const int ne = 1 << (K - l), nk = ne - 1;
      for (int q = blockIdx.x; q < nk; q += nb) {
        prefetch_l2(blk + (B.P[l] + q) * B.blk, bytes);
        prefetch_l2(blk + (B.Q[l] + q) * B.blk, bytes);
      }
      for (int q = blockIdx.x; q < ne; q += nb) {
        prefetch_l2(blk + (B.Binv[l] + q) * B.blk, bytes);
        prefetch_l2(blk + (B.G[l] + q) * B.blk, bytes);
        prefetch_l2(blk + (B.H[l] + q) * B.blk, bytes);
      }
    }
    const int r0 = blockIdx.x * B.tail_rpc, r1 = min(B.tail_n, r0 + B.tail_rpc);
    if (r1 > r0)
      prefetch_l2(d.bcr_tail + (long long)r0 * B.tail_np, (unsigned)((r1 - r0) * B.tail_np * sizeof(float)));
  }
  double bn = 0.0;
  if (mode & kBcrRho) {
    // rho, the initial guess and b at every node; |b|^2 over the grid
    double pb = 0.0;
    for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes; nd += stride) {
      const double bv = rho_node(d, I, 0, nd);
      pb += bv * bv;
    }
    const double tb = block_sum_any(pb, sh);
    if (threadIdx.x == 0) d.cred[0 * kCoopMaxBlocks + blockIdx.x] = tb;
    if (!grid_sync(d, nb)) return;
    bn = coop_sum(d, 0, 0, nb, sh);
  } else {
    // |b|^2 from the right-hand-side kernel's partials (fixed order)
    if (threadIdx.x == 0) {
      double s0 = 0.0;
      for (int k = 0; k < kRedBlocks; ++k) s0 += d.red[k];
      sh[34] = s0;
    }
    __syncthreads();
    bn = sh[34];
    __syncthreads();
  }
  for (int it = 0;; ++it) {
    // FP64 residual, stored as the FP32 right-hand side of the reduction
    double pr = 0.0;
    for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes; nd += stride) {
      const int i = (int)(nd / N), j = (int)(nd % N);
      if (i > 0 && i < I.n1) {
        double r = d.b[nd] - apply_st<double, double>(d.st64, I.nodes, x, nd, i, j, I.n2, N, 1);
        f[(long long)(i - 1) * N + j] = (float)r;
        pr += r * r;
      }
    }
    const double t = block_sum_any(pr, sh);
    if (threadIdx.x == 0) d.cred[2 * kCoopMaxBlocks + blockIdx.x] = t;
    if (!grid_sync(d, nb)) return;
    const double rn = coop_sum(d, 0, 2, nb, sh);
    const bool conv = rn <= I.tol * I.tol * bn, bad = !(rn == rn);
    if (conv || bad || it >= I.max_iter) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        SolverState& S = d.sol[0];
        S.res = bn > 0.0 ? sqrt(rn / bn) : 0.0;
        S.iters = it;
        S.done = 1;
        if (!conv) atomicOr(d.err, bad ? kErrNonFinite : kErrNotConverged);
      }
      break;
    }
    // forward reduction: f_i -= P_i f_{i-h} + Q_i f_{i+h} on the kept rows
    for (int l = 1; l <= B.Lt; ++l) {
      const int h = 1 << (l - 1);
      const int nk = (1 << (K - l)) - 1;
      for (int q = blockIdx.x; q < nk; q += nb) {
        const int i = 2 * h * (q + 1);
        for (int j = threadIdx.x; j < N; j += blockDim.x) {
          sv[0][j] = f[(long long)(i - h - 1) * N + j];
          sv[1][j] = f[(long long)(i + h - 1) * N + j];
        }
        __syncthreads();
        const float* Mt[2] = {blk + (B.P[l] + q) * B.blk, blk + (B.Q[l] + q) * B.blk};
        const float* vt[2] = {sv[0], sv[1]};
        if (!run_task<2>(c, Mt, vt)) return;
        for (int j = threadIdx.x; j < N; j += blockDim.x) f[(long long)(i - 1) * N + j] -= sres[j];
        __syncthreads();
      }
      if (!grid_sync(d, nb)) return;
    }
    // the rows left, i = 2^Lt (q + 1): e = T^-1 f with the dense inverse; each
    // CTA owns a contiguous range of its rows (staged in shared memory by one
    // bulk copy when the blocks are), one row per warp, lanes over the
    // columns, fixed-order shuffle sums
    {
      const int tn = B.tail_n, tnp = B.tail_np, hs = 1 << B.Lt;
      const int r0 = blockIdx.x * B.tail_rpc, r1 = min(tn, r0 + B.tail_rpc);
      float* rows = s_blocks;
      float* fs = s_blocks + (B.smem ? (long long)B.tail_rpc * tnp : 0);
      const bool stage = B.smem && r1 > r0;
      if (stage && threadIdx.x == 0) {
        const unsigned bytes = (unsigned)((r1 - r0) * tnp * sizeof(float));
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(c.bar, bytes);
        bulk_g2s(rows, d.bcr_tail + (long long)r0 * tnp, bytes, c.bar);
      }
      for (int o = threadIdx.x; o < tn; o += blockDim.x) {
        const int q = o / N, j = o - q * N;
        fs[o] = f[(long long)(hs * (q + 1) - 1) * N + j];
      }
      if (stage) {
        if (!mbar_wait(c.bar, c.parity, c.err)) return;
        c.parity ^= 1u;
      } else {
        __syncthreads();
      }
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      for (int o = r0 + warp; o < r1; o += kBcrWarps) {
        const float* row = stage ? rows + (long long)(o - r0) * tnp : d.bcr_tail + (long long)o * tnp;
        float a = 0.0f;
#pragma unroll 4
        for (int cc = lane; cc < tn; cc += 32) a = fmaf(row[cc], fs[cc], a);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(kFull, a, off);
        if (lane == 0) {
          const int q = o / N, j = o - q * N, i = hs * (q + 1);
          e[(long long)(i - 1) * N + j] = a;
          x[(long long)i * N + j] += (double)a;
        }
      }
      if (!grid_sync(d, nb)) return;
    }
    // back substitution: e_k = B_k^-1 f_k - G_k e_{k-h} - H_k e_{k+h}; x += e
    for (int l = B.Lt; l >= 1; --l) {
      const int h = 1 << (l - 1);
      const int ne = 1 << (K - l);
      for (int q = blockIdx.x; q < ne; q += nb) {
        const int k = h * (2 * q + 1);
        for (int j = threadIdx.x; j < N; j += blockDim.x) {
          sv[0][j] = f[(long long)(k - 1) * N + j];
          sv[1][j] = k - h >= 1 ? -e[(long long)(k - h - 1) * N + j] : 0.0f;
          sv[2][j] = k + h <= M ? -e[(long long)(k + h - 1) * N + j] : 0.0f;
        }
        __syncthreads();
        const float* Mt[3] = {blk + (B.Binv[l] + q) * B.blk, blk + (B.G[l] + q) * B.blk,
                              blk + (B.H[l] + q) * B.blk};
        const float* vt[3] = {sv[0], sv[1], sv[2]};
        if (!run_task<3>(c, Mt, vt)) return;
        for (int j = threadIdx.x; j < N; j += blockDim.x) {
          e[(long long)(k - 1) * N + j] = sres[j];
          x[(long long)k * N + j] += (double)sres[j];
        }
        __syncthreads();
      }
      if (!grid_sync(d, nb)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) d.cnt[0] += 1;
  }
  if (mode & kBcrFields) {
    // phi is final everywhere (the last pass ended at a grid barrier)
    for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes; nd += stride)
      grad_node<float, float2>(d, I, nd);
    if (blockIdx.x == nb - 1) surface_block(d, 0, sh);
  }
}

constexpr int kStaticSmem = 40 * 8 + 3 * kBcrMaxN * 4 + kBcrMaxN * 4 + kBcrWarps * kBcrMaxN * 4 + 64;

}  // namespace

// Dynamic shared memory: the staged blocks of one task (when they fit) or at
// least the tail right-hand side.
static long long dyn_bytes(const BcrPlan& b) {
  long long tail = (long long)b.tail_np * (long long)sizeof(float);  // right-hand side
  if (b.smem) tail += (long long)b.tail_rpc * b.tail_np * (long long)sizeof(float);  // + the CTA's rows
  const long long staged = b.smem ? 3ll * b.blk * (long long)sizeof(float) : 0;
  return staged > tail ? staged : tail;
}

const void* bcr_kernel() { return (const void*)k_solve_bcr; }

int bcr_blocks(SolvePlan& pl, int sms) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int nb = sms < kCoopMaxBlocks ? sms : kCoopMaxBlocks;
  pl.bcr.tail_rpc = (pl.bcr.tail_n + nb - 1) / nb;
  const long long staged = 3ll * pl.bcr.blk * (long long)sizeof(float);
  const long long tail = (long long)(pl.bcr.tail_rpc + 1) * pl.bcr.tail_np * (long long)sizeof(float);
  pl.bcr.smem = (staged > tail ? staged : tail) + kStaticSmem <= optin ? 1 : 0;
  if (const char* e = std::getenv("APIC_BCR_STAGE")) pl.bcr.smem = pl.bcr.smem && std::atoi(e) != 0;
  const int dyn = (int)dyn_bytes(pl.bcr);
  if (dyn + kStaticSmem > optin) return 0;
  if (cudaFuncSetAttribute(k_solve_bcr, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) != cudaSuccess) return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve_bcr, kBcrThreads, dyn) != cudaSuccess) return 0;
  if (per_sm < 1) return 0;
  return nb;
}

cudaError_t launch_solve_bcr(const DevPtrs& d, const SolvePlan& pl, int blocks, int mode, cudaStream_t s) {
  DevPtrs dd = d;
  SolvePlan pp = pl;
  int mm = mode;
  void* args[] = {&dd, &pp, &mm};
  const size_t dyn = (size_t)dyn_bytes(pl.bcr);
  return cudaLaunchCooperativeKernel((const void*)k_solve_bcr, dim3(blocks), dim3(kBcrThreads), args, dyn, s);
}

}  // namespace apic
