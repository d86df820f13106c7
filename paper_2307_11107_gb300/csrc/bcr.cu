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

#include "apic_internal.h"

namespace apic {
namespace {

#include "solver_common.cuh"

constexpr int kBcrThreads = 512;
constexpr int kBcrWarps = kBcrThreads / 32;
constexpr int kMC = kBcrMaxN / 32;  // outputs per lane

// res = sum_t M_t v_t for NT column-major N x N blocks M_t (v_t in shared
// memory), by the whole CTA: warp w takes the columns w, w + kBcrWarps, ...,
// lane l the rows l + 32 m; the per-warp partial sums are added in warp order
// (the result does not depend on scheduling).
template <int NT>
__device__ __forceinline__ void task_mv(const float* const* Mt, const float* const* vt, int N, float* red,
                                        float* res) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float acc[kMC];
#pragma unroll
  for (int m = 0; m < kMC; ++m) acc[m] = 0.0f;
  for (int c = warp; c < N; c += kBcrWarps) {
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const float* col = Mt[t] + (long long)c * N;
      const float x = vt[t][c];
#pragma unroll
      for (int m = 0; m < kMC; ++m) {
        const int j = lane + 32 * m;
        if (j < N) acc[m] = fmaf(__ldg(col + j), x, acc[m]);
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

__global__ void __launch_bounds__(kBcrThreads, 1) k_solve_bcr(DevPtrs d, SolvePlan pl) {
  __shared__ double sh[40];
  __shared__ float sv[3][kBcrMaxN];
  __shared__ float sres[kBcrMaxN];
  __shared__ float red[kBcrWarps * kBcrMaxN];
  const BcrPlan& B = pl.bcr;
  const int nb = gridDim.x;
  const Inst& I = d.inst[0];
  const int N = I.N2, K = B.K, M = (1 << K) - 1;
  const long long stride = (long long)nb * blockDim.x;
  const float* blk = d.bcr;
  float* f = d.bcr_f;
  float* e = d.bcr_e;
  double* x = d.phi;
  // |b|^2 from the right-hand-side kernel's partials (fixed order)
  if (threadIdx.x == 0) {
    double bn = 0.0;
    for (int k = 0; k < kRedBlocks; ++k) bn += d.red[k];
    sh[34] = bn;
  }
  __syncthreads();
  const double bn = sh[34];
  __syncthreads();
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
      return;
    }
    // forward reduction: f_i -= P_i f_{i-h} + Q_i f_{i+h} on the kept rows
    for (int l = 1; l < K; ++l) {
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
        task_mv<2>(Mt, vt, N, red, sres);
        for (int j = threadIdx.x; j < N; j += blockDim.x) {
          float v = f[(long long)(i - 1) * N + j] - sres[j];
          f[(long long)(i - 1) * N + j] = v;
          sv[2][j] = v;
        }
        __syncthreads();
        if (l == K - 1) {
          // the one row left: its correction directly
          const float* Ml[1] = {blk + B.last * B.blk};
          const float* vl[1] = {sv[2]};
          task_mv<1>(Ml, vl, N, red, sres);
          for (int j = threadIdx.x; j < N; j += blockDim.x) {
            e[(long long)(i - 1) * N + j] = sres[j];
            x[(long long)i * N + j] += (double)sres[j];
          }
          __syncthreads();
        }
      }
      if (!grid_sync(d, nb)) return;
    }
    // back substitution: e_k = B_k^-1 f_k - G_k e_{k-h} - H_k e_{k+h}; x += e
    for (int l = K - 1; l >= 1; --l) {
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
        task_mv<3>(Mt, vt, N, red, sres);
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
}

}  // namespace

int bcr_blocks(int sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve_bcr, kBcrThreads, 0) != cudaSuccess) return 0;
  if (per_sm < 1) return 0;
  int nb = sms < kCoopMaxBlocks ? sms : kCoopMaxBlocks;
  return nb;
}

cudaError_t launch_solve_bcr(const DevPtrs& d, const SolvePlan& pl, int blocks, cudaStream_t s) {
  DevPtrs dd = d;
  SolvePlan pp = pl;
  void* args[] = {&dd, &pp};
  return cudaLaunchCooperativeKernel((const void*)k_solve_bcr, dim3(blocks), dim3(kBcrThreads), args, 0, s);
}

}  // namespace apic
