// Device helpers shared by the Poisson solvers (multigrid-preconditioned
// BiCGSTAB and block cyclic reduction): the stencil product of one node, the
// bounded grid barrier of the cooperative kernels and fixed-order sums.
// Included inside namespace apic::{anonymous}.
#pragma once

constexpr unsigned kFull = 0xffffffffu;

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

// Grid barrier (co-residency is guaranteed by the cooperative launch).  The
// wait is bounded: on time-out the error word gets kErrTimeout and every CTA
// leaves the kernel at its next barrier.
__device__ bool grid_sync(const DevPtrs& d, unsigned nb) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = d.bar + 1;
    unsigned g = *vgen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(d.bar, 1u) == nb - 1) {
      d.bar[0] = 0u;
      __threadfence();
      atomicAdd(d.bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*vgen == g) {
        if ((++spins & 1023) == 0 && ((*(volatile int*)d.err) & kErrTimeout)) break;
        if (spins > (1ll << 24)) {
          atomicOr(d.err, kErrTimeout);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if ((*(volatile int*)d.err) & kErrTimeout) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Fixed-order sum of the nb partials of (inst, slot), done by warp 0.
__device__ double coop_sum(const DevPtrs& d, int inst, int slot, int nb, double* sh) {
  if (threadIdx.x < 32) {
    const double* p = d.cred + ((long long)inst * kNRed + slot) * kCoopMaxBlocks;
    double v = 0.0;
    for (int k = threadIdx.x; k < nb; k += 32) v += p[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    if (threadIdx.x == 0) *sh = v;
  }
  __syncthreads();
  double r = *sh;
  __syncthreads();
  return r;
}

// Block sum of one value per thread (any blockDim that is a multiple of 32).
__device__ double block_sum_any(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
    sh[32] = r;
  }
  __syncthreads();
  r = sh[32];
  __syncthreads();
  return r;
}
