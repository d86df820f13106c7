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

// Grid barrier (co-residency is guaranteed by the cooperative launch).  A
// 64-bit arrival counter that only grows: each CTA adds 1 (release) and waits
// (acquire) until the counter reaches the next multiple of the CTA count, so
// no reset and no generation word are needed; every launch of a simulation
// uses the same CTA count, so each starts on a multiple.  The wait is bounded
// (about two seconds of global time): on time-out the error word gets
// kErrTimeout and every CTA leaves the kernel at its next barrier.
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long atom_add_release_u64(unsigned long long* p, unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.add.release.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ bool grid_sync(const DevPtrs& d, unsigned nb) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long* cnt = (unsigned long long*)d.bar;
    const unsigned long long old = atom_add_release_u64(cnt, 1ull);
    const unsigned long long target = (old / nb + 1ull) * nb;
    int ok = 1;
    unsigned long long t0 = 0;
    for (long long spins = 0; ld_acquire_u64(cnt) < target; ++spins) {
      if ((spins & 255) == 255) {
        if ((*(volatile int*)d.err) & kErrTimeout) {
          ok = 0;
          break;
        }
        const unsigned long long now = global_ns();
        if (t0 == 0) t0 = now;
        else if (now - t0 > d.wait_ns) {
          atomicOr(d.err, kErrTimeout);
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
