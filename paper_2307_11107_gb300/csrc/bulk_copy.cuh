// Bulk asynchronous copies from global to shared memory with completion on
// an mbarrier (cp.async.bulk, the untiled form of TMA: both addresses 16-byte
// aligned, sizes multiples of 16 bytes), and the bounded wait for a copy
// barrier's phase.  Included inside namespace apic::{anonymous}.
#pragma once

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
