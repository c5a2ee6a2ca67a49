// Bulk-copy (TMA) and mbarrier helpers in inline PTX (sm_90+ forms, used on
// sm_103a).  Every wait is bounded: after ~kWaitCycles clock cycles it
// records GKO_TIMEOUT in the library's device error word and gives up.
#pragma once

#include "common.cuh"

namespace gko {

constexpr long long kWaitCycles = 1ll << 32;  // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arrive on the barrier and add `bytes` to its expected transaction count.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// try_wait: may suspend the thread in hardware until the phase completes or
// a hardware time limit passes, so waiting warps neither spin nor oversleep.
__device__ __forceinline__ bool mbar_try(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the barrier phase with the given parity for at most `limit`
// clock cycles; on time-out record GKO_TIMEOUT in *err and return false.
__device__ __forceinline__ bool mbar_wait_for(uint64_t* bar, unsigned parity, int* err, long long limit) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (clock64() - t0 > limit) {
      if (err) atomicOr(err, 1 << GKO_TIMEOUT);
      return false;
    }
  }
  return true;
}

// Bounded wait of the copy pipelines (~2 s).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int* err) {
  return mbar_wait_for(bar, parity, err, kWaitCycles);
}

// Order this thread's earlier generic-proxy accesses to shared memory before
// its later async-proxy ones (a bulk copy that overwrites a buffer these
// threads have read): every thread that read the buffer runs it, then a
// block barrier, then the thread that issues the copy.
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Global -> shared bulk copy completing on `bar`.  dst/src 16-byte aligned,
// bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Bulk prefetch of [src, src + bytes) into L2 (no completion to wait for).
// src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// The first `parts` blocks of a grid each prefetch one 16-byte-aligned slice
// of the `bytes` at `src` into L2 (thread 0 only), so that gathers from a
// vector read in random order hit L2 instead of waiting on DRAM.
__device__ __forceinline__ void prefetch_slice_l2(const void* src, size_t bytes, unsigned parts) {
  if (threadIdx.x != 0 || blockIdx.x >= parts || bytes < 16) return;
  const uintptr_t a = reinterpret_cast<uintptr_t>(src);
  const uintptr_t lo = (a + 15) & ~uintptr_t(15), hi = (a + bytes) & ~uintptr_t(15);
  if (hi <= lo) return;
  const uintptr_t span = hi - lo;
  const uintptr_t slice = ((span + parts - 1) / parts + 15) & ~uintptr_t(15);
  const uintptr_t s0 = lo + (uintptr_t)blockIdx.x * slice;
  if (s0 >= hi) return;
  const uintptr_t s1 = s0 + slice < hi ? s0 + slice : hi;
  bulk_prefetch_l2(reinterpret_cast<const void*>(s0), (unsigned)(s1 - s0));
}

}  // namespace gko
