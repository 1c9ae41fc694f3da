// Bulk asynchronous copies from global to shared memory (the TMA unit's
// untiled form, cp.async.bulk) completed through a shared-memory mbarrier.
//
// Rules the callers keep: source and destination 16-byte aligned, sizes a
// multiple of 16 bytes, at most 2^20 - 1 bytes expected per barrier phase; a
// copy lands in this CTA's own shared memory (no multicast).  Every wait is
// bounded: after NSFR_WAIT_LIMIT polls the caller gets false and records the
// timeout in the device error word instead of spinning on.
#pragma once

#include <cstdint>

#define NSFR_WAIT_LIMIT (1u << 22)
#define NSFR_FLAG_WAIT_TIMEOUT 4  // error-word bit: a bounded wait gave up

namespace nsfr_async {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make the initialised barrier visible to the async proxy before any copy uses it
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// bytes from global src to shared dst, counted against bar's transaction count
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t done;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return done != 0;
}

// wait for the barrier's phase to complete, at most NSFR_WAIT_LIMIT polls
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase) {
  for (uint32_t i = 0; i < NSFR_WAIT_LIMIT; ++i)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}

}  // namespace nsfr_async
