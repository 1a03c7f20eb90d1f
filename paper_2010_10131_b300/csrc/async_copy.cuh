// Bulk asynchronous copies into shared memory and bounded mbarrier waits
// (PTX ISA: cp.async.bulk, mbarrier), shared by the kernels that stream
// their operands with a producer thread.
#pragma once
#include <stdint.h>

namespace atk {
namespace ac {

constexpr unsigned long long WAIT_NS = 2000000000ULL;  // 2 s per wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
               : "=r"(done)
               : "r"(bar), "r"(parity));
  return done != 0;
}

// Wait for the phase of parity `parity` to complete.  Gives up after WAIT_NS,
// or at once when `abort` is set (pass nullptr for a wait that must not be cut
// short, such as a drain of work in flight).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtime();
  for (unsigned it = 1;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if (abort && *abort) return false;
    if ((it & 63) == 0 && gtime() - t0 > WAIT_NS) return false;
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Copy `bytes` (a multiple of 16; both addresses 16-byte aligned) from global
// memory to shared memory, counted on mbarrier `bar` as transaction bytes.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void arrive_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

}  // namespace ac
// 16-byte asynchronous copy global -> shared (cp.async, cached in L2 only).
// src_bytes = 0 writes 16 zero bytes and reads nothing (ragged edges); src
// must still be a valid address.  The thread waits for its own copies with
// cp_async_wait: the hardware completes them like loads, so no bound is needed.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace atk
