// Bulk asynchronous copies from global to shared memory (cp.async.bulk,
// completion counted in bytes on an mbarrier) and the mbarrier operations
// around them, as inline PTX for sm_103a.
//
// Every wait is bounded: wait_parity() gives up after limit_ns of wall-clock
// time (%globaltimer), sets the caller's status bit and returns false, so a
// copy that never completes ends the kernel with a status the host reads
// instead of a hung GPU.  A bulk copy needs 16-byte aligned source and
// destination addresses and a byte count that is a multiple of 16.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mcw {

// status bit set in the plan's device status word when a device wait ran out
constexpr int kStatusWaitTimeout = 1;
// wall-clock limit of one wait inside the solver's kernels (a tile of a few
// KB arrives in microseconds)
constexpr unsigned long long kWaitLimitNs = 1000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

// make initialized barriers visible to the async proxy (the copy engine)
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order this thread's earlier shared-memory accesses before later
// async-proxy accesses (reuse of a stage the threads have read)
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// one arrival that also announces the bytes the phase's copies will deliver
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// one plain arrival (count 1)
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// try_wait with an explicit suspend-time hint: the thread may sleep in
// hardware until the phase completes or about hint_ns pass, so a waiting
// warp issues no instructions meanwhile
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t* bar, uint32_t parity,
                                                   uint32_t hint_ns) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return done != 0;
}

// suspend-time hint of one try in the bounded waits below (far below the
// wall-clock limit, far above a tile's arrival time)
constexpr uint32_t kWaitHintNs = 20000;

// Wait for the phase of the given parity to complete, at most limit_ns;
// on timeout set kStatusWaitTimeout in *status and return false.
__device__ __forceinline__ bool wait_parity(uint64_t* bar, uint32_t parity, int* status,
                                            unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_timer_ns();
  while (true) {
    if (mbar_try_wait_hint(bar, parity, kWaitHintNs)) return true;
    if (global_timer_ns() - t0 > limit_ns) {
      atomicOr(status, kStatusWaitTimeout);
      return false;
    }
  }
}

// bytes (multiple of 16) from global src to shared dst, completion counted on bar
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"((unsigned long long)__cvta_generic_to_global(src)), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// a 4-D tile of a tensor map (coordinates innermost first) into shared dst,
// completion counted on bar; elements outside the tensor are filled with zero
__device__ __forceinline__ void tensor_copy_4d(void* dst, const void* tmap, int c0, int c1, int c2,
                                               int c3, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"((unsigned long long)tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace mcw
