// mbarrier and bulk-copy wrappers (inline PTX) shared by the kernels that
// stage operands asynchronously.  Every wait here is bounded: a phase that does
// not complete within the given time makes the wait return false, so a kernel
// can record an error and drain instead of hanging.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mahi {

constexpr uint32_t kSpinLimit = 1u << 26;  // iterations of one bounded wait, beside its time limit

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// non-blocking test of a phase
__device__ __forceinline__ bool mbar_test(uint64_t *b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// bounded wait: gives up after lim ns (or when another role of the CTA gave
// up), raising the abort flag; returns false then
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, volatile int *abort_flag, uint64_t lim) {
  if (mbar_test(b, parity)) return true;  // non-blocking test first: most waits find the phase complete
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    if (mbar_try_wait(b, parity)) return true;
    if (*abort_flag) return false;
    if ((it & 255) == 255 && global_ns() - t0 > lim) break;
  }
  *abort_flag = 1;
  return false;
}
// two bounded waits whose first (non-blocking) tests are issued together, so
// that their shared-memory latencies overlap when both phases are complete
__device__ __forceinline__ bool mbar_wait2(uint64_t *a, uint32_t pa, uint64_t *b, uint32_t pb, volatile int *abort_flag,
                                           uint64_t lim) {
  const bool ra = mbar_test(a, pa), rb = mbar_test(b, pb);
  if (ra && rb) return true;
  return (ra || mbar_wait(a, pa, abort_flag, lim)) && (rb || mbar_wait(b, pb, abort_flag, lim));
}
// bounded wait that no other thread can cut short (drains after a failure)
__device__ __forceinline__ bool mbar_wait_for(uint64_t *b, uint32_t parity, uint64_t lim) {
  if (mbar_test(b, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    if (mbar_try_wait(b, parity)) return true;
    if ((it & 255) == 255 && global_ns() - t0 > lim) break;
  }
  return false;
}
// orders this thread's generic-proxy shared-memory accesses before later
// async-proxy (bulk copy) accesses
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// bulk copy global -> shared of `bytes` (a multiple of 16; both addresses
// 16-byte aligned), completing on `bar` by its byte count
__device__ __forceinline__ void bulk_g2s(void *smem, const void *gmem, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(smem)),
      "l"(gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace mahi
