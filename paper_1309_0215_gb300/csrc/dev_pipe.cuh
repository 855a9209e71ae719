// Shared-memory pipeline primitives for sm_103a kernels: mbarriers with
// bounded waits, and contiguous global -> shared copies by the bulk copy
// engine (cp.async.bulk) whose completion is counted on an mbarrier.
#pragma once
#include <cstdint>

namespace mrgb {
namespace pipe {

constexpr long long SPIN_LIMIT = 1ll << 20;
constexpr uint32_t SUSPEND_NS = 1000;  // a waiting thread sleeps up to this long per poll

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
// Poll for the completion of the phase with the given parity; the thread is
// suspended until the phase completes or SUSPEND_NS elapse, so waiting warps
// do not take issue slots from the working ones.
__device__ __forceinline__ bool mbar_try(unsigned long long* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity), "r"(SUSPEND_NS)
      : "memory");
  return ok != 0;
}
// Bounded wait (at most `polls` polls of at most SUSPEND_NS each; the
// default SPIN_LIMIT is about a second) for the completion of the phase with
// the given parity; gives up early once *err is set, and sets it on timeout.
// polls = 0 gives up at once.
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, uint32_t parity, volatile int* err,
                                          long long polls = SPIN_LIMIT) {
  for (long long i = 0; i < polls; ++i) {
    if (mbar_try(b, parity)) return true;
    if ((i & 15) == 15 && *err) return false;
  }
  *err = 1;
  return false;
}
// Teardown wait for work that is certain to complete (a bulk copy already
// issued, MMAs already committed): polls up to SPIN_LIMIT times whatever
// *err says, so that a CTA that gave up elsewhere still lets its in-flight
// copies land and its MMAs finish before it frees TMEM or exits.
__device__ __forceinline__ bool mbar_drain(unsigned long long* b, uint32_t parity) {
  for (long long i = 0; i < SPIN_LIMIT; ++i)
    if (mbar_try(b, parity)) return true;
  return false;
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
// One contiguous global -> shared copy (both addresses 16-byte aligned, bytes
// a multiple of 16); completion is signalled as transaction bytes on b.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, unsigned long long* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(b))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

}  // namespace pipe
}  // namespace mrgb
