// Device helpers shared by the kernels of libsfs: programmatic dependent
// launch points, mbarriers, bulk copies into shared memory and bounded waits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sfs {

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  The kernels of the FISTA loop are launched
// so that the next one may start while the current one drains.  Each kernel
// does only work independent of its predecessor (shared-memory set-up,
// twiddles, first bulk copies of the constant table) before pdl_wait(), which
// returns once the predecessor grid has completed and its writes are
// visible; it then allows its own successor to launch.  Since a kernel lets
// its successor start only after its own wait, at most two grids overlap,
// and the successor's early work never touches data of the kernels before.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---------------------------------------------------------------------------
// mbarriers and bulk copies (cp.async.bulk, completion counted in bytes on
// an mbarrier)
// ---------------------------------------------------------------------------
// Bound of the drain that follows a timed-out wait (global time, ns).
constexpr uint64_t kDrainNs = 500000000ull;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
// Invalidates an mbarrier (before its shared memory is used again, or the
// barrier initialised again); nothing may still arrive on it.
__device__ __forceinline__ void mbar_inval(uint32_t bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
// Orders this thread's generic-proxy accesses of global and shared memory
// against its async-proxy (bulk / tensor copy, MMA operand) accesses, in
// both directions.
__device__ __forceinline__ void fence_proxy_async_all() {
  asm volatile("fence.proxy.async;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
// Plain arrive (count one) on an mbarrier.
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
// L2 policy for data read once per launch and larger than the L2 (the
// generator table of the large workloads): evict first, so that the
// spectra the kernels re-read stay resident.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
// bulk_g2s with an L2 cache policy.
__device__ __forceinline__ void bulk_g2s_hint(uint32_t dst, const void* src, uint32_t bytes,
                                              uint32_t bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, "
      "[%3], %4;" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar), "l"(policy)
      : "memory");
}
// The table copy of the contractions: with `stream` set, evict-first.
__device__ __forceinline__ void bulk_g2s_table(uint32_t dst, const void* src, uint32_t bytes,
                                               uint32_t bar, bool stream, uint64_t policy) {
  if (stream)
    bulk_g2s_hint(dst, src, bytes, bar, policy);
  else
    bulk_g2s(dst, src, bytes, bar);
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for phase `parity` of the mbarrier; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (true) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

}  // namespace sfs
