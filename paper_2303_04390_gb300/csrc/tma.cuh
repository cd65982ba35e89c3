// mbarrier and 1-D bulk-copy (cp.async.bulk, the TMA engine's untiled form)
// primitives in inline PTX for sm_100-class GPUs.
#pragma once

#include <cstdint>

namespace phylo {

// try_wait rounds before a wait gives up (each round may suspend the
// thread for a bounded, hardware-defined time).
constexpr unsigned kWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Initialise an mbarrier with `count` expected arrivals and make the
// initialisation visible to the asynchronous proxy.
__device__ __forceinline__ void mbar_init_fenced(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arrive once and announce `bytes` of asynchronous copies for this phase.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                   smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// Bounded wait for the phase with parity `parity`: at most `limit`
// try_wait rounds; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          unsigned limit = kWaitLimit) {
  const uint32_t addr = smem_addr(bar);
  for (unsigned i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 1-D bulk copy global -> shared; both addresses 16-byte aligned and the
// size a multiple of 16.  Completion is counted on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src,
                                         uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Per-thread asynchronous 16-byte copy global -> shared (cached in L2
// only); both addresses 16-byte aligned.  Copies are grouped by
// cp_async_commit; cp_async_wait<N> returns once at most N of the thread's
// groups are still in flight, and makes the completed ones visible to the
// thread (a barrier then makes them visible to the block).
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Programmatic dependent launch: wait until the kernel before this one in
// the stream has completed with its writes visible, then let the kernel
// after this one start launching its CTAs (they wait the same way before
// touching memory).  Without the launch attribute both are no-ops.  Since
// every kernel waits before it releases, a kernel that has started can only
// overlap the one directly before it: everything launched earlier has
// completed, so data those kernels wrote may be read before the wait.
__device__ __forceinline__ void pdl_wait_and_release() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

}  // namespace phylo
