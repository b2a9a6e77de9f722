// Inline-PTX helpers shared by the slab kernels: shared-memory addresses, the
// global timer, mbarriers with bounded waits, TMA bulk copies, proxy fences,
// programmatic dependent launch and L2-only loads.
#pragma once
#include "hz_internal.h"

namespace hz {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Orders this thread's earlier generic-proxy accesses (shared and global)
// before later async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async;" ::: "memory");
}
// Same for shared memory only: issued before a TMA copy overwrites a stage
// that the block has just read with ordinary loads (a warp may pass the block
// barrier with such loads still in flight).
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Transaction bytes without an arrival: the phase cannot complete before the
// (later) arrive.expect_tx of the same phase.
__device__ __forceinline__ void mbar_expect_tx_noarrive(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while its predecessor in the stream still runs;
// pdl_wait() returns once the predecessor has completed and its memory
// operations are visible (immediately for a kernel launched without the
// attribute).  pdl_trigger() lets the successor start early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after ~2 s, raises the device flag, returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* flag) {
  if (mbar_try_wait(bar, parity)) return true;
  uint64_t t0 = gtimer();
  while (!mbar_try_wait(bar, parity)) {
    if (gtimer() - t0 > 2000000000ull) {
      atomicExch(flag, DEV_TIMEOUT);
      return false;
    }
  }
  return true;
}

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }
__device__ __forceinline__ cplx<float> ldcg(const cplx<float>* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return mk(v.x, v.y);
}
__device__ __forceinline__ cplx<double> ldcg(const cplx<double>* p) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return mk(v.x, v.y);
}

}  // namespace hz
