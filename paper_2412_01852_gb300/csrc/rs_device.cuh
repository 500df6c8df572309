// rs_device.cuh -- small sm_103a device helpers shared by the rotation kernels:
// mbarrier and TMA (cp.async.bulk.tensor) wrappers in inline PTX, gpu-scope
// acquire/release flags, L2-only loads/stores and bounded waits.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace rs {

// Error codes a kernel can leave in its status word (host maps them to rot_status).
enum DeviceError : int {
  kDevOk = 0,
  kDevTimeoutDependency = 1,   // a wait on another item's progress flag ran out
  kDevTimeoutTma = 2,          // a wait on a TMA transaction barrier ran out
  kDevBadItem = 3,             // a work item decoded outside the problem
  kDevCancelled = 4,           // the host asked the kernel to stop (serving)
};

// Upper bound for one wait in a kernel, in nanoseconds of %globaltimer.
// A correct run never waits this long: every wait is on work that is already
// running on a resident warp.
constexpr unsigned long long kWaitLimitNs = 4000000000ull;  // 4 s

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- gpu-scope flags --------------------------------------------------------
__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed_gpu(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Record the first error in a status word (later errors do not overwrite it).
__device__ __forceinline__ void set_error(int* status, int code) {
  atomicCAS(status, 0, code);
}

// ---- L2-coherent data movement (A is shared between SMs through L2) ---------
template <typename T> __device__ __forceinline__ T ld_cg(const T* p) { return __ldcg(p); }
template <typename T> __device__ __forceinline__ void st_cg(T* p, T v) { __stcg(p, v); }
// An L2 policy that keeps lines resident ahead of others (evict_last), and an
// FP32 store under it.
__device__ __forceinline__ unsigned long long l2_evict_last_policy() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void st_l2_keep(float* p, float v, unsigned long long policy) {
  asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(policy) : "memory");
}

// ---- mbarrier ---------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbarrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;"
               ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// One bounded probe of phase `parity`; true when that phase has completed.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(1000000u)
      : "memory");
  return ok != 0;
}
// Wait with a wall-clock limit; returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer_ns() - t0 > kWaitLimitNs) return false;
  }
  return true;
}

// Barrier waits of warps that hand tiles to one another (the warp chain,
// the split column stream), all bounded by kWaitLimitNs.  A barrier that
// hands data over (a TMA stage filled, a ring slot written) is tested
// first without suspending (most are complete when a warp gets there) and
// waited on with acquire semantics; one that only reports a slot or stage
// read (free, consumed) is arrived on and waited on relaxed: the reads it
// reports have completed, since their values were used before the arrive.
__device__ __forceinline__ bool mbar_test_acquire(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_try_relaxed(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.relaxed.cta.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void mbar_arrive_relaxed(uint64_t* bar) {
  asm volatile("mbarrier.arrive.relaxed.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_wait_data(uint64_t* bar, uint32_t parity) {
  if (mbar_test_acquire(bar, parity)) return true;
  return mbar_wait_bounded(bar, parity);
}
__device__ __forceinline__ bool mbar_wait_read(uint64_t* bar, uint32_t parity) {
  if (mbar_try_relaxed(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  while (!mbar_try_relaxed(bar, parity))
    if (globaltimer_ns() - t0 > kWaitLimitNs) return false;
  return true;
}

// ---- TMA: 2-D tiled tensor load global -> shared, completes on an mbarrier ---
__device__ __forceinline__ void tma_load_2d(void* smem_dst, const void* tmap, uint64_t* bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cta.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(smem_dst)), "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// Untiled bulk copy global -> shared (16-byte aligned addresses, size a
// multiple of 16), completing on an mbarrier.
__device__ __forceinline__ void bulk_g2s(void* smem_dst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_u32(smem_dst)), "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void prefetch_tmap(const void* tmap) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(tmap) : "memory");
}

// ---- bounded spin on a progress counter -------------------------------------
// Lane 0 waits until *flag >= need (acquire), giving up after limit_ns
// (kWaitLimitNs unless a launch sets a shorter one) or when *status becomes
// non-zero.  Returns false if the wait did not succeed.
__device__ __forceinline__ bool wait_flag_geq(const int* flag, int need, const int* status,
                                              unsigned long long limit_ns = kWaitLimitNs) {
  if (ld_acquire_gpu(flag) >= need) return true;
  const unsigned long long t0 = globaltimer_ns();
  unsigned ns = 32;
  while (true) {
    __nanosleep(ns);
    if (ns < 1024) ns <<= 1;
    if (ld_acquire_gpu(flag) >= need) return true;
    if (ld_relaxed_gpu(status) != 0) return false;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

}  // namespace rs
