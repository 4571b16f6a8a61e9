// Device-side building blocks shared by the LINVIEW kernels: mbarrier and
// TMA (cp.async.bulk.tensor) wrappers in inline PTX for sm_103a, with every
// wait bounded so that a lost transaction turns into a latched error status
// instead of a hung GPU.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lv {

// Device status word bits (latched by kernels, read by linview_sync).
enum : unsigned {
  kStatusTimeout = 1u,
  kStatusNonFinite = 2u,
  kStatusSingular = 4u,
};

// ~ several seconds of polling on a 2 GHz part before a wait gives up.
constexpr long long kMaxPolls = 1ll << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// try_wait with an explicit suspend-time hint: a thread whose phase is not
// complete sleeps until it completes or kSuspendHintNs pass, instead of
// returning after the short default limit, so waiting warps issue few
// instructions and leave the issue slots to the warps that compute.
constexpr uint32_t kSuspendHintNs = 8192;

__device__ __forceinline__ bool mbar_try_wait_suspend(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendHintNs)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wall-clock limit of one bounded wait (2 s).
constexpr uint64_t kWaitLimitNs = 2000000000ull;

// Bounded wait on phase ``parity``; returns false (and latches a timeout in
// *status) if the barrier did not complete within limit_ns (kWaitLimitNs for
// the passes) or kMaxPolls polls, whichever comes first.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  unsigned* status,
                                                  uint64_t limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (long long i = 0; i < kMaxPolls; ++i) {
    if (mbar_try_wait_suspend(bar, parity)) return true;
    if ((i & 255) == 255 && global_ns() - t0 > limit_ns) break;
  }
  if (status) atomicOr(status, kStatusTimeout);
  return false;
}

// 2-D tiled TMA load of a box at element coordinates (x = column, y = row)
// into shared memory, completing ``bytes`` transaction bytes on ``bar``.
// x * sizeof(element) must be a multiple of 16 bytes (callers pass multiples
// of the box width, which is 1 KB).
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// 2-D tiled TMA store of a box from shared memory at element coordinates
// (x, y), committed to the thread's bulk async-group.  The writes of the box
// by other threads must be made visible to the async proxy first
// (fence_proxy_async by each writer, then a barrier).  Elements outside the
// tensor map's extent are not written.
__device__ __forceinline__ void tma_store_2d(const void* tmap, const void* src, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
          reinterpret_cast<uint64_t>(tmap)),
      "r"(x), "r"(y), "r"(smem_u32(src))
      : "memory");
}

__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// all but the newest N bulk groups of this thread have finished reading
// their shared-memory sources
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
// all bulk groups of this thread are complete (writes performed)
__device__ __forceinline__ void bulk_wait0() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
      : "memory");
}

// 4-byte asynchronous global->shared copy; valid == false writes zero.
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(smem_dst)),
               "l"(reinterpret_cast<uint64_t>(gsrc)), "r"(valid ? 4 : 0)
               : "memory");
}

// Arrive on ``bar`` once every cp.async this thread issued so far has landed
// (the barrier's expected count includes this arrival).
__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const void* tmap) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmap)) : "memory");
}

// q = idx / d, r = idx % d for a flat element index: 32-bit arithmetic
// whenever the index fits (a 64-bit division by a runtime divisor is a long
// instruction sequence, which dominates the small element-wise kernels).
__device__ __forceinline__ void split_index(int64_t idx, int d, int& q, int& r) {
  if (idx <= 0x7fffffffll) {
    const unsigned u = (unsigned)idx, ud = (unsigned)d;
    q = (int)(u / ud);
    r = (int)(u - (unsigned)q * ud);
  } else {
    q = (int)(idx / d);
    r = (int)(idx - (int64_t)q * d);
  }
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while the kernel before it drains; griddep_wait()
// blocks until that kernel has completed and its writes are visible, and
// griddep_launch_dependents() lets the next kernel start early.  Work before
// griddep_wait() may only touch data that the previous kernel does not write.
__device__ __forceinline__ void griddep_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// 16-byte vector helpers for float (4 lanes) and double (2 lanes).
template <typename T>
struct Vec;
template <>
struct Vec<float> {
  static constexpr int N = 4;
  using type = float4;
};
template <>
struct Vec<double> {
  static constexpr int N = 2;
  using type = double2;
};

}  // namespace lv
