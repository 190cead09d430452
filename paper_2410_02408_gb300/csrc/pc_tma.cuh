// Bulk asynchronous copies (cp.async.bulk, global -> shared, completing on an mbarrier)
// and the mbarrier operations used by the staged kernels.  Only data that no kernel
// writes while the copy may run (CSR arrays, block factors) is moved this way, so no
// cross-proxy fences are needed.
#pragma once

#include <stdint.h>

#include "pc_common.cuh"

namespace pc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* m, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* m, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}
// try_wait with a suspend-time hint (ns): a waiting thread sleeps instead of re-polling.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(m)), "r"(parity), "r"(20000u)
      : "memory");
  return ok != 0;
}
// dst, src 16-byte aligned; bytes a positive multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* m) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(m))
               : "memory");
}

// Bounded wait on an mbarrier phase (clock64 budget).  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* m, uint32_t parity, long long budget) {
  const long long t0 = clock64();
  while (!mbar_try_wait(m, parity)) {
    if (clock64() - t0 > budget) return false;
  }
  return true;
}

// The part of elements [e0, e1) of an array (element size ES, `total` elements) that one
// aligned bulk copy can bring in: whole 16-byte granules inside the array.  Elements
// [lo, hi) land in shared memory at (e - lo) * ES; elements of [e0, e1) outside it (only
// at an unaligned array start or at the array end) are read from global memory.
struct Window {
  int64_t lo;
  int64_t hi;
  uint32_t bytes;
};

__device__ __forceinline__ Window make_window(const void* base, int es, int64_t e0, int64_t e1, int64_t total) {
  const uint64_t b = (uint64_t)base;
  const uint64_t a0 = b + (uint64_t)e0 * es;
  const uint64_t a1 = b + (uint64_t)e1 * es;
  uint64_t lo = a0 & ~(uint64_t)15;
  const uint64_t blo = (b + 15) & ~(uint64_t)15;
  if (lo < blo) lo = blo;
  uint64_t hi = (a1 + 15) & ~(uint64_t)15;
  const uint64_t bhi = (b + (uint64_t)total * es) & ~(uint64_t)15;
  if (hi > bhi) hi = bhi;
  Window w;
  if (hi <= lo || e1 <= e0) {
    w.lo = e0;
    w.hi = e0;
    w.bytes = 0;
  } else {
    w.lo = (int64_t)((lo - b) / es);
    w.hi = (int64_t)((hi - b) / es);
    w.bytes = (uint32_t)(hi - lo);
  }
  return w;
}

__device__ __forceinline__ const void* window_src(const void* base, int es, const Window& w) {
  return (const unsigned char*)base + w.lo * es;
}

}  // namespace pc
