// L2 prefetch through the bulk-copy (TMA) unit.
//
// cp.async.bulk.prefetch.L2 asks the copy unit to bring a global-memory range
// into L2 and returns at once: no register, shared memory or barrier is
// involved and nothing waits for it, so it can run many tiles ahead of the
// loads that will use the data.  The range starts on a 16-byte boundary and
// its size is a multiple of 16 bytes; it must lie inside one allocation.
#pragma once
#include <cstdint>

namespace tma {

__device__ __forceinline__ void prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Prefetch elements [k0, k1) of an array of `esize`-byte elements whose base
// is 16-byte aligned: the range is widened to 16-byte boundaries (up to
// 16 / esize - 1 elements on either side, which the allocation must hold).
__device__ __forceinline__ void prefetch_l2_range(const void* base, int64_t k0, int64_t k1, int esize) {
  if (k1 <= k0) return;
  const int64_t b0 = (k0 * esize) & ~(int64_t)15;
  const int64_t b1 = (k1 * esize + 15) & ~(int64_t)15;
  prefetch_l2(static_cast<const char*>(base) + b0, (uint32_t)(b1 - b0));
}

}  // namespace tma
