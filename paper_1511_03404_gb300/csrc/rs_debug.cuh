// Bounds checks on global stores for debug builds (compiled with -DRS_DEBUG).
//
// Every global store of the kernels goes through dbg_ok(index, length,
// site): in a debug build an index outside its array is recorded in a device
// word of this translation unit -- the first failure only: its site number
// and index -- and the store is dropped; nothing traps.  rs_debug_status()
// reads and clears the words of every translation unit.  In a release build
// dbg_ok is the constant true and the check compiles away.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "rs_host.h"

namespace rs {

#ifdef RS_DEBUG
constexpr bool kDebugChecks = true;
#else
constexpr bool kDebugChecks = false;
#endif

// Store sites (the site field of rs_debug_status).
enum DbgSite : uint32_t {
  kSiteUpCounts = 1, kSiteUpOffsets, kSiteUpClear, kSiteTileStatus, kSiteGroupAgg,
  kSiteGroupInc, kSiteKeyScatter, kSiteValScatter, kSiteFusedCounts, kSiteFusedClear,
  kSiteClusterOut, kSiteSmallOut, kSiteSegPlan, kSiteSegCounts, kSiteSegClear, kSiteSegState,
  kSiteSegSmallOut, kSiteMergeTile, kSiteMergeSplit, kSiteMergeOut, kSiteSampleOff,
  kSiteSampleSample, kSiteSampleSplitter, kSiteSampleCount, kSiteSampleOut, kSiteSampleBucket
};

namespace {
// bit 63: a check failed; bits 48-62: its site; bits 0-47: the index
__device__ unsigned long long g_dbg_first;

#ifdef RS_DEBUG
bool dbg_read_and_clear(uint64_t* word) {
  unsigned long long v = 0ull;
  if (cudaMemcpyFromSymbol(&v, g_dbg_first, sizeof(v)) != cudaSuccess) return false;
  const unsigned long long zero = 0ull;
  if (v != 0ull && cudaMemcpyToSymbol(g_dbg_first, &zero, sizeof(zero)) != cudaSuccess)
    return false;
  *word = v;
  return true;
}
struct DbgRegistrar {
  DbgRegistrar() { register_dbg_reader(&dbg_read_and_clear); }
} g_dbg_registrar;
#endif
}  // namespace

__device__ __forceinline__ bool dbg_ok(uint64_t i, uint64_t len, uint32_t site) {
  if constexpr (kDebugChecks) {
    if (i >= len) {
      atomicCAS(&g_dbg_first, 0ull,
                (1ull << 63) | (uint64_t(site & 0x7fffu) << 48) | (i & ((1ull << 48) - 1)));
      return false;
    }
  }
  return true;
}

}  // namespace rs
