// Host-side plumbing shared by the translation units of the rs library:
// the arguments of one sort, the table of compiled variants, device
// properties and the optional per-kernel event timer.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "rs_common.h"

namespace rs {

struct SortArgs {
  void* keys;
  void* vals;
  void* keys_alt;
  void* vals_alt;
  uint32_t n;
  int begin_bit, end_bit;
  void* ws;
  size_t ws_bytes;
  cudaStream_t stream;
  Knobs knobs;
  int key_kind = 0;    // 0 unsigned, 1 signed, 2 float (see KeyXf)
  int descending = 0;
};

enum VariantKind { kOnesweep = 0, kSmall = 1, kOnesweepPersist = 2, kFused = 3, kCluster = 4 };

struct Variant {
  int key_bytes, val_bytes;
  int kind;
  int radix_bits, threads, items;
  uint32_t max_n;  // kSmall: largest n; kOnesweep: RS_MAX_N
  // workspace bytes for n elements over `passes` digit passes
  size_t (*workspace)(uint32_t n, int passes);
  // enqueue the whole sort; the sorted data ends in the alternate buffers
  // iff *in_alt is set on return
  cudaError_t (*run)(const SortArgs& a, int* in_alt);
  // upsweep + scan only: counts/offsets/exec mask land in the workspace
  cudaError_t (*count)(const SortArgs& a);
};

// All compiled variants of one (key_bytes, val_bytes) combination.
const Variant* variants(int key_bytes, int val_bytes, int* count);

struct DeviceInfo {
  int device;
  int sms;
  int smem_optin;
};
// Properties of the current device (cached).
const DeviceInfo& device_info();

// Opt a kernel in to `bytes` of dynamic shared memory on the current device
// (once per device) and return its resident CTAs per SM at `threads`.
int prepare_kernel(const void* func, int threads, int smem_bytes);

// Whether digit passes use programmatic dependent launch (on unless the
// environment sets RS_NO_PDL, read once; a diagnostic switch).
bool pdl_enabled();

// Per-kernel timing hooks (no-ops unless rs_profile_begin was called on this thread).
// A onesweep launch only moves data when its pass bit is set in the
// workspace's exec mask; prof_note_mask copies that mask to the host (only
// while profiling) and returns its slot, which prof_after then uses to count
// the launch's bytes exactly.
void prof_before(cudaStream_t s);
int prof_note_mask(cudaStream_t s, const uint32_t* d_exec_mask);
void prof_after(cudaStream_t s, int kind, double bytes, int mask_slot = -1, int pass = -1);

// Current fault-injection / wait-limit settings (rs_debug_set).
Knobs knobs_now();

// NVTX ranges around the library's calls and launches, for timeline tools
// (nsys, ncu --nvtx): on when the environment sets RS_NVTX (read once).
bool nvtx_enabled();
void nvtx_push(const char* name);
void nvtx_pop();
// "rs pass 0" ... "rs pass 15"
extern const char* const kPassNames[kMaxPasses];

// Debug builds: every translation unit with kernels registers a reader of its
// bounds-check word (rs_debug.cuh); rs_debug_status calls them all.  A
// reader returns false when the read failed.
using DbgReader = bool (*)(uint64_t* word);
void register_dbg_reader(DbgReader reader);

inline int num_passes(int begin_bit, int end_bit, int radix_bits) {
  return (end_bit - begin_bit + radix_bits - 1) / radix_bits;
}

}  // namespace rs
