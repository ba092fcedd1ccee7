// Device kernels of the LSD radix sort (arXiv 1511.03404, Sec. 2.6).
//
// One sort = one upsweep + one onesweep launch per digit pass:
//   k_upsweep   reads the keys once and builds the digit histogram of every
//               pass (the "count" step of each counting sort); its last CTA
//               takes the exclusive scan of each histogram (the "prefix"
//               step) and decides which passes move data.
//   k_onesweep  one digit pass: the tile's keys are ranked within the tile
//               (stable: ranking-unit-major, a unit being a warp or half a
//               warp, then item, then lane order), the tile's
//               digit counts are published for the following tiles, the
//               tile's global digit offsets come from a decoupled look-back
//               over the preceding tiles, and the tile is scattered through
//               shared memory so that each digit run is written contiguously
//               (the stable "scatter" step).
//   k_small_sort  arrays that fit one tile: all passes in one CTA, in shared
//               memory, in a single launch.
// All arithmetic is on unsigned integers; results are exact.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "rs_common.h"
#include "rs_debug.cuh"

namespace rs {

constexpr unsigned kFull = 0xffffffffu;

template <int VB>
using ValT = typename std::conditional<VB == 8, uint64_t, uint32_t>::type;

// ---------------------------------------------------------------- helpers

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint4 ld_relaxed_v4(const uint32_t* p) {
  uint4 v;
  asm volatile("ld.relaxed.gpu.global.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p)
               : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Stable rank of ITEMS digits per lane inside one warp.  Item j of lane l
// comes after item j' < j of every lane and after item j of lanes < l.
// The lanes holding the same digit (the "peers") are found with one shared
// atomic OR of the lane bit into a per-warp word for that digit (mm, all zero
// on entry and on exit): on sm_103a this sustains several times the rate of
// match.any.  The warp's running count per digit (wh) is updated by the peer
// group's highest lane; pos[j] receives the count of earlier equal digits.
template <int ITEMS>
__device__ __forceinline__ void warp_rank(const uint32_t (&dg)[ITEMS], uint32_t (&pos)[ITEMS],
                                          uint32_t* wh, uint32_t* mm, int lane) {
  const uint32_t bit = 1u << lane;
  const uint32_t lt = bit - 1u;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const uint32_t d = dg[j];
    atomicOr(&mm[d], bit);
    __syncwarp();
    const uint32_t peers = mm[d];
    __syncwarp();
    const int leader = 31 - __clz(peers);
    uint32_t before = 0u;
    if (lane == leader) {
      mm[d] = 0u;
      before = wh[d];
      wh[d] = before + uint32_t(__popc(peers));
    }
    __syncwarp();
    pos[j] = __shfl_sync(kFull, before, leader) + uint32_t(__popc(peers & lt));
  }
}

// The same rank with digit and result in one register per item: dp[j] holds
// the digit on entry and (digit << 16) | rank on exit (ITEMS * 32 <= 65536).
// Every lane reads the warp's running count of its digit next to the peer
// mask, so no shuffle is needed; only the peer group's highest lane (the one
// whose bit is the mask's top bit) writes back, by predicated stores.
template <int ITEMS>
__device__ __forceinline__ void warp_rank_packed(uint32_t (&dp)[ITEMS], uint32_t* wh,
                                                 uint32_t* mm, int lane) {
  static_assert(ITEMS * 32 <= 65536, "ranks fit 16 bits");
  const uint32_t bit = 1u << lane;
  const uint32_t lt = bit - 1u;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const uint32_t d = dp[j];
    atomicOr(&mm[d], bit);
    __syncwarp();
    const uint32_t peers = mm[d];
    __syncwarp();
    const int leader = 31 - __clz(peers);
    uint32_t before = 0u;
    if (lane == leader) {
      mm[d] = 0u;
      before = atomicAdd(&wh[d], uint32_t(__popc(peers)));
    }
    __syncwarp();
    dp[j] = (d << 16) | (__shfl_sync(kFull, before, leader) + uint32_t(__popc(peers & lt)));
  }
}

// Rank within half-warp units: lanes 0-15 and lanes 16-31 of a warp rank
// their items separately, each half against its own counter words.  A word
// holds the half's running count of the digit in its upper 16 bits and the
// peer mask of the current item (one bit per lane of the half) in its lower
// 16 bits, so an item costs a shared atomic OR, a load and the leader's store
// (the leader's store clears the mask and advances the count at once).  wh
// points at the half's own [RADIX] words; dp as in warp_rank_packed.
template <int ITEMS>
__device__ __forceinline__ void half_rank_packed(uint32_t (&dp)[ITEMS], uint32_t* wh, int lane) {
  static_assert(ITEMS * 16 < 65536, "counts fit 16 bits");
  const uint32_t sub = uint32_t(lane & 15);
  const uint32_t bit = 1u << sub;
  const uint32_t lt = bit - 1u;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const uint32_t d = dp[j];
    atomicOr(&wh[d], bit);
    __syncwarp();
    const uint32_t v = wh[d];
    __syncwarp();
    const uint32_t peers = v & 0xffffu;
    const uint32_t before = v >> 16;
    if (sub == uint32_t(31 - __clz(peers))) wh[d] = (before + uint32_t(__popc(peers))) << 16;
    __syncwarp();  // the next item's atomics come after the leader's store
    dp[j] = (d << 16) | (before + uint32_t(__popc(peers & lt)));
  }
}

template <class K>
__device__ __forceinline__ uint32_t digit_of(K key, uint32_t shift, uint32_t mask) {
  return static_cast<uint32_t>(key >> shift) & mask;
}

// Record the first device-side error of a call (later ones are dropped).
__device__ __forceinline__ void report_error(Ctrl* ctrl, uint32_t code, uint32_t info) {
  if (atomicCAS(&ctrl->error, 0u, code) == 0u) atomicExch(&ctrl->error_info, info);
}

// Per-call record read by rs_workspace_stats: the shape of the sort and the
// %globaltimer start of its first kernel (one thread), then times relative
// to that start, at least 1 so that 0 means "not reached".
__device__ __forceinline__ void stat_begin(Ctrl* ctrl, uint32_t n, uint32_t shape) {
  const uint64_t t = global_ns();
  ctrl->t0_lo = uint32_t(t);
  ctrl->t0_hi = uint32_t(t >> 32);
  ctrl->stat_n = n;
  ctrl->stat_shape = shape;
}

// The forms that do not start from a cleared control block clear the
// record's times themselves (one thread, before any other writes them).
__device__ __forceinline__ void stat_clear_times(Ctrl* ctrl) {
  ctrl->t_upsweep = 0u;
#pragma unroll
  for (int p = 0; p < kMaxPasses; ++p) ctrl->t_pass[p][0] = ctrl->t_pass[p][1] = 0u;
}

__device__ __forceinline__ uint32_t stat_now(const Ctrl* ctrl) {
  const uint64_t t0 = (uint64_t(ctrl->t0_hi) << 32) | ctrl->t0_lo;
  const uint64_t d = global_ns() - t0;
  return d >= 0xffffffffull ? 0xffffffffu : (d == 0 ? 1u : uint32_t(d));
}

// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialization may start while the kernel before it on the stream is still
// running; pdl_wait() blocks (in hardware) until that kernel has completed and
// its memory operations are visible, and is a no-op for an ordinary launch.
// pdl_launch_dependents() lets the next such kernel be scheduled once every
// CTA of this grid has called it or exited.
__device__ __forceinline__ void pdl_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded wait until *p >= target.  False when it ran out or another CTA
// already reported an error.
__device__ __noinline__ static bool wait_geq(const uint32_t* p, uint32_t target, Ctrl* ctrl,
                                             uint64_t timeout_ns, uint32_t info) {
  if (ld_acquire(p) >= target) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    if (ld_acquire(p) >= target) return true;
    if ((it & 63u) == 0u) {
      if (ld_relaxed(&ctrl->error) != 0u) return false;
      if (global_ns() - t0 > timeout_ns) {
        report_error(ctrl, kDevTimeout, info);
        return false;
      }
    }
  }
}


__device__ __forceinline__ uint32_t warp_inclusive_scan(uint32_t x, int lane) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    uint32_t y = __shfl_up_sync(kFull, x, off);
    if (lane >= off) x += y;
  }
  return x;
}

// Exclusive scan of one value per thread across the CTA.  s_tot holds 32
// words.  Every thread must call it; the caller separates two calls with a
// barrier.
template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* s_tot) {
  constexpr int WARPS = THREADS / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t inc = warp_inclusive_scan(x, lane);
  if (lane == 31) s_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const uint32_t t = lane < WARPS ? s_tot[lane] : 0u;
    const uint32_t ti = warp_inclusive_scan(t, lane);
    s_tot[lane] = ti - t;
  }
  __syncthreads();
  return inc - x + s_tot[warp];
}

// Wait (bounded) until a look-back status word has a flag.  Returns the word,
// or kFlagErr when the wait ran out or another CTA already reported an error.
static __device__ __noinline__ uint32_t wait_status(const uint32_t* p, Ctrl* ctrl, uint64_t timeout_ns,
                                             uint32_t tile) {
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    const uint32_t s = ld_relaxed(p);
    if (s & kFlagMask) return s;
    if ((it & 63u) == 0u) {
      if (ld_relaxed(&ctrl->error) != 0u) return kFlagErr;
      if (global_ns() - t0 > timeout_ns) {
        report_error(ctrl, kDevTimeout, tile);
        return kFlagErr;
      }
    }
  }
}

// --------------------------------------------------------------- upsweep

// Digit histograms of every pass in one read of the keys, then (last CTA)
// the exclusive scan of each and the set of passes that move data.
//
// Shared counters are laid out [pass][digit][slot] with slot = lane mod
// SLOTS: with 32 slots (32-bit keys) lane l only ever touches bank l, so a
// warp's 32 increments never meet on a bank whatever the digits are (the zero
// and sorted distributions included).  64-bit keys have twice the passes and
// use 16 slots to stay within shared memory.  FULL: the bit range is the whole
// key and r = 8, so every digit is one byte, taken with a byte permute.
template <class K, int RADIX_BITS, int THREADS, int MAXP, bool FULL>
__global__ void __launch_bounds__(THREADS, 1)
    k_upsweep(const K* __restrict__ keys, uint32_t n, int begin_bit, int end_bit, int passes,
              uint32_t* __restrict__ counts, uint32_t* __restrict__ offsets,
              Ctrl* __restrict__ ctrl, uint4* __restrict__ zero_base, uint64_t zero_vec4,
              KeyXf<K> xf, bool early_dependents, uint32_t shape) {
  constexpr int RADIX = 1 << RADIX_BITS;
  constexpr int SLOTS = sizeof(K) == 4 ? 32 : 16;
  constexpr int VEC = 16 / int(sizeof(K));
  constexpr int UNROLL = 4;
  static_assert(RADIX <= THREADS, "one thread per digit in the scan");
  static_assert(!FULL || RADIX_BITS == 8, "byte digits");

  extern __shared__ uint32_t sh[];  // [passes][RADIX][SLOTS]
  __shared__ uint32_t s_tot[32];
  __shared__ int s_last;
  // a first pass that fills the GPU may be scheduled beside this grid (one
  // that does not is scheduled as this grid's CTAs exit)
  if (early_dependents) pdl_launch_dependents();

  const int tid = threadIdx.x, lane = tid & 31;
  if (shape != 0u && blockIdx.x == 0 && tid == 0) stat_begin(ctrl, n, shape);
  const uint32_t slot = uint32_t(lane & (SLOTS - 1));
  uint32_t shiftp[MAXP], maskp[MAXP];
#pragma unroll
  for (int p = 0; p < MAXP; ++p) {
    const int lo = begin_bit + p * RADIX_BITS;
    const int hi = min(lo + RADIX_BITS, end_bit);
    shiftp[p] = p < passes ? uint32_t(lo) : 0u;
    maskp[p] = p < passes ? ((1u << (hi - lo)) - 1u) : 0u;
  }
  const int words = passes * RADIX * SLOTS;
  for (int i = tid; i < words; i += THREADS) sh[i] = 0u;
  __syncthreads();

  // XF: the digits are those of the transformed key (a compile-time switch,
  // so that plain unsigned sorts pay nothing for it)
  auto count_key = [&](K k, auto XF) {
    if constexpr (decltype(XF)::value) k = xf_fwd(k, xf);
#pragma unroll
    for (int p = 0; p < MAXP; ++p) {
      if (FULL || p < passes) {
        uint32_t d;
        if constexpr (FULL) {
          const uint32_t half = (sizeof(K) == 8 && p >= 4) ? uint32_t(uint64_t(k) >> 32)
                                                           : uint32_t(k);
          d = __byte_perm(half, 0u, 0x4440u | uint32_t(p & 3));
        } else {
          d = digit_of(k, shiftp[p], maskp[p]);
        }
        atomicAdd(&sh[(p * RADIX + int(d)) * SLOTS + int(slot)], 1u);
      }
    }
  };

  // 16-byte aligned body, scalar head and tail
  const uintptr_t addr = reinterpret_cast<uintptr_t>(keys);
  uint32_t head = uint32_t(((16u - (addr & 15u)) & 15u) / sizeof(K));
  if (head > n) head = n;
  const uint32_t nvec = (n - head) / VEC;
  const uint32_t tail = head + nvec * VEC;
  const uint4* vp = reinterpret_cast<const uint4*>(keys + head);
  const uint32_t stride = gridDim.x * THREADS;
  auto count_all = [&](auto XF) {
    if (blockIdx.x == 0) {
      if (uint32_t(tid) < head) count_key(keys[tid], XF);
      if (uint32_t(tid) < n - tail) count_key(keys[tail + tid], XF);
    }
    for (uint32_t base = blockIdx.x * THREADS + tid; base < nvec; base += stride * UNROLL) {
      uint4 buf[UNROLL];
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) {
        const uint32_t i = base + uint32_t(u) * stride;
        if (i < nvec) buf[u] = vp[i];
      }
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) {
        const uint32_t i = base + uint32_t(u) * stride;
        if (i < nvec) {
          const K* ks = reinterpret_cast<const K*>(&buf[u]);
#pragma unroll
          for (int e = 0; e < VEC; ++e) count_key(ks[e], XF);
        }
      }
    }
  };
  if (xf.on)
    count_all(std::true_type{});
  else
    count_all(std::false_type{});
  __syncthreads();
  // drain: one (pass, digit) per thread, summed over its slots
  for (int w = tid; w < passes * RADIX; w += THREADS) {
    const uint32_t* row = sh + w * SLOTS;
    uint32_t c = 0u;
#pragma unroll 8
    for (int l = 0; l < SLOTS; ++l) c += row[(l + lane) & (SLOTS - 1)];  // rotated: no bank conflicts
    if (c && dbg_ok(w, uint64_t(passes) * RADIX, kSiteUpCounts)) atomicAdd(&counts[w], c);
  }

  // clear the look-back status words of every pass of this call
  for (uint64_t i = uint64_t(blockIdx.x) * THREADS + tid; i < zero_vec4; i += stride)
    if (dbg_ok(i, zero_vec4, kSiteUpClear)) zero_base[i] = make_uint4(0u, 0u, 0u, 0u);

  // last CTA: scan each histogram, choose the passes that move data
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(&ctrl->hist_ticket, 1u) == gridDim.x - 1u);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  uint32_t exec = 0u;
  for (int p = 0; p < passes; ++p) {
    const uint32_t c = tid < RADIX ? ld_relaxed(&counts[p * RADIX + tid]) : 0u;
    const uint32_t e = block_exclusive_scan<THREADS>(c, s_tot);
    if (tid < RADIX && dbg_ok(uint64_t(p) * RADIX + tid, uint64_t(passes) * RADIX, kSiteUpOffsets))
      offsets[p * RADIX + tid] = e;
    // a pass in which one digit value holds every key leaves the order as it is
    const int one_digit = __syncthreads_or(tid < RADIX && c == n);
    if (!one_digit) exec |= 1u << p;
  }
  if (tid == 0) {
    // the sorted data must end in the buffer the host named (pass count
    // parity): if skipping changed the parity, the lowest skipped pass runs
    if ((__popc(exec) & 1) != (passes & 1)) {
      const uint32_t skipped = ~exec & ((1u << passes) - 1u);
      exec |= skipped & (0u - skipped);
    }
    ctrl->exec_mask = exec;
    if (shape != 0u) ctrl->t_upsweep = stat_now(ctrl);
  }
}

// -------------------------------------------------------------- onesweep

// Words of the zero source of the counter-clearing bulk copies: the counters
// of up to 32 half-warp units (512 threads) x 256 digits.
constexpr int kZeroWords = 8192;

// UNIT: lanes per ranking unit, 32 (a warp, warp_rank_packed) or 16 (half a
// warp, half_rank_packed).
// INPLACE (keys only, half-warp units): the keys are staged in (digit, input)
// order in the key buffer itself, which is free once every thread holds its
// keys in registers; there is no separate stage, so the tile costs its keys'
// bytes of shared memory once instead of twice.
template <class K, int VB, int RADIX_BITS, int THREADS, int ITEMS, int UNIT = 32,
          bool INPLACE = false>
struct OnesweepSmem {
  static_assert(UNIT == 32 || UNIT == 16, "warp or half-warp ranking units");
  static_assert(!INPLACE || (VB == 0 && UNIT == 16), "in-place stage: keys only, half-warp units");
  static constexpr int RADIX = 1 << RADIX_BITS;
  static constexpr int WARPS = THREADS / 32;
  static constexpr int UNITS = THREADS / UNIT;
  static constexpr int TILE = THREADS * ITEMS;
  static constexpr int ELEM = (int(sizeof(K)) > VB) ? int(sizeof(K)) : VB;
  static constexpr int WH = 0;                              // u32 [UNITS][RADIX] unit counters
  // half-warp units: the counters are cleared by a bulk copy with each tile's keys
  static constexpr uint32_t ZERO_BYTES = UNIT == 16 ? uint32_t(UNITS * RADIX * 4) : 0u;
  static_assert(ZERO_BYTES <= kZeroWords * 4 && ZERO_BYTES % 16 == 0, "one bulk copy of zeros");
  static constexpr int CNT = WH + UNITS * RADIX * 4;       // u32 [RADIX] tile counts
  static constexpr int TSTART = CNT + RADIX * 4;           // u32 [RADIX] tile digit starts
  static constexpr int GBASE = TSTART + RADIX * 4;         // u32 [RADIX] global base
  static constexpr int TOT = GBASE + RADIX * 4;            // u32 [32]
  static constexpr int MISC = TOT + 32 * 4;                // u32 [8]: tile, abort, next tile, ...
  static constexpr int MBAR = MISC + 32;                   // u64 [2] mbarriers: keys, values
  // the tile's keys as loaded (+16 B skew); once they are staged in OUT, the
  // tile's values are loaded here
  static constexpr int KIN = (MBAR + 16 + 15) / 16 * 16;
  // the tile in (digit, input) order: keys, then values; during the rank of
  // warp units it holds the warps' peer masks (u32 [WARPS][RADIX])
  static constexpr int OUT = INPLACE ? KIN : KIN + TILE * ELEM + 16;
  static constexpr int MM = OUT;
  static constexpr int OUT_BYTES =
      TILE * ELEM > WARPS * RADIX * 4 ? TILE * ELEM : WARPS * RADIX * 4;
  static constexpr int BYTES = INPLACE ? KIN + TILE * ELEM + 16 : OUT + OUT_BYTES;
};

// Operands of one tile of one digit pass over one array (or one segment).
template <class K, int VB>
struct TileArgs {
  const K* ksrc;
  K* kdst;
  const ValT<VB>* vsrc;
  ValT<VB>* vdst;
  uint32_t n;                   // elements of the array / segment
  uint32_t tile;                // tile index inside the array / segment
  uint32_t shift, mask;         // digit of this pass: (key >> shift) & mask
  const uint32_t* pass_offsets; // [RADIX] global digit offsets of this pass
  uint32_t* status;             // [tiles/4][RADIX][4] look-back words of this pass
  uint32_t tile0;               // index of this array's tile 0 in status (a segment's first tile)
  uint32_t* gagg;               // [groups/4][RADIX][4] group counts of this pass, or null (flat walk)
  uint32_t* ginc;               // [groups/4][RADIX][4] group inclusive prefixes of this pass
  uint32_t tiles;               // tiles of this array
  uint64_t lb_words;            // words in status (debug bounds checks only)
  uint64_t g_words;             // words in gagg / ginc (debug bounds checks only)
  bool silent;                  // test-only: publish nothing for this tile
  bool lb_small;                // test-only: 8-word look-back windows
  bool dbg_bad;                 // debug builds, test-only: scatter indices pushed past n
  uint64_t* trace;              // test-only: 16 phase stamps / counters of this tile, or null
  KeyXf<K> xf;                  // order-preserving key transform of the sort
  bool xin;                     // the source holds untransformed keys: apply xf on load
  bool xout;                    // write untransformed keys (apply xf's inverse)
};

__device__ __forceinline__ uint32_t sm_id() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}

// test-only phase stamp (thread 0)
__device__ __forceinline__ void stamp(uint64_t* tr, int k) {
  if (tr != nullptr && threadIdx.x == 0) tr[k] = global_ns();
}

// ---- look-back walks (one thread per digit)

// Bounded wait until a group word reports `need` contributing tiles.
static __device__ __noinline__ uint32_t wait_group(const uint32_t* p, uint32_t need, Ctrl* ctrl,
                                                   uint64_t timeout_ns, uint32_t tile, bool* ok) {
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    const uint32_t w = ld_relaxed(p);
    if ((w >> 24) >= need) {
      *ok = true;
      return w;
    }
    if ((it & 63u) == 0u) {
      if (ld_relaxed(&ctrl->error) != 0u) break;
      if (global_ns() - t0 > timeout_ns) {
        report_error(ctrl, kDevTimeout, tile);
        break;
      }
    }
  }
  *ok = false;
  return 0u;
}

// test-only counters of digit 0's look-back (thread 0)
__device__ __forceinline__ void trace_add(uint64_t* tr, int k, uint64_t v) {
  if (tr != nullptr && threadIdx.x == 0) tr[k] += v;
}

// Walk the tiles from, from-1, ..., lo (indices into status) of one digit,
// nearest first, adding their published counts to excl until an inclusive
// prefix (done).  NB 16-byte L2 loads fetch a window of 4*NB tiles at once;
// a warp's load is one contiguous 512-byte block (32 digits x 4 tiles).
template <int RADIX, int NB>
__device__ __forceinline__ void walk_tiles(const uint32_t* status, uint32_t d, int32_t from,
                                           int32_t lo, uint32_t& excl, bool& done, bool& gave_up,
                                           Ctrl* ctrl, uint64_t timeout_ns, uint32_t tile,
                                           uint64_t* tr) {
  int32_t hi = from;
  while (!done && !gave_up && hi >= lo) {
    trace_add(tr, 10, 1);
    const int32_t b0 = hi >> 2;
    uint4 v[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      const int32_t b = b0 - k;
      v[k] = (4 * b + 3 >= lo)
                 ? __ldcg(reinterpret_cast<const uint4*>(status + (size_t(b) * RADIX + d) * 4))
                 : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int k = 0; k < NB; ++k) {
#pragma unroll
      for (int c = 3; c >= 0; --c) {
        const int32_t a = 4 * (b0 - k) + c;
        if (done || gave_up || a > hi || a < lo) continue;
        uint32_t sw = c == 0 ? v[k].x : c == 1 ? v[k].y : c == 2 ? v[k].z : v[k].w;
        if ((sw & kFlagMask) == 0u) {
          trace_add(tr, 12, 1);
          sw = wait_status(status + lb_index<RADIX>(uint32_t(a), d), ctrl, timeout_ns, tile);
        }
        const uint32_t f = sw & kFlagMask;
        if (f == kFlagErr) {
          gave_up = true;
        } else {
          excl += sw & kValueMask;
          if (f == kFlagInc) done = true;
        }
      }
    }
    hi = 4 * (b0 - NB + 1) - 1;
  }
}

// ---- bulk (TMA engine) copies global -> shared, completed on an mbarrier

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Before the barrier's shared memory is used for anything else.
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
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
  return ok != 0u;
}

// dst and src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Bounded wait for phase `parity` of the tile-load barrier.  False when the
// limit ran out (the error is recorded); in that case the caller waits once
// more, again bounded, so that no copy is still landing when it leaves.
__device__ __noinline__ static bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                      Ctrl* ctrl, uint64_t timeout_ns,
                                                      uint32_t info) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > timeout_ns) {
      report_error(ctrl, kDevTimeout, info);
      return false;
    }
  }
}

// Shared-memory staging of elements [0, len) of src: element i lands at byte
// (skew + i * sizeof(T)) of `buf`, skew = src address mod 16, so that the
// 16-byte aligned middle ("body") goes by one bulk copy while the few head
// and tail elements are loaded by threads.
template <class T>
struct Stage {
  uint32_t skew, head, body, head_n, tail0;
  __device__ __forceinline__ Stage(const T* src, uint32_t len) {
    skew = uint32_t(reinterpret_cast<uintptr_t>(src) & 15u);
    const uint32_t bytes = len * uint32_t(sizeof(T));
    head = (16u - skew) & 15u;
    if (head > bytes) head = bytes;
    body = (bytes - head) & ~15u;
    head_n = head / uint32_t(sizeof(T));
    tail0 = (head + body) / uint32_t(sizeof(T));
  }
  __device__ __forceinline__ T* at(unsigned char* buf) const {
    return reinterpret_cast<T*>(buf + skew);
  }
  // thread 0 only
  __device__ __forceinline__ void issue(unsigned char* buf, const T* src, uint64_t* bar) const {
    if (body)
      bulk_load(buf + skew + head, reinterpret_cast<const unsigned char*>(src) + head, body, bar);
  }
  // every thread; L2 loads, since other CTAs of the same kernel may have
  // written the source
  __device__ __forceinline__ void edges(unsigned char* buf, const T* src, uint32_t len) const {
    T* s = at(buf);
    const uint32_t tid = threadIdx.x;
    if (tid < head_n) s[tid] = __ldcg(src + tid);
    if (tid < len - tail0) s[tail0 + tid] = __ldcg(src + tail0 + tid);
  }
};

// Zeros in global memory, the source of the bulk copies that clear the rank
// counters of a tile (one copy per TU; never written).
namespace {
__device__ __align__(128) uint32_t g_zero_words[kZeroWords];
}

// Start staging the keys of tile `tile` of an array of n keys into the key
// buffer: one bulk copy issued by thread 0 on `bar`, head/tail elements and
// the past-the-end sentinels written by every thread.  zero_dst (optional):
// zero_bytes (a multiple of 16, at most kZeroWords words) of shared memory cleared by a
// second bulk copy on the same barrier, so that the tile's counters are zero
// once its keys have landed, without a store loop on the shared-memory pipe.
template <class K, int THREADS, int TILE, bool CG>
__device__ __forceinline__ void stage_keys(unsigned char* kin, const K* ksrc, uint32_t n,
                                           uint32_t tile, uint64_t* bar,
                                           void* zero_dst = nullptr, uint32_t zero_bytes = 0u) {
  const uint32_t tile_base = tile * uint32_t(TILE);
  const uint32_t tile_len = min(uint32_t(TILE), n - tile_base);
  const K* gk = ksrc + tile_base;
  const Stage<K> sk(gk, tile_len);
  if (threadIdx.x == 0) {
    // shared memory this CTA used through ordinary loads and stores before is
    // about to be written by the copy engine; and, when the source was written
    // by other CTAs of this kernel, those stores must be ordered before the
    // copy engine reads them
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if constexpr (CG) asm volatile("fence.proxy.async.global;" ::: "memory");
    mbar_arrive_expect_tx(bar, sk.body + zero_bytes);
    sk.issue(kin, gk, bar);
    if (zero_bytes) bulk_load(zero_dst, g_zero_words, zero_bytes, bar);
  }
  sk.edges(kin, gk, tile_len);
  // past the end: the largest digit, so these items rank after every key of
  // the tile and are never written out
  K* s_kin = sk.at(kin);
  for (uint32_t i = tile_len + threadIdx.x; i < uint32_t(TILE); i += THREADS) s_kin[i] = ~K(0);
}

// Persistent CTAs: where the next tile id comes from.
struct Prefetch {
  uint32_t* counter;  // the pass's tile counter
  uint32_t tiles;
};

// One tile of one counting-sort pass (Sec. 2.6): stage the tile's keys in
// shared memory, rank them, publish the tile's digit counts, look back, and
// scatter stably; the values are fetched into the freed key buffer while the
// look-back and the key scatter run.  Every thread of the CTA calls it.
// Returns false (CTA-uniform) when a bounded wait gave up, in which case
// nothing of this tile was written and no copy into shared memory is pending.
//
// PERSIST: the calling kernel keeps the CTA resident over many tiles.  The
// barriers are initialised once by the kernel, this tile's keys were staged
// by the previous call (or the kernel's prologue) on barrier phase `parity`,
// and as soon as the key buffer is free again this call takes the next tile
// id (s_misc[3]) and starts staging its keys (s_misc[4] = 1), overlapping the
// end of this tile.
template <class K, int VB, int RADIX_BITS, int THREADS, int ITEMS, bool CG, bool PERSIST = false,
          int UNIT = 32, bool INPLACE = false>
__device__ __forceinline__ bool onesweep_tile(const TileArgs<K, VB>& t, Ctrl* ctrl,
                                              uint64_t timeout_ns, unsigned char* smem,
                                              uint32_t parity = 0u,
                                              const Prefetch* pf = nullptr) {
  using V = ValT<VB>;
  using S = OnesweepSmem<K, VB, RADIX_BITS, THREADS, ITEMS, UNIT, INPLACE>;
  constexpr int RADIX = S::RADIX, WARPS = S::WARPS, UNITS = S::UNITS, TILE = S::TILE;
  static_assert(RADIX <= THREADS, "one thread per digit");
  static_assert(TILE <= 65536, "stage slots fit 16 bits");
  uint32_t* s_wh = reinterpret_cast<uint32_t*>(smem + S::WH);
  uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem + S::CNT);
  uint32_t* s_tstart = reinterpret_cast<uint32_t*>(smem + S::TSTART);
  uint32_t* s_gbase = reinterpret_cast<uint32_t*>(smem + S::GBASE);
  uint32_t* s_tot = reinterpret_cast<uint32_t*>(smem + S::TOT);
  uint32_t* s_misc = reinterpret_cast<uint32_t*>(smem + S::MISC);
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + S::MBAR);  // [0] keys, [1] values
  uint32_t* s_mm = reinterpret_cast<uint32_t*>(smem + S::MM);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  const uint32_t tile = t.tile, n = t.n;
  const uint32_t tile_base = tile * uint32_t(TILE);
  const uint32_t tile_len = min(uint32_t(TILE), n - tile_base);
  stamp(t.trace, 0);
  if (t.trace != nullptr && tid == 0) t.trace[7] = sm_id();

  if constexpr (!PERSIST) {
    if (tid == 0) {
      mbar_init(&s_bar[0]);
      if constexpr (VB > 0) mbar_init(&s_bar[1]);
    }
    __syncthreads();
    // ---- stage the tile's keys (half-warp units: and clear the counters)
    stage_keys<K, THREADS, TILE, CG>(smem + S::KIN, t.ksrc, n, tile, &s_bar[0],
                                     smem + S::WH, S::ZERO_BYTES);
  }
  if (tid == 0) s_misc[1] = 0u;
  K* s_kin = Stage<K>(t.ksrc + tile_base, tile_len).at(smem + S::KIN);
  if constexpr (UNIT == 32) {
    for (int i = tid; i < WARPS * RADIX; i += THREADS) {
      s_wh[i] = 0u;
      s_mm[i] = 0u;
    }
  }  // half-warp units: the bulk copy that staged the keys cleared the counters
  bool landed = mbar_wait_bounded(&s_bar[0], parity, ctrl, timeout_ns, tile);
  if (!landed) landed = mbar_wait_bounded(&s_bar[0], parity, ctrl, timeout_ns, tile);
  if (__syncthreads_or(!landed)) {  // CTA-uniform
    if constexpr (!PERSIST) {
      if (tid == 0) {
        mbar_inval(&s_bar[0]);
        if constexpr (VB > 0) mbar_inval(&s_bar[1]);
      }
    }
    return false;
  }
  if (t.xin) {  // the first pass that moves data: from here on the keys are transformed
    for (uint32_t i = tid; i < tile_len; i += THREADS) s_kin[i] = xf_fwd(s_kin[i], t.xf);
    __syncthreads();
  }
  stamp(t.trace, 1);

  // ---- rank within the unit: unit u owns tile slots [u*ITEMS*UNIT, (u+1)*ITEMS*UNIT),
  // item j of the unit's lane l is slot u*ITEMS*UNIT + j*UNIT + l.  (With
  // half-warp units and ITEMS odd, the two halves of a warp read 16 banks
  // apart.)
  const int unit = tid / UNIT;
  const uint32_t slot0 = uint32_t(unit * ITEMS * UNIT + (tid % UNIT));
  uint32_t dp[ITEMS];  // digit << 16 | rank in the unit
  K kreg[VB > 0 ? 1 : ITEMS];  // keys only: the keys stay in registers until staged
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const K k = s_kin[slot0 + j * UNIT];
    if constexpr (VB == 0) kreg[j] = k;
    dp[j] = digit_of(k, t.shift, t.mask);
  }
  if constexpr (UNIT == 32)
    warp_rank_packed<ITEMS>(dp, s_wh + warp * RADIX, s_mm + warp * RADIX, lane);
  else
    half_rank_packed<ITEMS>(dp, s_wh + unit * RADIX, lane);
  __syncthreads();
  stamp(t.trace, 2);

  // ---- per digit: tile count, publish it; then the exclusive prefix over
  // the ranking units, which starts at the digit's first slot in the tile
  uint32_t my_cnt = 0u;
  constexpr int CSHIFT = UNIT == 32 ? 0 : 16;  // where the unit counters keep the count
  if (tid < RADIX) {
    uint32_t run = 0u;
#pragma unroll
    for (int w = 0; w < UNITS; ++w) run += s_wh[w * RADIX + tid] >> CSHIFT;
    my_cnt = run;
    if (!t.silent) {
      if (dbg_ok(lb_index<RADIX>(t.tile0 + tile, tid), t.lb_words, kSiteTileStatus))
        st_relaxed(&t.status[lb_index<RADIX>(t.tile0 + tile, tid)],
                   (tile == 0u ? kFlagInc : kFlagAgg) | run);
      if (t.gagg != nullptr &&
          dbg_ok(lb_index<RADIX>(tile / kGroupTiles, tid), t.g_words, kSiteGroupAgg))
        atomicAdd(&t.gagg[lb_index<RADIX>(tile / kGroupTiles, tid)], run | kGroupOne);
    }
  }
  const uint32_t my_start = block_exclusive_scan<THREADS>(my_cnt, s_tot);
  if (tid < RADIX) {
    s_cnt[tid] = my_cnt;
    s_tstart[tid] = my_start;
    uint32_t run = my_start;
#pragma unroll
    for (int w = 0; w < UNITS; ++w) {
      const uint32_t c = s_wh[w * RADIX + tid] >> CSHIFT;
      s_wh[w * RADIX + tid] = run;
      run += c;
    }
  }
  __syncthreads();
  stamp(t.trace, 3);

  // ---- keys into the stage in (digit, input) order (the peer masks are done)
  K* s_out = reinterpret_cast<K*>(smem + S::OUT);
  uint32_t pos[VB > 0 ? ITEMS : 1];  // stage slots, for the values
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const uint32_t p = (dp[j] & 0xffffu) + s_wh[unit * RADIX + (dp[j] >> 16)];
    if constexpr (VB == 0)
      s_out[p] = kreg[j];
    else
      s_out[p] = s_kin[slot0 + j * UNIT];
    if constexpr (VB > 0) pos[j] = p;
  }
  stamp(t.trace, 8);

  // ---- the values into the key buffer, while the look-back and the key
  // scatter run
  V* s_vin = nullptr;
  if constexpr (VB > 0) {
    __syncthreads();  // every key has left the buffer
    const V* gv = t.vsrc + tile_base;
    const Stage<V> sv(gv, tile_len);
    s_vin = sv.at(smem + S::KIN);
    if (tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive_expect_tx(&s_bar[1], sv.body);
      sv.issue(smem + S::KIN, gv, &s_bar[1]);
    }
    sv.edges(smem + S::KIN, gv, tile_len);
  }

  // ---- decoupled look-back: the sum of the counts of the preceding tiles for
  // my digit.  With groups: the earlier tiles of my group, then earlier
  // groups nearest first, each giving either its inclusive prefix (stop) or
  // its complete count (go on).  The walk then no longer grows with the
  // number of tiles in flight.
  if (tid < RADIX) {
    uint32_t excl = 0u;
    bool gave_up = false;
    if (tile > 0u) {
      bool done = false;
      if (t.gagg == nullptr) {
        walk_tiles<RADIX, 2>(t.status, tid, int32_t(t.tile0 + tile) - 1, int32_t(t.tile0), excl,
                             done, gave_up, ctrl, timeout_ns, tile, t.trace);
        if (!done && !gave_up) {  // tile 0 is inclusive: only if words were not cleared
          report_error(ctrl, kDevIndex, tile);
          gave_up = true;
        }
      } else {
        const int32_t g = int32_t(tile / kGroupTiles);
        walk_tiles<RADIX, 1>(t.status, tid, int32_t(tile) - 1, g * kGroupTiles, excl, done,
                             gave_up, ctrl, timeout_ns, tile, t.trace);
        stamp(t.trace, 14);
        // earlier groups, 8 per round trip (two 16-byte loads per array)
        for (int32_t h = g - 1; !done && !gave_up && h >= 0;) {
          trace_add(t.trace, 11, 1);
          const int32_t b0 = h >> 2;
          uint4 vi[2], va[2];
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const bool in = b0 - k >= 0;
            const size_t off = (size_t(b0 - k) * RADIX + tid) * 4;
            vi[k] = in ? __ldcg(reinterpret_cast<const uint4*>(t.ginc + off)) : make_uint4(0, 0, 0, 0);
            va[k] = in ? __ldcg(reinterpret_cast<const uint4*>(t.gagg + off)) : make_uint4(0, 0, 0, 0);
          }
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int32_t hh = 4 * b0 + 3 - q;  // groups of this window, nearest first
            if (hh > h || hh < 0 || done || gave_up) continue;
            const int c = 3 - (q & 3);
            const uint4& vq = vi[q >> 2];
            const uint4& aq = va[q >> 2];
            const uint32_t wi = c == 0 ? vq.x : c == 1 ? vq.y : c == 2 ? vq.z : vq.w;
            uint32_t ag = c == 0 ? aq.x : c == 1 ? aq.y : c == 2 ? aq.z : aq.w;
            const uint32_t fi = wi & kFlagMask;
            if (fi == kFlagErr) {
              gave_up = true;
            } else if (fi == kFlagInc) {
              excl += wi & kValueMask;
              done = true;
            } else {
              const uint32_t need = min(uint32_t(kGroupTiles), t.tiles - uint32_t(hh) * kGroupTiles);
              if ((ag >> 24) < need) {
                trace_add(t.trace, 13, 1);
                bool ok = false;
                ag = wait_group(&t.gagg[lb_index<RADIX>(uint32_t(hh), tid)], need, ctrl,
                                timeout_ns, tile, &ok);
                if (!ok) gave_up = true;
              }
              if (!gave_up) excl += ag & kGroupCountMask;
            }
          }
          h = 4 * b0 - 5;  // below the lowest group of this window (4*b0 - 4)
        }
        // a walk that ran past group 0 without an inclusive prefix has summed
        // every earlier group completely
      }
      if (!t.silent && dbg_ok(lb_index<RADIX>(t.tile0 + tile, tid), t.lb_words, kSiteTileStatus))
        st_relaxed(&t.status[lb_index<RADIX>(t.tile0 + tile, tid)],
                   gave_up ? kFlagErr : (kFlagInc | ((excl + my_cnt) & kValueMask)));
    }
    if (t.ginc != nullptr && !t.silent &&
        ((tile + 1) % kGroupTiles == 0 || tile + 1 == t.tiles) &&
        dbg_ok(lb_index<RADIX>(tile / kGroupTiles, tid), t.g_words, kSiteGroupInc))
      st_relaxed(&t.ginc[lb_index<RADIX>(tile / kGroupTiles, tid)],
                 gave_up ? kFlagErr : (kFlagInc | ((excl + my_cnt) & kValueMask)));
    // every key of digit tid goes to [pass offset + excl, ... + its count):
    // checked here once, so that the scatters below need no per-element
    // bound.  The past-the-end sentinels of a partial tile were counted under
    // the largest digit; they are never written.
    const uint32_t base = t.pass_offsets[tid] + excl;
    const uint32_t real = my_cnt - (uint32_t(tid) == t.mask ? uint32_t(TILE) - tile_len : 0u);
    if (!gave_up && (base > n || real > n - base)) {
      report_error(ctrl, kDevIndex, tile);
      gave_up = true;
    }
    if (gave_up) s_misc[1] = 1u;
    stamp(t.trace, 9);
    s_gbase[tid] = base - my_start;
  }
  __syncthreads();
  if (s_misc[1]) {
    // the output of this call is void (ctrl->error says why); let the value
    // copy land before leaving
    if constexpr (VB > 0) {
      bool ok = mbar_wait_bounded(&s_bar[1], parity, ctrl, timeout_ns, tile);
      if (!ok) mbar_wait_bounded(&s_bar[1], parity, ctrl, timeout_ns, tile);
      __syncthreads();
    }
    if constexpr (!PERSIST) {
      if (tid == 0) {
        mbar_inval(&s_bar[0]);
        if constexpr (VB > 0) mbar_inval(&s_bar[1]);
      }
    }
    return false;
  }
  stamp(t.trace, 4);
  // keys only: the key buffer is free (keys are staged in OUT) -- start the next tile
  if constexpr (PERSIST && VB == 0 && !INPLACE) {
    if (tid == 0) {
      const uint32_t nxt = atomicAdd(pf->counter, 1u);
      s_misc[3] = nxt;
      s_misc[4] = nxt < pf->tiles ? 1u : 0u;
    }
    __syncthreads();
    if (s_misc[4])
      stage_keys<K, THREADS, TILE, CG>(smem + S::KIN, t.ksrc, n, s_misc[3], &s_bar[0],
                                       smem + S::WH, S::ZERO_BYTES);
  }

  // ---- scatter: consecutive threads take consecutive stage slots, which map
  // to consecutive output addresses inside each digit run
  const bool full = tile_len == uint32_t(TILE);
  uint32_t gidx[VB > 0 ? ITEMS : 1];  // the values' destinations
  // XO: the last pass that moves data writes the keys back untransformed
  // debug builds, test-only: every destination of this tile past the array,
  // so that the bounds checks must drop the stores (0 otherwise)
  const uint32_t dbg_push = (kDebugChecks && t.dbg_bad) ? n : 0u;
  auto scatter_keys = [&](auto XO) {
    auto out = [&](K k) {
      if constexpr (decltype(XO)::value) return xf_inv(k, t.xf);
      else return k;
    };
    if (full) {
#pragma unroll
      for (int s = 0; s < ITEMS; ++s) {
        const uint32_t i = uint32_t(s * THREADS + tid);
        const K k = s_out[i];
        const uint32_t g = s_gbase[digit_of(k, t.shift, t.mask)] + i + dbg_push;
        if (dbg_ok(g, n, kSiteKeyScatter)) t.kdst[g] = out(k);
        if constexpr (VB > 0) gidx[s] = g;
      }
    } else {
#pragma unroll
      for (int s = 0; s < ITEMS; ++s) {
        const uint32_t i = uint32_t(s * THREADS + tid);
        if constexpr (VB > 0) gidx[s] = 0u;
        if (i < tile_len) {
          const K k = s_out[i];
          const uint32_t g = s_gbase[digit_of(k, t.shift, t.mask)] + i + dbg_push;
          if (dbg_ok(g, n, kSiteKeyScatter)) t.kdst[g] = out(k);
          if constexpr (VB > 0) gidx[s] = g;
        }
      }
    }
  };
  if (t.xout)
    scatter_keys(std::true_type{});
  else
    scatter_keys(std::false_type{});
  // in place: the key buffer is free once every staged key has left -- start the next tile
  if constexpr (PERSIST && INPLACE) {
    __syncthreads();
    if (tid == 0) {
      const uint32_t nxt = atomicAdd(pf->counter, 1u);
      s_misc[3] = nxt;
      s_misc[4] = nxt < pf->tiles ? 1u : 0u;
    }
    __syncthreads();
    if (s_misc[4])
      stage_keys<K, THREADS, TILE, CG>(smem + S::KIN, t.ksrc, n, s_misc[3], &s_bar[0],
                                       smem + S::WH, S::ZERO_BYTES);
  }
  stamp(t.trace, 5);
  bool ok = true;
  if constexpr (VB > 0) {
    ok = mbar_wait_bounded(&s_bar[1], parity, ctrl, timeout_ns, tile);
    if (!ok) ok = mbar_wait_bounded(&s_bar[1], parity, ctrl, timeout_ns, tile);
    // every key has left the stage and the value edges are in place
    if (!__syncthreads_or(!ok)) {
      V* s_vout = reinterpret_cast<V*>(smem + S::OUT);
#pragma unroll
      for (int j = 0; j < ITEMS; ++j) s_vout[pos[j]] = s_vin[slot0 + j * UNIT];
      if constexpr (PERSIST) {
        // the key buffer is free (values are staged in OUT): start the next tile
        if (tid == 0) {
          const uint32_t nxt = atomicAdd(pf->counter, 1u);
          s_misc[3] = nxt;
          s_misc[4] = nxt < pf->tiles ? 1u : 0u;
        }
      }
      __syncthreads();
      if constexpr (PERSIST) {
        if (s_misc[4])
          stage_keys<K, THREADS, TILE, CG>(smem + S::KIN, t.ksrc, n, s_misc[3], &s_bar[0],
                                           smem + S::WH, S::ZERO_BYTES);
      }
      if (full) {
#pragma unroll
        for (int s = 0; s < ITEMS; ++s)
          if (dbg_ok(gidx[s], n, kSiteValScatter)) t.vdst[gidx[s]] = s_vout[s * THREADS + tid];
      } else {
#pragma unroll
        for (int s = 0; s < ITEMS; ++s) {
          const uint32_t i = uint32_t(s * THREADS + tid);
          if (i < tile_len && dbg_ok(gidx[s], n, kSiteValScatter)) t.vdst[gidx[s]] = s_vout[i];
        }
      }
    } else {
      ok = false;
    }
  }
  if constexpr (!PERSIST) {
    if (tid == 0) {
      mbar_inval(&s_bar[0]);
      if constexpr (VB > 0) mbar_inval(&s_bar[1]);
    }
  }
  stamp(t.trace, 6);
  return ok;
}

// One digit pass, one tile per CTA.  The grid has one CTA per tile; tile ids
// come from an atomic counter so that a tile's predecessors have always
// started before it (forward progress of the look-back).
template <class K, int VB, int RADIX_BITS, int THREADS, int ITEMS, int MINB, int UNIT = 32,
          bool INPLACE = false>
__global__ void __launch_bounds__(THREADS, MINB)
    k_onesweep(K* __restrict__ k0, K* __restrict__ k1, ValT<VB>* __restrict__ v0,
               ValT<VB>* __restrict__ v1, uint32_t n, int pass, uint32_t shift, uint32_t mask,
               const uint32_t* __restrict__ pass_offsets, uint32_t* __restrict__ status,
               uint32_t* __restrict__ gagg, uint32_t* __restrict__ ginc, uint32_t tiles,
               Ctrl* __restrict__ ctrl, Knobs knobs, KeyXf<K> xf, bool early_dependents) {
  using S = OnesweepSmem<K, VB, RADIX_BITS, THREADS, ITEMS, UNIT, INPLACE>;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* s_misc = reinterpret_cast<uint32_t*>(smem + S::MISC);
  pdl_wait();  // the kernel before (upsweep or previous pass) is complete
  // a grid of more tiles than CTA slots lets the next pass be scheduled
  // during its last wave; a one-wave grid lets it in as its CTAs exit, so
  // that the next pass's CTAs spread over the SMs
  if (early_dependents) pdl_launch_dependents();

  const uint32_t exec = ctrl->exec_mask;
  if (!((exec >> pass) & 1u)) return;  // every key has the same digit: nothing moves
  const bool from_alt = (__popc(exec & ((1u << pass) - 1u)) & 1) != 0;
  if (threadIdx.x == 0) {
    s_misc[0] = atomicAdd(&ctrl->tile_counter[pass], 1u);
    s_misc[2] = ld_relaxed(&ctrl->error);  // an earlier pass of this call gave up
    if (s_misc[0] == 0u) ctrl->t_pass[pass][0] = stat_now(ctrl);
  }
  __syncthreads();
  if (s_misc[2] != 0u) return;  // CTA-uniform
  TileArgs<K, VB> t;
  t.ksrc = from_alt ? k1 : k0;
  t.kdst = from_alt ? k0 : k1;
  t.vsrc = from_alt ? v1 : v0;
  t.vdst = from_alt ? v0 : v1;
  t.n = n;
  t.tile = s_misc[0];
  t.shift = shift;
  t.mask = mask;
  t.pass_offsets = pass_offsets;
  t.status = status;
  t.tile0 = 0u;
  t.gagg = gagg;
  t.ginc = ginc;
  t.tiles = tiles;
  t.lb_words = uint64_t((tiles + 3u) / 4u * 4u) * S::RADIX;
  t.g_words = uint64_t((tiles + kGroupTiles - 1) / kGroupTiles + 3u) / 4u * 4u * S::RADIX;
  t.silent = (int(t.tile) == knobs.drop_tile) && (pass == knobs.drop_pass);
  t.dbg_bad = kDebugChecks && int(t.tile) == knobs.dbg_bad_tile && pass == 0;
  t.lb_small = knobs.lb_small != 0;
  t.trace = (knobs.trace != nullptr && pass == knobs.trace_pass && t.tile < knobs.trace_tiles)
                ? knobs.trace + size_t(t.tile) * 16
                : nullptr;
  t.xf = xf;
  t.xin = xf.on && pass == __ffs(int(exec)) - 1;  // first and last pass that move data
  t.xout = xf.on && pass == 31 - __clz(exec);
  onesweep_tile<K, VB, RADIX_BITS, THREADS, ITEMS, false, false, UNIT, INPLACE>(
      t, ctrl, knobs.timeout_ns, smem);
  __syncthreads();
  if (threadIdx.x == 0) atomicMax(&ctrl->t_pass[pass][1], stat_now(ctrl));
}

// One digit pass with resident CTAs (a grid of SMs x resident CTAs): each CTA
// takes tiles from the pass's atomic counter one after another and starts
// loading its next tile while it finishes the current one.  Tile ids are
// still taken in order by running CTAs, so the look-back keeps making
// progress: the lowest unfinished tile is always being worked on.
template <class K, int VB, int RADIX_BITS, int THREADS, int ITEMS, int MINB, int UNIT = 32,
          bool INPLACE = false>
__global__ void __launch_bounds__(THREADS, MINB)
    k_onesweep_persist(K* __restrict__ k0, K* __restrict__ k1, ValT<VB>* __restrict__ v0,
                       ValT<VB>* __restrict__ v1, uint32_t n, int pass, uint32_t shift,
                       uint32_t mask, const uint32_t* __restrict__ pass_offsets,
                       uint32_t* __restrict__ status, uint32_t* __restrict__ gagg,
                       uint32_t* __restrict__ ginc, uint32_t tiles, Ctrl* __restrict__ ctrl,
                       Knobs knobs, KeyXf<K> xf, bool early_dependents) {
  using S = OnesweepSmem<K, VB, RADIX_BITS, THREADS, ITEMS, UNIT, INPLACE>;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* s_misc = reinterpret_cast<uint32_t*>(smem + S::MISC);
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + S::MBAR);
  pdl_wait();  // the kernel before (upsweep or previous pass) is complete
  if (early_dependents) pdl_launch_dependents();

  const uint32_t exec = ctrl->exec_mask;
  if (!((exec >> pass) & 1u)) return;  // every key has the same digit: nothing moves
  const bool from_alt = (__popc(exec & ((1u << pass) - 1u)) & 1) != 0;
  Prefetch pf{&ctrl->tile_counter[pass], tiles};
  if (threadIdx.x == 0) {
    mbar_init(&s_bar[0]);
    if constexpr (VB > 0) mbar_init(&s_bar[1]);
    s_misc[3] = atomicAdd(pf.counter, 1u);
    s_misc[2] = ld_relaxed(&ctrl->error);  // an earlier pass of this call gave up
    if (s_misc[3] == 0u) ctrl->t_pass[pass][0] = stat_now(ctrl);
  }
  __syncthreads();
  TileArgs<K, VB> t;
  t.ksrc = from_alt ? k1 : k0;
  t.kdst = from_alt ? k0 : k1;
  t.vsrc = from_alt ? v1 : v0;
  t.vdst = from_alt ? v0 : v1;
  t.n = n;
  t.shift = shift;
  t.mask = mask;
  t.pass_offsets = pass_offsets;
  t.status = status;
  t.tile0 = 0u;
  t.gagg = gagg;
  t.ginc = ginc;
  t.tiles = tiles;
  t.lb_words = uint64_t((tiles + 3u) / 4u * 4u) * S::RADIX;
  t.g_words = uint64_t((tiles + kGroupTiles - 1) / kGroupTiles + 3u) / 4u * 4u * S::RADIX;
  t.lb_small = knobs.lb_small != 0;
  t.xf = xf;
  t.xin = xf.on && pass == __ffs(int(exec)) - 1;  // first and last pass that move data
  t.xout = xf.on && pass == 31 - __clz(exec);
  uint32_t tile = s_misc[3];
  if (tile < tiles && s_misc[2] == 0u)
    stage_keys<K, THREADS, S::TILE, false>(smem + S::KIN, t.ksrc, n, tile, &s_bar[0],
                                           smem + S::WH, S::ZERO_BYTES);
  else
    tile = tiles;  // nothing to do
  if (threadIdx.x == 0) s_misc[4] = 0u;
  __syncthreads();
  for (uint32_t it = 0; tile < tiles; ++it) {
    t.tile = tile;
    t.silent = (int(tile) == knobs.drop_tile) && (pass == knobs.drop_pass);
    t.dbg_bad = kDebugChecks && int(tile) == knobs.dbg_bad_tile && pass == 0;
    t.trace = (knobs.trace != nullptr && pass == knobs.trace_pass && tile < knobs.trace_tiles)
                  ? knobs.trace + size_t(tile) * 16
                  : nullptr;
    const bool ok = onesweep_tile<K, VB, RADIX_BITS, THREADS, ITEMS, false, true, UNIT, INPLACE>(
        t, ctrl, knobs.timeout_ns, smem, it & 1u, &pf);
    __syncthreads();
    const bool next = s_misc[4] != 0u;
    const uint32_t next_tile = s_misc[3];
    __syncthreads();  // every thread has read the next tile before it is cleared
    if (threadIdx.x == 0) s_misc[4] = 0u;
    if (!ok) {
      // a bounded wait gave up: let the next tile's key copy land, then stop
      if (next) {
        bool done = mbar_wait_bounded(&s_bar[0], (it + 1u) & 1u, ctrl, knobs.timeout_ns, tile);
        if (!done) mbar_wait_bounded(&s_bar[0], (it + 1u) & 1u, ctrl, knobs.timeout_ns, tile);
        __syncthreads();
      }
      break;
    }
    tile = next ? next_tile : tiles;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_inval(&s_bar[0]);
    if constexpr (VB > 0) mbar_inval(&s_bar[1]);
    atomicMax(&ctrl->t_pass[pass][1], stat_now(ctrl));
  }
}

// ------------------------------------------------------------ small sort

template <class K, int VB, int RADIX_BITS, int THREADS, int ITEMS>
struct SmallSmem {
  static constexpr int RADIX = 1 << RADIX_BITS;
  static constexpr int WARPS = THREADS / 32;
  static constexpr int TILE = THREADS * ITEMS;
  static constexpr int ELEM = (int(sizeof(K)) > VB) ? int(sizeof(K)) : VB;
  static constexpr int WH = 0;                      // u32 [WARPS][RADIX]
  static constexpr int MM = WH + WARPS * RADIX * 4;  // u32 [WARPS][RADIX] peer masks
  static constexpr int TOT = MM + WARPS * RADIX * 4; // u32 [32]
  static constexpr int STAGE = (TOT + 32 * 4 + 15) / 16 * 16;
  static constexpr int BYTES = STAGE + TILE * ELEM;
};

// All digit passes of one array of len <= TILE elements inside one CTA.  The
// input and output may be the same buffers: everything is read before the
// first write.
template <class K, int VB, int RADIX_BITS, int THREADS, int ITEMS>
__device__ __forceinline__ void cta_sort(const K* kin, const ValT<VB>* vin, K* kout,
                                         ValT<VB>* vout, uint32_t len, int begin_bit,
                                         int end_bit, unsigned char* smem, const KeyXf<K>& xf) {
  using V = ValT<VB>;
  using S = SmallSmem<K, VB, RADIX_BITS, THREADS, ITEMS>;
  constexpr int RADIX = S::RADIX, WARPS = S::WARPS;
  uint32_t* s_wh = reinterpret_cast<uint32_t*>(smem + S::WH);
  uint32_t* s_tot = reinterpret_cast<uint32_t*>(smem + S::TOT);
  K* s_k = reinterpret_cast<K*>(smem + S::STAGE);
  V* s_v = reinterpret_cast<V*>(smem + S::STAGE);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t slot0 = uint32_t(warp * ITEMS * 32 + lane);
  K key[ITEMS];
  V val[ITEMS];
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const uint32_t i = slot0 + j * 32;
    // past the end: largest digit in every pass
    key[j] = i < len ? (xf.on ? xf_fwd(kin[i], xf) : kin[i]) : ~K(0);
    if constexpr (VB > 0) val[j] = i < len ? vin[i] : V(0);
  }
  for (int lo = begin_bit; lo < end_bit; lo += RADIX_BITS) {
    const uint32_t shift = uint32_t(lo);
    const uint32_t mask = (1u << (min(lo + RADIX_BITS, end_bit) - lo)) - 1u;
    for (int i = tid; i < 2 * WARPS * RADIX; i += THREADS) s_wh[i] = 0u;  // counters + masks
    __syncthreads();
    uint32_t pos[ITEMS], dg[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) dg[j] = digit_of(key[j], shift, mask);
    warp_rank<ITEMS>(dg, pos, s_wh + warp * RADIX,
                     reinterpret_cast<uint32_t*>(smem + S::MM) + warp * RADIX, lane);
    __syncthreads();
    uint32_t cnt = 0u;
    if (tid < RADIX) {
#pragma unroll
      for (int w = 0; w < WARPS; ++w) {
        const uint32_t c = s_wh[w * RADIX + tid];
        s_wh[w * RADIX + tid] = cnt;
        cnt += c;
      }
    }
    const uint32_t start = block_exclusive_scan<THREADS>(cnt, s_tot);
    if (tid < RADIX) {
#pragma unroll
      for (int w = 0; w < WARPS; ++w) s_wh[w * RADIX + tid] += start;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      pos[j] += s_wh[warp * RADIX + digit_of(key[j], shift, mask)];
      s_k[pos[j]] = key[j];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) key[j] = s_k[slot0 + j * 32];
    if constexpr (VB > 0) {
      __syncthreads();
#pragma unroll
      for (int j = 0; j < ITEMS; ++j) s_v[pos[j]] = val[j];
      __syncthreads();
#pragma unroll
      for (int j = 0; j < ITEMS; ++j) val[j] = s_v[slot0 + j * 32];
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const uint32_t i = slot0 + j * 32;
    if (i < len && dbg_ok(i, len, kSiteSmallOut)) {
      kout[i] = xf.on ? xf_inv(key[j], xf) : key[j];
      if constexpr (VB > 0) vout[i] = val[j];
    }
  }
}

// ctrl (may be null): the caller's workspace, whose status words this call
// resets so that a later status read reports this call.
template <class K, int VB, int RADIX_BITS, int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS, 1)
    k_small_sort(K* keys, ValT<VB>* vals, uint32_t n, int begin_bit, int end_bit, Ctrl* ctrl,
                 KeyXf<K> xf) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int passes = (end_bit - begin_bit + RADIX_BITS - 1) / RADIX_BITS;
  if (ctrl != nullptr && threadIdx.x == 0) {
    ctrl->error = 0u;
    ctrl->error_info = 0u;
    ctrl->exec_mask = (1u << passes) - 1u;  // every pass runs (in shared memory)
    stat_clear_times(ctrl);
    stat_begin(ctrl, n, uint32_t(sizeof(K)) | uint32_t(VB) << 8 | uint32_t(passes) << 16 |
                            3u << 24);
  }
  cta_sort<K, VB, RADIX_BITS, THREADS, ITEMS>(keys, vals, keys, vals, n, begin_bit, end_bit,
                                              smem, xf);
  __syncthreads();
  if (ctrl != nullptr && threadIdx.x == 0) ctrl->t_upsweep = stat_now(ctrl);
}

}  // namespace rs
