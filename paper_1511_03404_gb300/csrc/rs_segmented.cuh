// Batched segmented sort: the counting-sort passes of Sec. 2.6 applied
// independently to every segment [off[s], off[s+1]) of one array, for all
// segments in one persistent launch.
//
//   k_seg_plan        one CTA: classifies segments (short ones fit one CTA,
//                     long ones are tiled), numbers the work items and maps
//                     every histogram chunk to its segment.
//   k_seg_small       short segments, each sorted whole in one CTA's shared
//                     memory (every pass), grid-stride over the short list;
//   k_seg_hist        the digit histograms of the long segments, chunk by
//                     chunk; each segment's last chunk scans them and writes
//                     the descriptors of the segment's pass tiles;
//   k_seg_persistent  SMs x resident CTAs, each looping over one global work
//                     queue (an atomic counter) in this order:
//                       [pass 0 tiles of long segments] ... [pass P-1 tiles]
//                     (kept apart from the short segments so that it needs
//                     few registers and four CTAs fit on an SM)
//                     A tile reads its descriptor (written by the histogram
//                     kernel, launched before); a tile of pass p > 0 waits
//                     (bounded) until every tile of pass p-1 of its segment is
//                     written.  Every wait is on items taken from the queue
//                     earlier, which are held by running CTAs, so the queue
//                     always makes progress.
#pragma once

#include "rs_kernels.cuh"

namespace rs {

constexpr uint32_t kDevInvalid = 1;  // RS_ERR_INVALID seen on the device

struct SegDesc {
  uint64_t off;    // first element
  uint32_t len;    // elements
  uint32_t tile0;  // first global pass tile
  uint32_t chunk0; // first global histogram chunk
  uint32_t seg;    // segment id
  uint32_t pad[2];
};
static_assert(sizeof(SegDesc) == 32, "SegDesc is 32 bytes");

// Everything a pass tile needs to start, in one 32-byte read: written for
// every tile of a long segment by the segment's last histogram chunk, so the
// tile needs no dependent read of a tile map, a segment descriptor and the
// segment's state before it can load its keys.
struct TileDesc {
  uint64_t off;    // the segment's first element
  uint32_t len;    // the segment's elements
  uint32_t li;     // long-segment index (state, counts, offsets)
  uint32_t tile0;  // the segment's first global pass tile
  uint32_t exec;   // passes of the segment that move data (after the parity rule)
  uint32_t pad[2];
};
static_assert(sizeof(TileDesc) == 32, "TileDesc is 32 bytes");

// Per long segment: histogram ticket, ready word (bit 0: the histograms are
// scanned; bits 1..: the mask of passes that move data; kept for inspection,
// the pass kernel takes the mask from its tile descriptor), done counters.
constexpr int kSegStateWords = 16;
enum SegStateField { kSegTicket = 0, kSegReady = 1, kSegDone0 = 3 };

// Plan results in Ctrl::tile_counter[]
enum SegCtrlField {
  kQueue = 0,    // work-queue ticket
  kNSmall = 1,
  kNLarge = 2,
  kNTiles = 3,   // pass tiles of all long segments (one pass)
  kNChunks = 4,  // histogram chunks of all long segments
  kPlanned = 5   // 1 once the plan is complete
};

struct SegLayout {
  size_t small_ids, descs, tdesc, chunk_seg, state, counts, offsets, status, total;
  size_t memset_bytes;  // Ctrl + state + counts
  size_t tiles_max, chunks_max;
};

inline SegLayout seg_layout(size_t n, size_t nseg, int passes, int radix_bits, int tile,
                            int chunk) {
  SegLayout L{};
  const size_t radix = size_t(1) << radix_bits;
  L.tiles_max = align_up((n + tile - 1) / tile + nseg, 4);
  L.chunks_max = (n + chunk - 1) / chunk + nseg;
  L.state = 256;
  L.counts = align_up(L.state + nseg * kSegStateWords * 4, 256);
  L.memset_bytes = align_up(L.counts + nseg * passes * radix * 4, 256);
  L.offsets = L.memset_bytes;
  L.small_ids = align_up(L.offsets + nseg * passes * radix * 4, 256);
  L.descs = align_up(L.small_ids + nseg * 4, 256);
  L.tdesc = align_up(L.descs + nseg * sizeof(SegDesc), 256);
  L.chunk_seg = align_up(L.tdesc + L.tiles_max * sizeof(TileDesc), 256);
  L.status = align_up(L.chunk_seg + L.chunks_max * 4, 256);
  L.total = align_up(L.status + size_t(passes) * L.tiles_max * radix * 4, 256);
  return L;
}

// One CTA numbers the work.  Segments longer than small_max are "long".
template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1)
    k_seg_plan(const uint64_t* __restrict__ off, uint64_t nseg, uint64_t n, uint32_t small_max,
               uint32_t tile, uint32_t chunk, Ctrl* __restrict__ ctrl,
               uint32_t* __restrict__ small_ids, SegDesc* __restrict__ descs,
               uint32_t* __restrict__ chunk_seg,
               uint64_t tiles_max, uint64_t chunks_max) {
  __shared__ uint32_t s_tot[32];
  __shared__ uint32_t s_run[4];
  __shared__ int s_bad;
  const int tid = threadIdx.x;
  if (tid < 4) s_run[tid] = 0u;
  if (tid == 0) s_bad = 0;
  __syncthreads();
  if (off[0] != 0ull || off[nseg] != n) s_bad = 1;  // benign race: same value
  for (uint64_t base = 0; base < nseg; base += THREADS) {
    const uint64_t s = base + tid;
    uint64_t len = 0;
    bool valid = s < nseg;
    if (valid) {
      const uint64_t a = off[s], b = off[s + 1];
      if (b < a || b > n || b - a > uint64_t((1u << 30) - 1u)) {
        s_bad = 1;
        valid = false;
      } else {
        len = b - a;
      }
    }
    const bool is_long = valid && len > small_max;
    const uint32_t small = (valid && !is_long) ? 1u : 0u;
    const uint32_t lng = is_long ? 1u : 0u;
    const uint32_t nt = is_long ? uint32_t((len + tile - 1) / tile) : 0u;
    const uint32_t nc = is_long ? uint32_t((len + chunk - 1) / chunk) : 0u;
    const uint32_t e_small = block_exclusive_scan<THREADS>(small, s_tot);
    __syncthreads();
    const uint32_t e_long = block_exclusive_scan<THREADS>(lng, s_tot);
    __syncthreads();
    const uint32_t e_tile = block_exclusive_scan<THREADS>(nt, s_tot);
    __syncthreads();
    const uint32_t e_chunk = block_exclusive_scan<THREADS>(nc, s_tot);
    const uint32_t r_small = s_run[0], r_long = s_run[1], r_tile = s_run[2],
                   r_chunk = s_run[3];
    if (small && dbg_ok(r_small + e_small, nseg, kSiteSegPlan))
      small_ids[r_small + e_small] = uint32_t(s);
    const uint32_t li = r_long + e_long;
    bool map_ok = false;
    if (is_long) {
      SegDesc d;
      d.off = off[s];
      d.len = uint32_t(len);
      d.tile0 = r_tile + e_tile;
      d.chunk0 = r_chunk + e_chunk;
      d.seg = uint32_t(s);
      d.pad[0] = d.pad[1] = 0u;
      if (dbg_ok(li, nseg, kSiteSegPlan)) descs[li] = d;
      map_ok = uint64_t(d.tile0) + nt <= tiles_max && uint64_t(d.chunk0) + nc <= chunks_max;
      if (!map_ok) s_bad = 1;
    }
    // the chunk map of these long segments: each warp writes its lanes'
    // segments one after another, 32 consecutive entries per store (one
    // thread writing its own segment's entries issued one store each)
    {
      const int lane = tid & 31;
      const uint32_t c0 = r_chunk + e_chunk;
      for (uint32_t m = __ballot_sync(kFull, map_ok); m != 0u; m &= m - 1u) {
        const int src = __ffs(int(m)) - 1;
        const uint32_t sli = __shfl_sync(kFull, li, src), sc0 = __shfl_sync(kFull, c0, src);
        const uint32_t snc = __shfl_sync(kFull, nc, src);
        for (uint32_t i = uint32_t(lane); i < snc; i += 32)
          if (dbg_ok(uint64_t(sc0) + i, chunks_max, kSiteSegPlan)) chunk_seg[sc0 + i] = sli;
      }
    }
    __syncthreads();
    if (tid == THREADS - 1) {  // the last thread's inclusive sums are the block totals
      s_run[0] = r_small + e_small + small;
      s_run[1] = r_long + e_long + lng;
      s_run[2] = r_tile + e_tile + nt;
      s_run[3] = r_chunk + e_chunk + nc;
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (s_bad) {
      report_error(ctrl, kDevInvalid, 0u);
      ctrl->tile_counter[kNSmall] = ctrl->tile_counter[kNLarge] = 0u;
      ctrl->tile_counter[kNTiles] = ctrl->tile_counter[kNChunks] = 0u;
    } else {
      ctrl->tile_counter[kNSmall] = s_run[0];
      ctrl->tile_counter[kNLarge] = s_run[1];
      ctrl->tile_counter[kNTiles] = s_run[2];
      ctrl->tile_counter[kNChunks] = s_run[3];
    }
    ctrl->tile_counter[kPlanned] = 1u;
  }
}

// Shared memory of one short-segment sort: the warps' counters and peer
// masks, and the segment's keys and values, each in a buffer of its own.
template <class K, int VB, int RADIX_BITS, int THREADS, int ITEMS>
struct SegSmallSmem {
  static constexpr int RADIX = 1 << RADIX_BITS;
  static constexpr int WARPS = THREADS / 32;
  static constexpr int TILE = THREADS * ITEMS;
  static constexpr int WH = 0;                        // u32 [WARPS][RADIX] warp counters
  static constexpr int MM = WH + WARPS * RADIX * 4;   // u32 [WARPS][RADIX] peer masks
  static constexpr int TOT = MM + WARPS * RADIX * 4;  // u32 [32]
  static constexpr int KEYS = (TOT + 32 * 4 + 15) / 16 * 16;  // K [TILE]
  static constexpr int VALS = KEYS + TILE * int(sizeof(K));   // V [TILE]
  static constexpr int BYTES = VALS + (VB > 0 ? TILE * VB : 0);
};

// UNIT: lanes per ranking unit of the pass tiles (32 or 16, as for the
// onesweep pass); SMALL_ITEMS: keys per thread of the short-segment sort,
// whose tile bounds a short segment.
template <class K, int VB, int RADIX_BITS, int THREADS, int ITEMS, int CHUNK_TILES, int UNIT = 32,
          int SMALL_ITEMS = ITEMS>
struct SegKernelCfg {
  static constexpr int RADIX = 1 << RADIX_BITS;
  static constexpr int TILE = THREADS * ITEMS;
  static constexpr int SMALL_TILE = THREADS * SMALL_ITEMS;
  static constexpr int CHUNK = TILE * CHUNK_TILES;
  static constexpr int MAXP = (8 * int(sizeof(K)) + RADIX_BITS - 1) / RADIX_BITS;
  // histogram kernel: [pass][digit][16 lane slots] u32 counters, 1024 threads
  static constexpr int HIST_THREADS = 1024;
  static constexpr int HIST_SLOTS = 16;
  static constexpr int HIST_BYTES = MAXP * RADIX * HIST_SLOTS * 4;
  // two CTAs per SM while their counters fit (32-bit keys), else one
  static constexpr int HIST_MINB = HIST_BYTES <= 100 * 1024 ? 2 : 1;
  using OS = OnesweepSmem<K, VB, RADIX_BITS, THREADS, ITEMS, UNIT>;
  using SS = SegSmallSmem<K, VB, RADIX_BITS, THREADS, SMALL_ITEMS>;
  static constexpr int MISC = (OS::BYTES + 15) / 16 * 16;  // u32 [8]
  static constexpr int BYTES = MISC + 32;
};

struct SegArgs {
  const uint64_t* off;
  int begin_bit, end_bit, passes;
  Ctrl* ctrl;
  const uint32_t* small_ids;
  const SegDesc* descs;
  TileDesc* tdesc;    // [tiles_max]
  const uint32_t* chunk_seg;
  uint32_t* state;    // [nseg][kSegStateWords]
  uint32_t* counts;   // [nseg][passes][RADIX]
  uint32_t* offsets;  // [nseg][passes][RADIX]
  uint32_t* status;   // [passes][tiles_max][RADIX]
  uint64_t tiles_max;
  uint64_t nseg;      // segments (debug bounds checks)
  Knobs knobs;
};

// Every digit pass (Sec. 2.6) of one segment of len <= TILE elements inside
// one CTA.  The segment lives in shared memory from the first load to the
// last store; a pass reads each thread's items from it, ranks them, and
// writes them back at their stable positions (a barrier separates the reads
// from the writes), keys first, then values.  So no more than one item array
// and the positions are live in registers at a time, and four CTAs fit on an
// SM.  Past the end the keys are the largest key: they rank after every real
// key in every pass and are never written out.
template <class K, int VB, int RADIX_BITS, int THREADS, int ITEMS>
__device__ __forceinline__ void seg_cta_sort(const K* kin, const ValT<VB>* vin, K* kout,
                                             ValT<VB>* vout, uint32_t len, int begin_bit,
                                             int end_bit, unsigned char* smem) {
  using V = ValT<VB>;
  using S = SegSmallSmem<K, VB, RADIX_BITS, THREADS, ITEMS>;
  constexpr int RADIX = S::RADIX, WARPS = S::WARPS, TILE = S::TILE;
  uint32_t* s_wh = reinterpret_cast<uint32_t*>(smem + S::WH);
  uint32_t* s_mm = reinterpret_cast<uint32_t*>(smem + S::MM);
  uint32_t* s_tot = reinterpret_cast<uint32_t*>(smem + S::TOT);
  K* s_k = reinterpret_cast<K*>(smem + S::KEYS);
  V* s_v = reinterpret_cast<V*>(smem + S::VALS);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t slot0 = uint32_t(warp * ITEMS * 32 + lane);

  for (uint32_t i = tid; i < uint32_t(TILE); i += THREADS) {
    s_k[i] = i < len ? kin[i] : ~K(0);
    if constexpr (VB > 0) s_v[i] = i < len ? vin[i] : V(0);
  }
  for (int lo = begin_bit; lo < end_bit; lo += RADIX_BITS) {
    const uint32_t shift = uint32_t(lo);
    const uint32_t mask = (1u << (min(lo + RADIX_BITS, end_bit) - lo)) - 1u;
    for (int i = tid; i < 2 * WARPS * RADIX; i += THREADS) s_wh[i] = 0u;  // counters + masks
    __syncthreads();
    K key[ITEMS];
    uint32_t dp[ITEMS];  // digit << 16 | rank in the warp, then the item's position
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      key[j] = s_k[slot0 + j * 32];
      dp[j] = digit_of(key[j], shift, mask);
    }
    warp_rank_packed<ITEMS>(dp, s_wh + warp * RADIX, s_mm + warp * RADIX, lane);
    __syncthreads();
    // per digit: exclusive prefix over the warps, from the digit's start
    uint32_t cnt = 0u;
    if (tid < RADIX) {
#pragma unroll
      for (int w = 0; w < WARPS; ++w) cnt += s_wh[w * RADIX + tid];
    }
    const uint32_t start = block_exclusive_scan<THREADS>(cnt, s_tot);
    if (tid < RADIX) {
      uint32_t run = start;
#pragma unroll
      for (int w = 0; w < WARPS; ++w) {
        const uint32_t c = s_wh[w * RADIX + tid];
        s_wh[w * RADIX + tid] = run;
        run += c;
      }
    }
    __syncthreads();  // every key of the pass was read above
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      dp[j] = (dp[j] & 0xffffu) + s_wh[warp * RADIX + (dp[j] >> 16)];
      s_k[dp[j]] = key[j];
    }
    if constexpr (VB > 0) {
      V val[ITEMS];
#pragma unroll
      for (int j = 0; j < ITEMS; ++j) val[j] = s_v[slot0 + j * 32];
      __syncthreads();  // every value was read
#pragma unroll
      for (int j = 0; j < ITEMS; ++j) s_v[dp[j]] = val[j];
    }
    __syncthreads();
  }
  for (uint32_t i = tid; i < len; i += THREADS) {
    if (!dbg_ok(i, len, kSiteSegSmallOut)) continue;
    kout[i] = s_k[i];
    if constexpr (VB > 0) vout[i] = s_v[i];
  }
}

template <class K, int VB, int RADIX_BITS, int THREADS, int ITEMS, int MINB = 4>
__global__ void __launch_bounds__(THREADS, MINB)
    k_seg_small(K* __restrict__ k0, ValT<VB>* __restrict__ v0, K* __restrict__ k1,
                ValT<VB>* __restrict__ v1, SegArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int passes = a.passes;
  K* kout = (passes & 1) ? k1 : k0;  // where the pass count parity puts the result
  ValT<VB>* vout = (passes & 1) ? v1 : v0;
  const uint32_t n_small = a.ctrl->tile_counter[kNSmall];
  for (uint32_t i = blockIdx.x; i < n_small; i += gridDim.x) {
    const uint32_t s = a.small_ids[i];
    const uint64_t b = a.off[s];
    const uint32_t len = uint32_t(a.off[s + 1] - b);
    seg_cta_sort<K, VB, RADIX_BITS, THREADS, ITEMS>(k0 + b, v0 + b, kout + b, vout + b, len,
                                                    a.begin_bit, a.end_bit, smem);
    __syncthreads();
  }
}

// Digit histograms of the long segments, every pass (Sec. 2.6, the counting
// step), one chunk of CHUNK keys at a time, grid-stride over the chunks.  As in
// the whole-array upsweep: 16-byte loads, every pass's digit counted into
// per-lane-slot shared counters, then the chunk's counts added to its
// segment's.  The chunk also clears the look-back words of its tiles.  The
// last chunk of a segment (ticket) scans the segment's histograms, chooses the
// passes that move data and marks the segment ready for its pass tiles.
template <class K, int RADIX_BITS, int THREADS, int MAXP, int SLOTS, int CHUNK, int TILE,
          int CHUNK_TILES, int MINB = 2>
__global__ void __launch_bounds__(THREADS, MINB)
    k_seg_hist(const K* __restrict__ k0, SegArgs a) {
  constexpr int RADIX = 1 << RADIX_BITS;
  constexpr int VEC = 16 / int(sizeof(K));
  static_assert(RADIX <= THREADS, "one thread per digit in the scan");
  extern __shared__ uint32_t sh[];  // [passes][RADIX][SLOTS]
  __shared__ uint32_t s_tot[32];
  __shared__ int s_last;
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t slot = uint32_t(lane & (SLOTS - 1));
  const int passes = a.passes;
  uint32_t shiftp[MAXP], maskp[MAXP];
#pragma unroll
  for (int p = 0; p < MAXP; ++p) {
    const int lo = a.begin_bit + p * RADIX_BITS;
    const int hi = min(lo + RADIX_BITS, a.end_bit);
    shiftp[p] = p < passes ? uint32_t(lo) : 0u;
    maskp[p] = p < passes ? ((1u << (hi - lo)) - 1u) : 0u;
  }
  auto count_key = [&](K k) {
#pragma unroll
    for (int p = 0; p < MAXP; ++p)
      if (p < passes)
        atomicAdd(&sh[(p * RADIX + int(digit_of(k, shiftp[p], maskp[p]))) * SLOTS + int(slot)],
                  1u);
  };
  const uint32_t n_chunks = a.ctrl->tile_counter[kNChunks];
  const int words = passes * RADIX * SLOTS;
  for (uint32_t item = blockIdx.x; item < n_chunks; item += gridDim.x) {
    const uint32_t li = a.chunk_seg[item];
    const SegDesc d = a.descs[li];
    const uint32_t lc = item - d.chunk0;
    const uint32_t start = lc * uint32_t(CHUNK);
    const uint32_t len = min(uint32_t(CHUNK), d.len - start);
    const K* keys = k0 + d.off + start;
    for (int i = tid; i < words; i += THREADS) sh[i] = 0u;
    __syncthreads();
    // 16-byte aligned body, scalar head and tail
    const uintptr_t addr = reinterpret_cast<uintptr_t>(keys);
    uint32_t head = uint32_t(((16u - (addr & 15u)) & 15u) / sizeof(K));
    if (head > len) head = len;
    const uint32_t nvec = (len - head) / VEC;
    const uint32_t tail = head + nvec * VEC;
    if (uint32_t(tid) < head) count_key(keys[tid]);
    if (uint32_t(tid) < len - tail) count_key(keys[tail + tid]);
    const uint4* vp = reinterpret_cast<const uint4*>(keys + head);
    // two 16-byte loads in flight per thread before their keys are counted
    // (four need more than the 32 registers two CTAs of 1024 threads leave)
    constexpr int UNROLL = 2;
    for (uint32_t i0 = tid; i0 < nvec; i0 += THREADS * UNROLL) {
      uint4 buf[UNROLL];
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) {
        const uint32_t i = i0 + uint32_t(u) * THREADS;
        if (i < nvec) buf[u] = vp[i];
      }
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) {
        if (i0 + uint32_t(u) * THREADS < nvec) {
          const K* ks = reinterpret_cast<const K*>(&buf[u]);
#pragma unroll
          for (int e = 0; e < VEC; ++e) count_key(ks[e]);
        }
      }
    }
    __syncthreads();
    // the chunk's counts into the segment's: one (pass, digit) per thread
    uint32_t* cnt = a.counts + size_t(li) * passes * RADIX;
    for (int w = tid; w < passes * RADIX; w += THREADS) {
      const uint32_t* row = sh + w * SLOTS;
      uint32_t c = 0u;
#pragma unroll
      for (int l = 0; l < SLOTS; ++l) c += row[(l + lane) & (SLOTS - 1)];  // rotated: no conflicts
      if (c && dbg_ok(uint64_t(li) * passes * RADIX + w, a.nseg * passes * RADIX, kSiteSegCounts))
        atomicAdd(&cnt[w], c);
    }
    // clear the look-back words of this chunk's tiles [ta, tb), every pass.
    // In the [tile/4][digit][tile%4] layout one digit's words of four
    // consecutive tiles are 16 contiguous bytes: consecutive threads clear
    // consecutive 16-byte groups, a whole group when its four tiles are all
    // this chunk's, else word by word (the neighbouring segment owns the rest)
    const uint32_t t_first = lc * uint32_t(CHUNK_TILES);
    const uint32_t t_last = min(t_first + uint32_t(CHUNK_TILES), (d.len + TILE - 1) / TILE);
    const uint32_t ta = d.tile0 + t_first, tb = d.tile0 + t_last;
    const uint32_t g0 = ta / 4u, ng = (tb - 1u) / 4u - g0 + 1u;
    for (int p = 0; p < passes; ++p) {
      uint32_t* st = a.status + size_t(p) * a.tiles_max * RADIX;
      for (uint32_t i = tid; i < ng * RADIX; i += THREADS) {
        const uint32_t g = g0 + i / RADIX;
        const size_t q = size_t(g) * RADIX + i % RADIX;  // the 16-byte group
        if (!dbg_ok(q, a.tiles_max * RADIX / 4, kSiteSegClear)) continue;
        if (4u * g >= ta && 4u * g + 3u < tb) {
          reinterpret_cast<uint4*>(st)[q] = make_uint4(0u, 0u, 0u, 0u);
        } else {
#pragma unroll
          for (uint32_t c = 0; c < 4u; ++c)
            if (4u * g + c >= ta && 4u * g + c < tb) st[q * 4 + c] = 0u;
        }
      }
    }
    __syncthreads();
    uint32_t* state = a.state + size_t(li) * kSegStateWords;
    if (tid == 0) {
      // the CTA's counts and cleared words (ordered before by the barrier)
      // become visible before the ticket
      __threadfence();
      const uint32_t chunks = (d.len + CHUNK - 1) / CHUNK;
      s_last = dbg_ok(li, a.nseg, kSiteSegState) &&
               atomicAdd(&state[kSegTicket], 1u) == chunks - 1u;
    }
    __syncthreads();
    if (s_last) {
      // last chunk of the segment: scan each pass's histogram
      __threadfence();
      uint32_t* offs = a.offsets + size_t(li) * passes * RADIX;
      uint32_t exec = 0u;
      for (int p = 0; p < passes; ++p) {
        const uint32_t c = tid < RADIX ? ld_relaxed(&cnt[p * RADIX + tid]) : 0u;
        const uint32_t e = block_exclusive_scan<THREADS>(c, s_tot);
        if (tid < RADIX && dbg_ok(uint64_t(li) * passes * RADIX + p * RADIX + tid,
                                  a.nseg * passes * RADIX, kSiteSegCounts))
          offs[p * RADIX + tid] = e;
        if (!__syncthreads_or(tid < RADIX && c == d.len)) exec |= 1u << p;
      }
      if ((__popc(exec) & 1) != (passes & 1)) {  // every thread: the same exec
        const uint32_t skipped = ~exec & ((1u << passes) - 1u);
        exec |= skipped & (0u - skipped);
      }
      // every pass tile of the segment learns where it is and which passes
      // move data from one descriptor (read by the pass kernel, launched after)
      const uint32_t ntiles = (d.len + TILE - 1) / TILE;
      for (uint32_t t = tid; t < ntiles; t += THREADS) {
        if (!dbg_ok(uint64_t(d.tile0) + t, a.tiles_max, kSiteSegState)) continue;
        TileDesc td;
        td.off = d.off;
        td.len = d.len;
        td.li = li;
        td.tile0 = d.tile0;
        td.exec = exec;
        td.pad[0] = td.pad[1] = 0u;
        a.tdesc[d.tile0 + t] = td;
      }
      if (tid == 0) {
        __threadfence();
        st_release(&state[kSegReady], 1u | (exec << 1));
      }
    }
    __syncthreads();
  }
}

template <class K, int VB, int RADIX_BITS, int THREADS, int ITEMS, int CHUNK_TILES, int UNIT = 32,
          int MINB = 4>
__global__ void __launch_bounds__(THREADS, MINB)
    k_seg_persistent(K* __restrict__ k0, ValT<VB>* __restrict__ v0, K* __restrict__ k1,
                     ValT<VB>* __restrict__ v1, SegArgs a) {
  using V = ValT<VB>;
  using C = SegKernelCfg<K, VB, RADIX_BITS, THREADS, ITEMS, CHUNK_TILES, UNIT>;
  constexpr int RADIX = C::RADIX, TILE = C::TILE;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* s_misc = reinterpret_cast<uint32_t*>(smem + C::MISC);
  const int tid = threadIdx.x;
  Ctrl* ctrl = a.ctrl;
  const int passes = a.passes;

  const uint32_t n_tiles = ctrl->tile_counter[kNTiles];
  const uint32_t q_end = uint32_t(passes) * n_tiles;

  for (;;) {
    if (tid == 0) {
      s_misc[0] = atomicAdd(&ctrl->tile_counter[kQueue], 1u);
      s_misc[1] = ld_relaxed(&ctrl->error);
    }
    __syncthreads();
    const uint32_t item = s_misc[0];
    if (item >= q_end || s_misc[1] != 0u) break;  // CTA-uniform

    // ---- one tile of one pass of a long segment.  The histogram kernel
    // (launched before this one) has written the tile's descriptor and every
    // segment's scans; a tile of pass p > 0 waits (bounded) until every tile of
    // pass p - 1 of its segment is written, whether that pass moved data or not
    const int p = int(item / n_tiles);
    const uint32_t gt = item - uint32_t(p) * n_tiles;
    const TileDesc d = a.tdesc[gt];
    const uint32_t li = d.li;
    uint32_t* state = a.state + size_t(li) * kSegStateWords;
    const uint32_t ntiles = (d.len + TILE - 1) / TILE;
    const uint32_t exec = d.exec;
    bool ok = true;
    if (p > 0) {
      if (tid == 0) {
        bool w = ld_relaxed(&state[kSegDone0 + p - 1]) >= ntiles;
        if (w)
          __threadfence();  // acquire: the previous pass's output
        else
          w = wait_geq(&state[kSegDone0 + p - 1], ntiles, ctrl, a.knobs.timeout_ns, gt);
        s_misc[3] = w ? 1u : 0u;
      }
      __syncthreads();
      ok = s_misc[3] != 0u;
    }
    if (ok && ((exec >> p) & 1u)) {
      const bool from_alt = (__popc(exec & ((1u << p) - 1u)) & 1) != 0;
      TileArgs<K, VB> t;
      t.ksrc = (from_alt ? k1 : k0) + d.off;
      t.kdst = (from_alt ? k0 : k1) + d.off;
      if constexpr (VB > 0) {
        t.vsrc = (from_alt ? v1 : v0) + d.off;
        t.vdst = (from_alt ? v0 : v1) + d.off;
      } else {
        t.vsrc = nullptr;
        t.vdst = nullptr;
      }
      t.n = d.len;
      t.tile = gt - d.tile0;
      const int lo = a.begin_bit + p * RADIX_BITS;
      t.shift = uint32_t(lo);
      t.mask = (1u << (min(lo + RADIX_BITS, a.end_bit) - lo)) - 1u;
      t.pass_offsets = a.offsets + (size_t(li) * passes + p) * RADIX;
      t.status = a.status + size_t(p) * a.tiles_max * RADIX;
      t.tile0 = d.tile0;
      t.gagg = nullptr;  // segments are short: flat walk
      t.ginc = nullptr;
      t.tiles = ntiles;
      t.lb_words = a.tiles_max * RADIX;
      t.g_words = 0;
      t.silent = false;
      t.dbg_bad = false;
      t.trace = nullptr;
      t.lb_small = false;
      t.xf = KeyXf<K>{};
      t.xin = false;
      t.xout = false;
      onesweep_tile<K, VB, RADIX_BITS, THREADS, ITEMS, true, false, UNIT>(
          t, ctrl, a.knobs.timeout_ns, smem);
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();  // the tile's output, ordered before by the barrier, then the count
      if (dbg_ok(li, a.nseg, kSiteSegState)) atomicAdd(&state[kSegDone0 + p], 1u);
    }
    __syncthreads();
  }
}

}  // namespace rs
