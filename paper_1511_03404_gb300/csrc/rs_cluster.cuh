// The whole sort inside one thread-block cluster, for arrays up to
// CL x SLICE elements (SLICE = THREADS x ITEMS per CTA): every digit pass
// (Sec. 2.6) runs on data held in the cluster's shared memory, with no trip
// through global memory and no kernel boundary between passes.
//
// CTA c of the cluster owns positions [c * SLICE, (c + 1) * SLICE) of the
// array.  One pass:
//   1. each thread takes its ITEMS keys (warp-striped) from the CTA's source
//      buffer and the warps rank them stably (shared peer masks, per-warp
//      running counts); per-digit prefixes over the warps give every key's
//      place among the CTA's keys of its digit, and the CTA's digit counts;
//   2. every CTA stores its digit counts into every CTA's count table
//      (remote shared-memory stores); after a cluster barrier each CTA reads
//      its own table: the start of digit d is the count of all smaller
//      digits, plus the count of digit d in lower-ranked CTAs;
//   3. the CTA first stages its keys (and values) in digit order in its own
//      source buffer (its keys are in registers by then), then its threads
//      take the staged keys in order and store each at its global position,
//      in the destination buffer of the CTA that owns that position (a
//      remote shared-memory store): consecutive threads store consecutive
//      keys of a digit run to consecutive addresses of one CTA, instead of
//      scattering single keys over the cluster;
//   4. cluster barrier; the destination buffer becomes the next source.
// Past the end of the array the slices hold the largest key, which sorts
// after every real key in every pass and is never written out.  The
// cluster barriers are hardware barriers that every CTA passes the same
// number of times; no CTA waits on a flag.
#pragma once

#include "rs_kernels.cuh"

namespace rs {

__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
               ::: "memory");
}

// The shared::cluster address of `p` (a shared-memory pointer of this CTA)
// in the CTA of cluster rank `rank`.
__device__ __forceinline__ uint32_t map_shared(const void* p, uint32_t rank) {
  const uint32_t local = static_cast<uint32_t>(__cvta_generic_to_shared(p));
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(rank));
  return remote;
}

__device__ __forceinline__ void st_cluster(uint32_t addr, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

__device__ __forceinline__ void st_cluster(uint32_t addr, uint64_t v) {
  asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}

template <class K, int VB, int RADIX_BITS, int THREADS, int ITEMS>
struct ClusterSmem {
  static constexpr int RADIX = 1 << RADIX_BITS;
  static constexpr int WARPS = THREADS / 32;
  static constexpr int SLICE = THREADS * ITEMS;
  static constexpr int KB = int(sizeof(K));
  static constexpr int WH = 0;                              // u32 [WARPS][RADIX] running counts
  static constexpr int MM = WH + WARPS * RADIX * 4;         // u32 [WARPS][RADIX] peer masks
  static constexpr int MAX_CL = 8;
  static constexpr int CNT = MM + WARPS * RADIX * 4;        // u32 [MAX_CL][RADIX] every CTA's counts
  static constexpr int BASE = CNT + MAX_CL * RADIX * 4;     // u32 [RADIX] global digit bases
  static constexpr int LST = BASE + RADIX * 4;              // u32 [RADIX] digit starts in the CTA
  static constexpr int TOT = LST + RADIX * 4;               // u32 [32]
  static constexpr int KEYS = (TOT + 32 * 4 + 15) / 16 * 16;  // K [2][SLICE]
  static constexpr int VALS = KEYS + 2 * SLICE * KB;        // V [2][SLICE]
  static constexpr int BYTES = VALS + (VB > 0 ? 2 * SLICE * VB : 0);
};

template <class K, int VB, int RADIX_BITS, int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS, 1)
    k_cluster_sort(K* __restrict__ keys, ValT<VB>* __restrict__ vals, uint32_t n, int begin_bit,
                   int end_bit, Ctrl* ctrl, KeyXf<K> xf) {
  using V = ValT<VB>;
  using S = ClusterSmem<K, VB, RADIX_BITS, THREADS, ITEMS>;
  constexpr int RADIX = S::RADIX, WARPS = S::WARPS, SLICE = S::SLICE;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* s_wh = reinterpret_cast<uint32_t*>(smem + S::WH);
  uint32_t* s_mm = reinterpret_cast<uint32_t*>(smem + S::MM);
  uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem + S::CNT);
  uint32_t* s_base = reinterpret_cast<uint32_t*>(smem + S::BASE);
  uint32_t* s_lst = reinterpret_cast<uint32_t*>(smem + S::LST);
  uint32_t* s_tot = reinterpret_cast<uint32_t*>(smem + S::TOT);
  K* s_k = reinterpret_cast<K*>(smem + S::KEYS);
  V* s_v = reinterpret_cast<V*>(smem + S::VALS);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t rank = cluster_ctarank();
  const uint32_t ncta = gridDim.x;  // the grid is one cluster
  const int passes = (end_bit - begin_bit + RADIX_BITS - 1) / RADIX_BITS;
  if (ctrl != nullptr && blockIdx.x == 0 && tid == 0) {
    ctrl->error = 0u;
    ctrl->error_info = 0u;
    ctrl->exec_mask = (1u << passes) - 1u;  // every pass runs (in shared memory)
    stat_clear_times(ctrl);
    stat_begin(ctrl, n, uint32_t(sizeof(K)) | uint32_t(VB) << 8 | uint32_t(passes) << 16 |
                            3u << 24);
  }

  // load this CTA's slice (transformed keys; the largest key past the end)
  const uint32_t base0 = rank * uint32_t(SLICE);
  for (uint32_t i = tid; i < uint32_t(SLICE); i += THREADS) {
    const uint32_t g = base0 + i;
    K k = ~K(0);
    if (g < n) k = xf.on ? xf_fwd(keys[g], xf) : keys[g];
    s_k[i] = k;
    if constexpr (VB > 0) s_v[i] = g < n ? vals[g] : V(0);
  }
  for (int i = tid; i < WARPS * RADIX; i += THREADS) s_mm[i] = 0u;
  __syncthreads();

  const uint32_t slot0 = uint32_t(warp * ITEMS * 32 + lane);
  int src = 0;
  for (int lo = begin_bit; lo < end_bit; lo += RADIX_BITS) {
    const uint32_t shift = uint32_t(lo);
    const uint32_t mask = (1u << (min(lo + RADIX_BITS, end_bit) - lo)) - 1u;
    K* ks = s_k + src * SLICE;
    V* vs = s_v + src * SLICE;
    // ---- 1. local rank
    for (int i = tid; i < WARPS * RADIX; i += THREADS) s_wh[i] = 0u;
    __syncthreads();
    K key[ITEMS];
    V val[ITEMS];
    uint32_t dp[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      key[j] = ks[slot0 + j * 32];
      if constexpr (VB > 0) val[j] = vs[slot0 + j * 32];
      dp[j] = digit_of(key[j], shift, mask);
    }
    warp_rank_packed<ITEMS>(dp, s_wh + warp * RADIX, s_mm + warp * RADIX, lane);
    __syncthreads();
    uint32_t run = 0u;
    if (tid < RADIX) {
#pragma unroll
      for (int w = 0; w < WARPS; ++w) {
        const uint32_t c = s_wh[w * RADIX + tid];
        s_wh[w * RADIX + tid] = run;
        run += c;
      }
      // ---- 2. this CTA's counts into every CTA's table
      for (uint32_t c = 0; c < ncta; ++c)
        st_cluster(map_shared(s_cnt + rank * RADIX + tid, c), run);
    }
    // ---- 3a. the CTA's keys in digit order, staged in its source buffer
    const uint32_t lstart = block_exclusive_scan<THREADS>(run, s_tot);
    if (tid < RADIX) s_lst[tid] = lstart;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const uint32_t d = dp[j] >> 16;
      const uint32_t at = s_lst[d] + s_wh[warp * RADIX + d] + (dp[j] & 0xffffu);
      ks[at] = key[j];
      if constexpr (VB > 0) vs[at] = val[j];
    }
    // every CTA's counts have landed and the stage is complete
    cluster_sync_all();
    uint32_t total = 0u, below = 0u;
    if (tid < RADIX) {
      for (uint32_t c = 0; c < ncta; ++c) {
        const uint32_t x = s_cnt[c * RADIX + tid];
        total += x;
        if (c < rank) below += x;
      }
    }
    const uint32_t start = block_exclusive_scan<THREADS>(total, s_tot);
    // staged key i of digit d goes to global position s_base[d] + i
    if (tid < RADIX) s_base[tid] = start + below - s_lst[tid];
    __syncthreads();
    // ---- 3b. remote stores of the staged runs into the owners' destination buffers
    K* kd = s_k + (src ^ 1) * SLICE;
    V* vd = s_v + (src ^ 1) * SLICE;
#pragma unroll 4
    for (int i = tid; i < SLICE; i += THREADS) {
      const K k = ks[i];
      const uint32_t g = s_base[digit_of(k, shift, mask)] + uint32_t(i);
      const uint32_t owner = g / uint32_t(SLICE), at = g % uint32_t(SLICE);
      st_cluster(map_shared(kd + at, owner), k);
      if constexpr (VB > 0) st_cluster(map_shared(vd + at, owner), vs[i]);
    }
    // ---- 4. the destination buffers are complete
    cluster_sync_all();
    src ^= 1;
  }

  // write this CTA's slice out (untransformed)
  const K* ks = s_k + src * SLICE;
  const V* vs = s_v + src * SLICE;
  for (uint32_t i = tid; i < uint32_t(SLICE); i += THREADS) {
    const uint32_t g = base0 + i;
    if (g < n && dbg_ok(g, n, kSiteClusterOut)) {
      keys[g] = xf.on ? xf_inv(ks[i], xf) : ks[i];
      if constexpr (VB > 0) vals[g] = vs[i];
    }
  }
  if (ctrl != nullptr) {
    __syncthreads();
    if (tid == 0) atomicMax(&ctrl->t_upsweep, stat_now(ctrl));
  }
}

}  // namespace rs
