// One-launch form of the sort for arrays of moderate size, where the
// separate launches of the upsweep and of each digit pass, each waiting for
// the previous one, cost more than the passes themselves.  A cooperative
// grid (every CTA resident) runs:
//   1. the digit histograms of every pass over a grid-stride share of the
//      keys (shared counters, then one global add per digit), and clears
//      the look-back words;
//   -- grid barrier --
//   2. in every CTA, the exclusive scans and the set of passes that move
//      data (the same rule as the upsweep's last CTA), kept in shared memory;
//   3. each moving pass: tiles taken from the pass's counter and sorted by
//      the onesweep tile (rank, decoupled look-back, stable scatter), with
//      L2-coherent loads of the previous pass's output;
//   -- grid barrier after each pass --
// Every barrier wait is bounded; a CTA that gives up records
// RS_ERR_TIMEOUT and returns, and the others' bounded waits end as well.
#pragma once

#include <type_traits>

#include "rs_kernels.cuh"

namespace rs {

template <class K, int VB, int RADIX_BITS, int THREADS, int ITEMS>
struct FusedSmem {
  using S = OnesweepSmem<K, VB, RADIX_BITS, THREADS, ITEMS>;
  static constexpr int RADIX = 1 << RADIX_BITS;
  static constexpr int MAXP = (8 * int(sizeof(K)) + RADIX_BITS - 1) / RADIX_BITS;
  static constexpr int OFF = (S::BYTES + 15) / 16 * 16;  // u32 [MAXP][RADIX] digit offsets
  static constexpr int FLAG = OFF + MAXP * RADIX * 4;    // u32: barrier outcome
  static constexpr int BYTES = FLAG + 16;
  // the histograms of step 1 use the warp-counter region of the tile
  static_assert(MAXP * RADIX <= S::WARPS * RADIX, "histograms fit the warp counters");
};

// All CTAs of the grid meet; false if the wait ran out or an error was
// reported (CTA-uniform).
__device__ __forceinline__ bool grid_barrier(Ctrl* ctrl, uint32_t gen, uint64_t timeout_ns,
                                             uint32_t* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&ctrl->grid_bar, 1u);
    const bool ok = wait_geq(&ctrl->grid_bar, gen * gridDim.x, ctrl, timeout_ns, 0xffffffffu);
    __threadfence();
    *s_flag = ok ? 1u : 0u;
  }
  __syncthreads();
  return *s_flag != 0u;
}

template <class K, int VB, int RADIX_BITS, int THREADS, int ITEMS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB)
    k_fused(K* __restrict__ k0, K* __restrict__ k1, ValT<VB>* __restrict__ v0,
            ValT<VB>* __restrict__ v1, uint32_t n, int begin_bit, int end_bit, int passes,
            uint32_t* __restrict__ counts, uint32_t* __restrict__ status,
            uint32_t* __restrict__ gagg, uint32_t* __restrict__ ginc, uint32_t tiles,
            uint32_t tiles_pad, uint32_t groups_pad, uint4* __restrict__ zero_base,
            uint64_t zero_vec4, Ctrl* __restrict__ ctrl, Knobs knobs, KeyXf<K> xf,
            uint32_t shape) {
  using F = FusedSmem<K, VB, RADIX_BITS, THREADS, ITEMS>;
  using S = typename F::S;
  constexpr int RADIX = F::RADIX, MAXP = F::MAXP;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* s_hist = reinterpret_cast<uint32_t*>(smem + S::WH);
  uint32_t* s_tot = reinterpret_cast<uint32_t*>(smem + S::TOT);
  uint32_t* s_misc = reinterpret_cast<uint32_t*>(smem + S::MISC);
  uint32_t* s_off = reinterpret_cast<uint32_t*>(smem + F::OFF);
  uint32_t* s_flag = reinterpret_cast<uint32_t*>(smem + F::FLAG);
  const int tid = threadIdx.x;
  const bool rec = blockIdx.x == 0 && tid == 0;  // keeps the per-call record
  if (rec) stat_begin(ctrl, n, shape);

  // ---- 1. histograms of every pass, and the look-back words cleared
  for (int i = tid; i < passes * RADIX; i += THREADS) s_hist[i] = 0u;
  __syncthreads();
  auto count_all = [&](auto XF) {
    for (uint32_t i = blockIdx.x * THREADS + tid; i < n; i += gridDim.x * THREADS) {
      K k = k0[i];
      if constexpr (decltype(XF)::value) k = xf_fwd(k, xf);
#pragma unroll
      for (int p = 0; p < MAXP; ++p) {
        if (p < passes) {
          const int lo = begin_bit + p * RADIX_BITS;
          const uint32_t mask = (1u << min(RADIX_BITS, end_bit - lo)) - 1u;
          atomicAdd(&s_hist[p * RADIX + int(digit_of(k, uint32_t(lo), mask))], 1u);
        }
      }
    }
  };
  if (xf.on)
    count_all(std::true_type{});
  else
    count_all(std::false_type{});
  for (uint64_t i = uint64_t(blockIdx.x) * THREADS + tid; i < zero_vec4;
       i += uint64_t(gridDim.x) * THREADS)
    if (dbg_ok(i, zero_vec4, kSiteFusedClear)) zero_base[i] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  for (int w = tid; w < passes * RADIX; w += THREADS)
    if (s_hist[w] && dbg_ok(w, uint64_t(passes) * RADIX, kSiteFusedCounts))
      atomicAdd(&counts[w], s_hist[w]);
  uint32_t gen = 1;
  if (!grid_barrier(ctrl, gen, knobs.timeout_ns, s_flag)) return;

  // ---- 2. scans and moving passes, in every CTA
  uint32_t exec = 0u;
  for (int p = 0; p < passes; ++p) {
    const uint32_t c = tid < RADIX ? ld_relaxed(&counts[p * RADIX + tid]) : 0u;
    const uint32_t e = block_exclusive_scan<THREADS>(c, s_tot);
    if (tid < RADIX) s_off[p * RADIX + tid] = e;
    if (!__syncthreads_or(tid < RADIX && c == n)) exec |= 1u << p;
  }
  if ((__popc(exec) & 1) != (passes & 1)) {  // keep the result in buffer (passes mod 2)
    const uint32_t skipped = ~exec & ((1u << passes) - 1u);
    exec |= skipped & (0u - skipped);
  }
  if (rec) {
    ctrl->exec_mask = exec;
    ctrl->t_upsweep = stat_now(ctrl);
  }

  // ---- 3. the passes that move data
  for (int p = 0; p < passes; ++p) {
    if (!((exec >> p) & 1u)) continue;
    const bool from_alt = (__popc(exec & ((1u << p) - 1u)) & 1) != 0;
    TileArgs<K, VB> t;
    t.ksrc = from_alt ? k1 : k0;
    t.kdst = from_alt ? k0 : k1;
    t.vsrc = from_alt ? v1 : v0;
    t.vdst = from_alt ? v0 : v1;
    t.n = n;
    const int lo = begin_bit + p * RADIX_BITS;
    t.shift = uint32_t(lo);
    t.mask = (1u << min(RADIX_BITS, end_bit - lo)) - 1u;
    t.pass_offsets = s_off + p * RADIX;
    t.status = status + size_t(p) * tiles_pad * RADIX;
    t.tile0 = 0u;
    t.gagg = gagg + size_t(p) * groups_pad * RADIX;
    t.ginc = ginc + size_t(p) * groups_pad * RADIX;
    t.tiles = tiles;
    t.lb_words = uint64_t(tiles_pad) * RADIX;
    t.g_words = uint64_t(groups_pad) * RADIX;
    t.lb_small = knobs.lb_small != 0;
    t.xf = xf;
    t.xin = xf.on && p == __ffs(int(exec)) - 1;
    t.xout = xf.on && p == 31 - __clz(exec);
    if (rec) ctrl->t_pass[p][0] = stat_now(ctrl);
    for (;;) {
      __syncthreads();  // the previous tile is done with s_misc
      if (tid == 0) {
        s_misc[2] = ld_relaxed(&ctrl->error);
        s_misc[0] = s_misc[2] ? tiles : atomicAdd(&ctrl->tile_counter[p], 1u);
      }
      __syncthreads();
      const uint32_t tile = s_misc[0];
      if (tile >= tiles) break;  // CTA-uniform
      t.tile = tile;
      t.silent = (int(tile) == knobs.drop_tile) && (p == knobs.drop_pass);
      t.dbg_bad = false;
      t.trace = nullptr;
      onesweep_tile<K, VB, RADIX_BITS, THREADS, ITEMS, true>(t, ctrl, knobs.timeout_ns, smem);
    }
    ++gen;
    if (!grid_barrier(ctrl, gen, knobs.timeout_ns, s_flag)) return;
    if (rec) ctrl->t_pass[p][1] = stat_now(ctrl);
  }
}

}  // namespace rs
