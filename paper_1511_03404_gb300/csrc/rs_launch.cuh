// Host launchers of the sort variants (one instantiation per compiled tile
// shape).  Each launcher enqueues a complete sort on the caller's stream:
//   memset(ctrl + counts) -> k_upsweep -> k_onesweep x passes
// or, for arrays that fit one tile, a single k_small_sort.
#pragma once

#include <algorithm>

#include "rs_cluster.cuh"
#include "rs_fused.cuh"
#include "rs_host.h"
#include "rs_kernels.cuh"

namespace rs {

// PERSIST: the passes run as k_onesweep_persist on a grid of SMs x resident
// CTAs instead of one CTA per tile.  UNIT: lanes per ranking unit (32: warps,
// 16: half warps).  INPLACE: keys only, staged in the key buffer itself.
template <class K, int VB, int R, int THREADS, int ITEMS, int MINB, bool PERSIST = false,
          int UNIT = 32, bool INPLACE = false>
struct OnesweepSort {
  static constexpr int RADIX = 1 << R;
  static constexpr int TILE = THREADS * ITEMS;
  static constexpr int UP_THREADS = 1024;
  static constexpr int MAXP = (8 * int(sizeof(K)) + R - 1) / R;
  using S = OnesweepSmem<K, VB, R, THREADS, ITEMS, UNIT, INPLACE>;

  static size_t tiles(uint32_t n) { return (size_t(n) + TILE - 1) / TILE; }

  static size_t workspace(uint32_t n, int passes) {
    return onesweep_layout(passes, R, tiles(n)).total;
  }

  // early: the kernel after this one (the first pass) may be scheduled as
  // soon as this one starts, because its grid fills the GPU anyway
  // shape: the per-call record of rs_workspace_stats (0: none)
  static cudaError_t upsweep(const SortArgs& a, int passes, const Layout& L, bool clear_status,
                             bool early = false, uint32_t shape = 0u) {
    char* ws = static_cast<char*>(a.ws);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws);
    cudaError_t e = cudaMemsetAsync(ws, 0, L.memset_bytes, a.stream);
    if (e != cudaSuccess) return e;
    const bool full = R == 8 && a.begin_bit == 0 && a.end_bit == 8 * int(sizeof(K));
    auto kern = full ? &k_upsweep<K, R, UP_THREADS, MAXP, (R == 8)>
                     : &k_upsweep<K, R, UP_THREADS, MAXP, false>;
    constexpr int SLOTS = sizeof(K) == 4 ? 32 : 16;
    const int max_smem = MAXP * RADIX * SLOTS * 4;
    const int occ = prepare_kernel(reinterpret_cast<const void*>(kern), UP_THREADS, max_smem);
    if (occ <= 0) return cudaErrorInvalidConfiguration;
    const int smem = passes * RADIX * SLOTS * 4;
    constexpr uint32_t per_cta = UP_THREADS * (16 / sizeof(K)) * 4;
    const uint32_t want = (a.n + per_cta - 1) / per_cta;
    const uint32_t grid =
        std::max(1u, std::min(uint32_t(device_info().sms * occ), want));
    const uint64_t zero_vec4 = clear_status ? L.status_bytes / 16 : 0;
    prof_before(a.stream);
    kern<<<grid, UP_THREADS, smem, a.stream>>>(
        static_cast<const K*>(a.keys), a.n, a.begin_bit, a.end_bit, passes,
        reinterpret_cast<uint32_t*>(ws + L.counts), reinterpret_cast<uint32_t*>(ws + L.offsets),
        ctrl, reinterpret_cast<uint4*>(ws + L.status), zero_vec4,
        make_key_xf<K>(a.key_kind, a.descending), early, shape);
    e = cudaGetLastError();
    prof_after(a.stream, 0, double(a.n) * sizeof(K));
    return e;
  }

  static cudaError_t run(const SortArgs& a, int* in_alt) {
    const int passes = num_passes(a.begin_bit, a.end_bit, R);
    *in_alt = passes & 1;
    const size_t nt = tiles(a.n);
    const Layout L = onesweep_layout(passes, R, nt);
    using V = ValT<VB>;
    auto kern = [] {  // instantiate only the kernel this variant launches
      if constexpr (PERSIST)
        return &k_onesweep_persist<K, VB, R, THREADS, ITEMS, MINB, UNIT, INPLACE>;
      else
        return &k_onesweep<K, VB, R, THREADS, ITEMS, MINB, UNIT, INPLACE>;
    }();
    const int occ = prepare_kernel(reinterpret_cast<const void*>(kern), THREADS, S::BYTES);
    if (occ <= 0) return cudaErrorInvalidConfiguration;
    // a pass grid that fills the GPU (resident CTAs, or more tiles than CTA
    // slots) is scheduled early, while the kernel before it runs; a one-wave
    // grid scheduled that early lands on whichever SMs have room, so it is
    // let in only as the kernel before it exits
    const bool pdl = pdl_enabled();
    const bool fills = pdl && (PERSIST || nt > size_t(device_info().sms) * occ);
    const uint32_t shape = uint32_t(sizeof(K)) | uint32_t(VB) << 8 | uint32_t(passes) << 16 |
                           1u << 24;
    nvtx_push("rs upsweep");
    cudaError_t e = upsweep(a, passes, L, true, fills, shape);
    nvtx_pop();
    if (e != cudaSuccess) return e;
    char* ws = static_cast<char*>(a.ws);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws);
    const int slot = prof_note_mask(a.stream, &ctrl->exec_mask);
    const unsigned grid =
        PERSIST ? unsigned(std::min<size_t>(nt, size_t(device_info().sms) * occ)) : unsigned(nt);
    const double bytes = 2.0 * double(a.n) * double(sizeof(K) + VB);
    const KeyXf<K> xf = make_key_xf<K>(a.key_kind, a.descending);
    for (int p = 0; p < passes; ++p) {
      const int lo = a.begin_bit + p * R;
      const int width = std::min(R, a.end_bit - lo);
      const uint32_t mask = (1u << width) - 1u;
      prof_before(a.stream);
      // programmatic dependent launch: the pass's CTAs may be scheduled before
      // the kernel ahead of it has finished (when that one lets them in);
      // each waits for it (pdl_wait) first, so the launch gap is hidden
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(grid);
      cfg.blockDim = dim3(THREADS);
      cfg.dynamicSmemBytes = S::BYTES;
      cfg.stream = a.stream;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = pdl ? 1 : 0;
      nvtx_push(kPassNames[p]);
      e = cudaLaunchKernelEx(
          &cfg, kern, static_cast<K*>(a.keys), static_cast<K*>(a.keys_alt),
          static_cast<V*>(a.vals), static_cast<V*>(a.vals_alt), a.n, p, uint32_t(lo), mask,
          static_cast<const uint32_t*>(reinterpret_cast<const uint32_t*>(ws + L.offsets) +
                                       size_t(p) * RADIX),
          reinterpret_cast<uint32_t*>(ws + L.status) + size_t(p) * L.tiles * RADIX,
          reinterpret_cast<uint32_t*>(ws + L.gagg) + size_t(p) * L.groups * RADIX,
          reinterpret_cast<uint32_t*>(ws + L.ginc) + size_t(p) * L.groups * RADIX, uint32_t(nt),
          ctrl, a.knobs, xf, fills);
      if (e == cudaSuccess) e = cudaGetLastError();
      nvtx_pop();
      prof_after(a.stream, 1, bytes, slot, p);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }

  static cudaError_t count(const SortArgs& a) {
    const int passes = num_passes(a.begin_bit, a.end_bit, R);
    const Layout L = onesweep_layout(passes, R, tiles(a.n));
    return upsweep(a, passes, L, false);
  }

  static Variant describe() {
    Variant v{};
    v.key_bytes = int(sizeof(K));
    v.val_bytes = VB;
    v.kind = PERSIST ? kOnesweepPersist : kOnesweep;
    v.radix_bits = R;
    v.threads = THREADS;
    v.items = ITEMS;
    v.max_n = (1u << 30) - 1u;
    v.workspace = &workspace;
    v.run = &run;
    v.count = &count;
    return v;
  }
};

// The whole sort in one cooperative launch (k_fused): for moderate sizes,
// where the launches of the multi-kernel form dominate.
template <class K, int VB, int R, int THREADS, int ITEMS, int MINB>
struct FusedSort {
  using Base = OnesweepSort<K, VB, R, THREADS, ITEMS, MINB>;
  using F = FusedSmem<K, VB, R, THREADS, ITEMS>;
  static constexpr int RADIX = 1 << R;

  static cudaError_t run(const SortArgs& a, int* in_alt) {
    const int passes = num_passes(a.begin_bit, a.end_bit, R);
    *in_alt = passes & 1;
    const size_t nt = Base::tiles(a.n);
    const Layout L = onesweep_layout(passes, R, nt);
    char* ws = static_cast<char*>(a.ws);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws);
    cudaError_t e = cudaMemsetAsync(ws, 0, L.memset_bytes, a.stream);
    if (e != cudaSuccess) return e;
    using V = ValT<VB>;
    auto kern = &k_fused<K, VB, R, THREADS, ITEMS, MINB>;
    const int occ = prepare_kernel(reinterpret_cast<const void*>(kern), THREADS, F::BYTES);
    if (occ <= 0) return cudaErrorInvalidConfiguration;
    const unsigned grid =
        unsigned(std::max<size_t>(1, std::min<size_t>(nt, size_t(device_info().sms) * occ)));
    K* k0 = static_cast<K*>(a.keys);
    K* k1 = static_cast<K*>(a.keys_alt);
    V* v0 = static_cast<V*>(a.vals);
    V* v1 = static_cast<V*>(a.vals_alt);
    uint32_t n = a.n;
    int begin = a.begin_bit, end = a.end_bit, np = passes;
    uint32_t* counts = reinterpret_cast<uint32_t*>(ws + L.counts);
    uint32_t* status = reinterpret_cast<uint32_t*>(ws + L.status);
    uint32_t* gagg = reinterpret_cast<uint32_t*>(ws + L.gagg);
    uint32_t* ginc = reinterpret_cast<uint32_t*>(ws + L.ginc);
    uint32_t tiles = uint32_t(nt), tiles_pad = uint32_t(L.tiles), groups_pad = uint32_t(L.groups);
    uint4* zero_base = reinterpret_cast<uint4*>(ws + L.status);
    uint64_t zero_vec4 = L.status_bytes / 16;
    Knobs knobs = a.knobs;
    KeyXf<K> xf = make_key_xf<K>(a.key_kind, a.descending);
    uint32_t shape = uint32_t(sizeof(K)) | uint32_t(VB) << 8 | uint32_t(passes) << 16 | 2u << 24;
    void* args[] = {&k0, &k1, &v0, &v1, &n, &begin, &end, &np, &counts, &status, &gagg, &ginc,
                    &tiles, &tiles_pad, &groups_pad, &zero_base, &zero_vec4, &ctrl, &knobs, &xf,
                    &shape};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = F::BYTES;
    cfg.stream = a.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident: the barriers need it
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    prof_before(a.stream);
    e = cudaLaunchKernelExC(&cfg, reinterpret_cast<const void*>(kern), args);
    prof_after(a.stream, 1, double(a.n) * (sizeof(K) + passes * 2.0 * (sizeof(K) + VB)));
    return e;
  }

  static Variant describe() {
    Variant v = Base::describe();
    v.kind = kFused;
    v.max_n = 1u << 24;
    v.run = &run;
    return v;
  }
};

// The whole sort in one thread-block cluster of up to CL CTAs
// (k_cluster_sort): arrays of up to CL x THREADS x ITEMS elements stay in
// the cluster's shared memory for every pass.
template <class K, int VB, int R, int THREADS, int ITEMS, int CL>
struct ClusterSort {
  using S = ClusterSmem<K, VB, R, THREADS, ITEMS>;
  static_assert(CL >= 1 && CL <= S::MAX_CL, "portable cluster sizes");

  static size_t workspace(uint32_t, int) { return 0; }

  static cudaError_t run(const SortArgs& a, int* in_alt) {
    using V = ValT<VB>;
    *in_alt = 0;  // sorted in place
    auto kern = &k_cluster_sort<K, VB, R, THREADS, ITEMS>;
    if (prepare_kernel(reinterpret_cast<const void*>(kern), THREADS, S::BYTES) <= 0)
      return cudaErrorInvalidConfiguration;
    const unsigned ncta = unsigned((size_t(a.n) + S::SLICE - 1) / S::SLICE);
    if (ncta < 1 || ncta > unsigned(CL)) return cudaErrorInvalidValue;
    Ctrl* ctrl = (a.ws != nullptr && a.ws_bytes >= sizeof(Ctrl)) ? static_cast<Ctrl*>(a.ws)
                                                                  : nullptr;
    K* keys = static_cast<K*>(a.keys);
    V* vals = static_cast<V*>(a.vals);
    uint32_t n = a.n;
    int begin = a.begin_bit, end = a.end_bit;
    KeyXf<K> xf = make_key_xf<K>(a.key_kind, a.descending);
    void* args[] = {&keys, &vals, &n, &begin, &end, &ctrl, &xf};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ncta);
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = S::BYTES;
    cfg.stream = a.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;  // the whole grid is one cluster
    attr[0].val.clusterDim.x = ncta;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    prof_before(a.stream);
    const cudaError_t e = cudaLaunchKernelExC(&cfg, reinterpret_cast<const void*>(kern), args);
    prof_after(a.stream, 2, 2.0 * double(a.n) * double(sizeof(K) + VB));
    return e;
  }

  static Variant describe() {
    Variant v{};
    v.key_bytes = int(sizeof(K));
    v.val_bytes = VB;
    v.kind = kCluster;
    v.radix_bits = R;
    v.threads = THREADS;
    v.items = ITEMS;
    v.max_n = uint32_t(CL) * uint32_t(S::SLICE);
    v.workspace = &workspace;
    v.run = &run;
    v.count = nullptr;
    return v;
  }
};

template <class K, int VB, int R, int THREADS, int ITEMS>
struct SmallSort {
  static constexpr int TILE = THREADS * ITEMS;
  using S = SmallSmem<K, VB, R, THREADS, ITEMS>;

  static size_t workspace(uint32_t, int) { return 0; }

  static cudaError_t run(const SortArgs& a, int* in_alt) {
    using V = ValT<VB>;
    *in_alt = 0;  // sorted in place
    auto kern = &k_small_sort<K, VB, R, THREADS, ITEMS>;
    if (prepare_kernel(reinterpret_cast<const void*>(kern), THREADS, S::BYTES) <= 0)
      return cudaErrorInvalidConfiguration;
    prof_before(a.stream);
    Ctrl* ctrl = (a.ws != nullptr && a.ws_bytes >= sizeof(Ctrl)) ? static_cast<Ctrl*>(a.ws)
                                                                  : nullptr;
    kern<<<1, THREADS, S::BYTES, a.stream>>>(static_cast<K*>(a.keys), static_cast<V*>(a.vals),
                                             a.n, a.begin_bit, a.end_bit, ctrl,
                                             make_key_xf<K>(a.key_kind, a.descending));
    const cudaError_t e = cudaGetLastError();
    prof_after(a.stream, 2, 2.0 * double(a.n) * double(sizeof(K) + VB));
    return e;
  }

  static Variant describe() {
    Variant v{};
    v.key_bytes = int(sizeof(K));
    v.val_bytes = VB;
    v.kind = kSmall;
    v.radix_bits = R;
    v.threads = THREADS;
    v.items = ITEMS;
    v.max_n = TILE;
    v.workspace = &workspace;
    v.run = &run;
    v.count = nullptr;
    return v;
  }
};

}  // namespace rs
