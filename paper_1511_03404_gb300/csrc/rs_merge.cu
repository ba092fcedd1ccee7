// Merge sort (Sec. 2.4, the parallel merge sort of Satish et al.): a
// comparison sort, stable, for keys that the radix passes do not take
// (128-bit keys) as well as 32- and 64-bit keys.
//   k_ms_tile   sorts each tile of kTile (4096) elements in one CTA: a stable
//               odd-even transposition sort of each thread's kItems
//               consecutive elements in registers, then merge rounds of
//               doubling width in shared memory;
//   k_ms_split  for a global merge of runs of width w, finds where each
//               output tile of the merged pair begins in the left run (the
//               merge path: a binary search along the tile's diagonal);
//   k_ms_merge  merges one output tile per CTA from the two input ranges its
//               split delimits.
// Ties always take the element of the left run, which holds the earlier
// input positions, so every merge (and the whole sort) is stable.
#include <algorithm>

#include "../../include/rs.h"
#include "rs_debug.cuh"
#include "rs_host.h"

namespace rs {

namespace {

constexpr int kMsThreads = 256;
constexpr int kMsItems = 16;
constexpr int kTile = kMsThreads * kMsItems;

// A 128-bit unsigned key: value = lo + 2^64 * hi (little-endian words).
struct alignas(16) Key128 {
  uint64_t lo, hi;
};

__device__ __forceinline__ bool key_less(uint32_t a, uint32_t b) { return a < b; }
__device__ __forceinline__ bool key_less(uint64_t a, uint64_t b) { return a < b; }
__device__ __forceinline__ bool key_less(const Key128& a, const Key128& b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}

template <class K>
__device__ __forceinline__ K key_max();
template <>
__device__ __forceinline__ uint32_t key_max<uint32_t>() { return ~0u; }
template <>
__device__ __forceinline__ uint64_t key_max<uint64_t>() { return ~0ull; }
template <>
__device__ __forceinline__ Key128 key_max<Key128>() { return Key128{~0ull, ~0ull}; }

struct NoVal {};

// Shared-memory slot of element i: one pad slot after every 32 elements, so
// that a warp reading or writing each thread's kMsItems consecutive elements
// (stride kMsItems) spreads over the banks instead of hitting a few.
__device__ __forceinline__ uint32_t pad(uint32_t i) { return i + (i >> 5); }

// A run of elements in shared memory, indexed through pad().
template <class T>
struct Padded {
  T* base;
  uint32_t first;  // element index of run[0]
  __device__ __forceinline__ T& operator[](uint32_t i) const { return base[pad(first + i)]; }
};

// Elements taken from the left run a[0 .. na) at diagonal `diag` of the merge
// of a and b[0 .. nb): the largest i with a[i-1] <= b[diag-i] (ties: a first).
template <class A, class B>
__device__ __forceinline__ uint32_t merge_path(const A& a, uint32_t na, const B& b, uint32_t nb,
                                               uint32_t diag) {
  uint32_t lo = diag > nb ? diag - nb : 0u;
  uint32_t hi = min(diag, na);
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (!key_less(b[diag - 1 - mid], a[mid])) lo = mid + 1;  // a[mid] <= b[...]: take it
    else hi = mid;
  }
  return lo;
}

// Merge min(kMsItems, na - i + nb - j) outputs, starting at (a + i, b + j),
// into registers.
template <class K, class V, bool HAS_V, class RK, class RV>
__device__ __forceinline__ void merge_items(const RK& a, const RV& av, uint32_t na, const RK& b,
                                            const RV& bv, uint32_t nb, uint32_t i, uint32_t j,
                                            K (&k)[kMsItems], V (&v)[kMsItems]) {
#pragma unroll
  for (int t = 0; t < kMsItems; ++t) {
    if (i >= na && j >= nb) break;  // both runs used up (the last, partial tile)
    const bool take_a = j >= nb || (i < na && !key_less(b[j], a[i]));
    if (take_a) {
      k[t] = a[i];
      if constexpr (HAS_V) v[t] = av[i];
      ++i;
    } else {
      k[t] = b[j];
      if constexpr (HAS_V) v[t] = bv[j];
      ++j;
    }
  }
}

template <class K, class V, bool HAS_V>
struct MsSmem {
  static constexpr int SLOTS = kTile + kTile / 32;  // with the pad slots
  static constexpr int KEYS = 0;
  static constexpr int VALS = (SLOTS * int(sizeof(K)) + 15) / 16 * 16;
  static constexpr int BYTES = VALS + (HAS_V ? SLOTS * int(sizeof(V)) : 0);
};

// One tile per CTA, sorted in place (src may equal dst).
template <class K, class V, bool HAS_V>
__global__ void __launch_bounds__(kMsThreads) k_ms_tile(const K* src, const V* vsrc, K* dst,
                                                        V* vdst, uint32_t n) {
  using S = MsSmem<K, V, HAS_V>;
  extern __shared__ __align__(16) unsigned char smem[];
  K* sk = reinterpret_cast<K*>(smem + S::KEYS);
  V* sv = reinterpret_cast<V*>(smem + S::VALS);
  const uint32_t base = blockIdx.x * uint32_t(kTile);
  const uint32_t len = min(uint32_t(kTile), n - base);
  const int tid = threadIdx.x;
  // past the end: the largest key; being last in input order too, the
  // padding stays behind every real key (stability)
  for (uint32_t i = tid; i < uint32_t(kTile); i += kMsThreads) {
    sk[pad(i)] = i < len ? src[base + i] : key_max<K>();
    if constexpr (HAS_V) sv[pad(i)] = i < len ? vsrc[base + i] : V{};
  }
  __syncthreads();
  K k[kMsItems];
  V v[kMsItems];
  const uint32_t o = uint32_t(tid) * kMsItems;
#pragma unroll
  for (int t = 0; t < kMsItems; ++t) {
    k[t] = sk[pad(o + t)];
    if constexpr (HAS_V) v[t] = sv[pad(o + t)];
  }
  // odd-even transposition: swaps only strictly out-of-order neighbours, so
  // equal keys keep their order
#pragma unroll
  for (int r = 0; r < kMsItems; ++r) {
#pragma unroll
    for (int t = r & 1; t + 1 < kMsItems; t += 2) {
      if (key_less(k[t + 1], k[t])) {
        const K tk = k[t];
        k[t] = k[t + 1];
        k[t + 1] = tk;
        if constexpr (HAS_V) {
          const V tv = v[t];
          v[t] = v[t + 1];
          v[t + 1] = tv;
        }
      }
    }
  }
  for (uint32_t w = kMsItems; w < uint32_t(kTile); w *= 2) {
    __syncthreads();
#pragma unroll
    for (int t = 0; t < kMsItems; ++t) {
      sk[pad(o + t)] = k[t];
      if constexpr (HAS_V) sv[pad(o + t)] = v[t];
    }
    __syncthreads();
    const uint32_t pair = o / (2 * w) * (2 * w);
    const uint32_t d = o - pair;
    const Padded<K> a{sk, pair}, b{sk, pair + w};
    const Padded<V> av{sv, pair}, bv{sv, pair + w};
    const uint32_t i = merge_path(a, w, b, w, d);
    merge_items<K, V, HAS_V>(a, av, w, b, bv, w, i, d - i, k, v);
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < kMsItems; ++t) {
    sk[pad(o + t)] = k[t];
    if constexpr (HAS_V) sv[pad(o + t)] = v[t];
  }
  __syncthreads();
  for (uint32_t i = tid; i < len; i += kMsThreads) {
    if (!dbg_ok(uint64_t(base) + i, n, kSiteMergeTile)) continue;
    dst[base + i] = sk[pad(i)];
    if constexpr (HAS_V) vdst[base + i] = sv[pad(i)];
  }
}

// Runs of width w (a multiple of kTile) are merged in pairs; output tile c
// starts at p = c * kTile inside the pair [base, base + 2w).  split[c] = how
// many of the pair's left-run elements precede that tile.
template <class K>
__global__ void k_ms_split(const K* __restrict__ src, uint32_t n, uint32_t w,
                           uint32_t* __restrict__ split, uint32_t tiles) {
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < tiles;
       c += gridDim.x * blockDim.x) {
    const uint64_t p = uint64_t(c) * kTile;
    const uint64_t base = p / (2ull * w) * (2ull * w);
    const uint32_t na = uint32_t(min(uint64_t(w), n - base));
    const uint32_t nb = uint32_t(n - base - na < w ? n - base - na : w);
    const uint32_t at = merge_path(src + base, na, src + base + na, nb, uint32_t(p - base));
    if (dbg_ok(c, tiles, kSiteMergeSplit)) split[c] = at;
  }
}

template <class K, class V, bool HAS_V>
__global__ void __launch_bounds__(kMsThreads) k_ms_merge(const K* __restrict__ src,
                                                         const V* __restrict__ vsrc,
                                                         K* __restrict__ dst,
                                                         V* __restrict__ vdst, uint32_t n,
                                                         uint32_t w,
                                                         const uint32_t* __restrict__ split) {
  using S = MsSmem<K, V, HAS_V>;
  extern __shared__ __align__(16) unsigned char smem[];
  K* sk = reinterpret_cast<K*>(smem + S::KEYS);
  V* sv = reinterpret_cast<V*>(smem + S::VALS);
  const uint32_t c = blockIdx.x;
  const uint64_t p0 = uint64_t(c) * kTile;
  const uint64_t p1 = min(p0 + kTile, uint64_t(n));
  const uint64_t base = p0 / (2ull * w) * (2ull * w);  // kTile divides 2w: one pair per CTA
  const uint32_t na = uint32_t(min(uint64_t(w), n - base));
  const uint32_t nb = uint32_t(n - base - na < w ? n - base - na : w);
  const uint32_t d0 = uint32_t(p0 - base), d1 = uint32_t(p1 - base);
  const uint32_t i0 = split[c];
  const uint32_t i1 = (p1 < base + na + nb) ? split[c + 1] : na;  // the pair's end: all of a
  const uint32_t j0 = d0 - i0, j1 = d1 - i1;
  const uint32_t la = i1 - i0, lb = j1 - j0;
  const K* a = src + base;
  const K* b = src + base + na;
  const int tid = threadIdx.x;
  for (uint32_t t = tid; t < la + lb; t += kMsThreads) {
    if (t < la) {
      sk[pad(t)] = a[i0 + t];
      if constexpr (HAS_V) sv[pad(t)] = vsrc[base + i0 + t];
    } else {
      sk[pad(t)] = b[j0 + t - la];
      if constexpr (HAS_V) sv[pad(t)] = vsrc[base + na + j0 + t - la];
    }
  }
  __syncthreads();
  K k[kMsItems];
  V v[kMsItems];
  const uint32_t o = uint32_t(tid) * kMsItems;
  const uint32_t total = la + lb;
  if (o < total) {
    const Padded<K> ra{sk, 0u}, rb{sk, la};
    const Padded<V> rav{sv, 0u}, rbv{sv, la};
    const uint32_t i = merge_path(ra, la, rb, lb, o);
    merge_items<K, V, HAS_V>(ra, rav, la, rb, rbv, lb, i, o - i, k, v);
  }
  __syncthreads();
  if (o < total) {
#pragma unroll
    for (int t = 0; t < kMsItems; ++t) {
      if (o + t < total) {
        sk[pad(o + t)] = k[t];
        if constexpr (HAS_V) sv[pad(o + t)] = v[t];
      }
    }
  }
  __syncthreads();
  for (uint32_t t = tid; t < total; t += kMsThreads) {
    if (!dbg_ok(p0 + t, n, kSiteMergeOut)) continue;
    dst[p0 + t] = sk[pad(t)];
    if constexpr (HAS_V) vdst[p0 + t] = sv[pad(t)];
  }
}

template <class K, class V, bool HAS_V>
struct MergeSort {
  using S = MsSmem<K, V, HAS_V>;

  static uint32_t tiles(size_t n) { return uint32_t((n + kTile - 1) / kTile); }
  static size_t workspace(size_t n) { return align_up((size_t(tiles(n)) + 1) * 4, 256); }

  static cudaError_t run(void* keys, void* vals, void* keys_alt, void* vals_alt, size_t n,
                         void* ws, cudaStream_t s, int* in_alt) {
    auto tile_k = &k_ms_tile<K, V, HAS_V>;
    auto merge_k = &k_ms_merge<K, V, HAS_V>;
    if (prepare_kernel(reinterpret_cast<const void*>(tile_k), kMsThreads, S::BYTES) <= 0 ||
        prepare_kernel(reinterpret_cast<const void*>(merge_k), kMsThreads, S::BYTES) <= 0)
      return cudaErrorInvalidConfiguration;
    K* bufk[2] = {static_cast<K*>(keys), static_cast<K*>(keys_alt)};
    V* bufv[2] = {static_cast<V*>(vals), static_cast<V*>(vals_alt)};
    const uint32_t nt = tiles(n);
    prof_before(s);
    tile_k<<<nt, kMsThreads, S::BYTES, s>>>(bufk[0], bufv[0], bufk[0], bufv[0], uint32_t(n));
    cudaError_t e = cudaGetLastError();
    prof_after(s, RS_KERNEL_MERGE, 2.0 * double(n) * double(sizeof(K) + (HAS_V ? sizeof(V) : 0)));
    if (e != cudaSuccess) return e;
    int cur = 0;
    uint32_t* split = static_cast<uint32_t*>(ws);
    for (uint64_t w = kTile; w < n; w *= 2) {
      const unsigned sg = unsigned(std::min<uint64_t>((nt + 255) / 256, 4096));
      k_ms_split<K><<<sg, 256, 0, s>>>(bufk[cur], uint32_t(n), uint32_t(w), split, nt);
      prof_before(s);
      merge_k<<<nt, kMsThreads, S::BYTES, s>>>(bufk[cur], bufv[cur], bufk[cur ^ 1],
                                                bufv[cur ^ 1], uint32_t(n), uint32_t(w), split);
      e = cudaGetLastError();
      prof_after(s, RS_KERNEL_MERGE,
                 2.0 * double(n) * double(sizeof(K) + (HAS_V ? sizeof(V) : 0)));
      if (e != cudaSuccess) return e;
      cur ^= 1;
    }
    *in_alt = cur;
    return cudaSuccess;
  }
};

bool merge_types(int kb, int vb) {
  return (kb == 4 && (vb == 0 || vb == 4)) || (kb == 8 && (vb == 0 || vb == 8)) ||
         (kb == 16 && (vb == 0 || vb == 8));
}

size_t merge_workspace(size_t n) { return MergeSort<uint32_t, NoVal, false>::workspace(n); }

}  // namespace

}  // namespace rs

using namespace rs;

extern "C" {

rs_status rs_merge_workspace_bytes(int key_bytes, int val_bytes, size_t n, size_t* bytes) {
  if (!bytes || !merge_types(key_bytes, val_bytes) || n > RS_MAX_N) return RS_ERR_INVALID;
  *bytes = n <= 1 ? 0 : merge_workspace(n);
  return RS_OK;
}

rs_status rs_merge_sort(int key_bytes, int val_bytes, void* keys, void* vals, void* keys_alt,
                        void* vals_alt, size_t n, void* ws, size_t ws_bytes, rs_stream_t stream,
                        int* result_in_alt) {
  if (!result_in_alt || !merge_types(key_bytes, val_bytes) || n > RS_MAX_N)
    return RS_ERR_INVALID;
  *result_in_alt = 0;
  if (n <= 1) return RS_OK;
  auto al = [](const void* p, size_t a) { return reinterpret_cast<uintptr_t>(p) % a == 0; };
  if (!keys || !keys_alt || keys == keys_alt || !al(keys, size_t(key_bytes)) ||
      !al(keys_alt, size_t(key_bytes)))
    return RS_ERR_INVALID;
  if (val_bytes) {
    if (!vals || !vals_alt || vals == vals_alt || !al(vals, size_t(val_bytes)) ||
        !al(vals_alt, size_t(val_bytes)))
      return RS_ERR_INVALID;
  } else if (vals || vals_alt) {
    return RS_ERR_INVALID;
  }
  if (!ws || ws_bytes < merge_workspace(n) || !al(ws, 256)) return RS_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int in_alt = 0;
  cudaError_t e;
  if (key_bytes == 4 && val_bytes == 0)
    e = MergeSort<uint32_t, NoVal, false>::run(keys, vals, keys_alt, vals_alt, n, ws, s, &in_alt);
  else if (key_bytes == 4)
    e = MergeSort<uint32_t, uint32_t, true>::run(keys, vals, keys_alt, vals_alt, n, ws, s,
                                                 &in_alt);
  else if (key_bytes == 8 && val_bytes == 0)
    e = MergeSort<uint64_t, NoVal, false>::run(keys, vals, keys_alt, vals_alt, n, ws, s, &in_alt);
  else if (key_bytes == 8)
    e = MergeSort<uint64_t, uint64_t, true>::run(keys, vals, keys_alt, vals_alt, n, ws, s,
                                                 &in_alt);
  else if (val_bytes == 0)
    e = MergeSort<Key128, NoVal, false>::run(keys, vals, keys_alt, vals_alt, n, ws, s, &in_alt);
  else
    e = MergeSort<Key128, uint64_t, true>::run(keys, vals, keys_alt, vals_alt, n, ws, s, &in_alt);
  if (e != cudaSuccess) return RS_ERR_CUDA;
  *result_in_alt = in_alt;
  return RS_OK;
}

}  // extern "C"
