// Host side of the batched segmented sort (each of the four data types):
// workspace sizing and the launch sequence memset -> k_seg_plan ->
// k_seg_small -> k_seg_hist -> k_seg_persistent, all on the caller's stream
// (capturable in a CUDA graph).
#include <algorithm>

#include "../../include/rs.h"
#include "rs_host.h"
#include "rs_segmented.cuh"

namespace rs {

namespace {

// MINB: resident CTAs per SM the short-segment kernel is compiled for (its
// register budget); PASS_MINB: the same for the pass kernel.
template <class K, int VB, int R, int THREADS, int ITEMS, int CHUNK_TILES, int UNIT,
          int SMALL_ITEMS, int MINB = 4, int PASS_MINB = MINB>
struct SegSort {
  using C = SegKernelCfg<K, VB, R, THREADS, ITEMS, CHUNK_TILES, UNIT, SMALL_ITEMS>;
  static constexpr int PLAN_THREADS = 1024;

  static SegLayout layout(size_t n, size_t nseg, int passes) {
    return seg_layout(n, nseg, passes, R, C::TILE, C::CHUNK);
  }

  static cudaError_t run(void* keys, void* vals, void* keys_alt, void* vals_alt, size_t n,
                         const uint64_t* d_off, size_t nseg, int begin_bit, int end_bit,
                         void* ws, cudaStream_t s, Knobs knobs) {
    const int passes = num_passes(begin_bit, end_bit, R);
    const SegLayout L = layout(n, nseg, passes);
    char* w = static_cast<char*>(ws);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(w);
    cudaError_t e = cudaMemsetAsync(w, 0, L.memset_bytes, s);
    if (e != cudaSuccess) return e;
    k_seg_plan<PLAN_THREADS><<<1, PLAN_THREADS, 0, s>>>(
        d_off, nseg, n, uint32_t(C::SMALL_TILE), uint32_t(C::TILE), uint32_t(C::CHUNK), ctrl,
        reinterpret_cast<uint32_t*>(w + L.small_ids), reinterpret_cast<SegDesc*>(w + L.descs),
        reinterpret_cast<uint32_t*>(w + L.chunk_seg),
        L.tiles_max, L.chunks_max);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // short segments: one CTA each, before the persistent kernel
    auto small = &k_seg_small<K, VB, R, THREADS, SMALL_ITEMS, MINB>;
    using SS = typename C::SS;
    const int occ_small = prepare_kernel(reinterpret_cast<const void*>(small), THREADS, SS::BYTES);
    if (occ_small <= 0) return cudaErrorInvalidConfiguration;
    auto hist = &k_seg_hist<K, R, C::HIST_THREADS, C::MAXP, C::HIST_SLOTS, C::CHUNK, C::TILE,
                            CHUNK_TILES, C::HIST_MINB>;
    const int occ_hist =
        prepare_kernel(reinterpret_cast<const void*>(hist), C::HIST_THREADS, C::HIST_BYTES);
    if (occ_hist <= 0) return cudaErrorInvalidConfiguration;
    auto kern = &k_seg_persistent<K, VB, R, THREADS, ITEMS, CHUNK_TILES, UNIT, PASS_MINB>;
    const int occ = prepare_kernel(reinterpret_cast<const void*>(kern), THREADS, C::BYTES);
    if (occ <= 0) return cudaErrorInvalidConfiguration;
    SegArgs a;
    a.off = d_off;
    a.begin_bit = begin_bit;
    a.end_bit = end_bit;
    a.passes = passes;
    a.ctrl = ctrl;
    a.small_ids = reinterpret_cast<const uint32_t*>(w + L.small_ids);
    a.descs = reinterpret_cast<const SegDesc*>(w + L.descs);
    a.tdesc = reinterpret_cast<TileDesc*>(w + L.tdesc);
    a.chunk_seg = reinterpret_cast<const uint32_t*>(w + L.chunk_seg);
    a.state = reinterpret_cast<uint32_t*>(w + L.state);
    a.counts = reinterpret_cast<uint32_t*>(w + L.counts);
    a.offsets = reinterpret_cast<uint32_t*>(w + L.offsets);
    a.status = reinterpret_cast<uint32_t*>(w + L.status);
    a.tiles_max = L.tiles_max;
    a.nseg = nseg;
    a.knobs = knobs;
    using V = ValT<VB>;
    // grids no larger than the work can be: at most tiles_max pass tiles per
    // pass and chunks_max histogram chunks (bounds the host knows without
    // the plan), so that a small batch does not spread idle CTAs over every
    // SM while other streams' kernels want them
    const size_t sms = size_t(device_info().sms);
    const unsigned grid = unsigned(std::max<size_t>(
        1, std::min<size_t>(sms * occ, size_t(passes) * L.tiles_max)));
    const unsigned grid_hist =
        unsigned(std::max<size_t>(1, std::min<size_t>(sms * occ_hist, L.chunks_max)));
    const unsigned grid_small =
        unsigned(std::max<size_t>(1, std::min<size_t>(nseg, sms * occ_small)));
    prof_before(s);
    small<<<grid_small, THREADS, SS::BYTES, s>>>(static_cast<K*>(keys), static_cast<V*>(vals),
                                                 static_cast<K*>(keys_alt),
                                                 static_cast<V*>(vals_alt), a);
    hist<<<grid_hist, C::HIST_THREADS,
           passes * C::RADIX * C::HIST_SLOTS * 4, s>>>(static_cast<const K*>(keys), a);
    kern<<<grid, THREADS, C::BYTES, s>>>(static_cast<K*>(keys), static_cast<V*>(vals),
                                         static_cast<K*>(keys_alt), static_cast<V*>(vals_alt), a);
    e = cudaGetLastError();
    prof_after(s, RS_KERNEL_SEGMENTED,
               double(n) * (sizeof(K) + passes * 2.0 * (sizeof(K) + VB)));
    return e;
  }
};

// u32 pairs: pass tiles of 256 x 45 keys ranked in half-warp units, two CTAs
// per SM; short segments up to 4096 elements sorted whole by one CTA
using SegU32Pairs = SegSort<uint32_t, 4, 8, 256, 45, 12, 16, 16, 4, 2>;
// u32 keys: 256 x 37 keys in half-warp units, two CTAs per SM; short
// segments up to 4096
using SegU32Keys = SegSort<uint32_t, 0, 8, 256, 37, 16, 16, 16, 4, 2>;
// 64-bit keys and pairs: 256 x 23 elements in half-warp units, two CTAs per
// SM; short segments up to 2048 (pairs: that kernel at three CTAs per SM)
using SegU64Keys = SegSort<uint64_t, 0, 8, 256, 23, 24, 16, 8, 4, 2>;
using SegU64Pairs = SegSort<uint64_t, 8, 8, 256, 23, 24, 16, 8, 3, 2>;

bool seg_types(int kb, int vb) { return (kb == 4 || kb == 8) && (vb == 0 || vb == kb); }

SegLayout seg_layout_for(int kb, int vb, size_t n, size_t nseg, int passes) {
  if (kb == 4) return vb ? SegU32Pairs::layout(n, nseg, passes) : SegU32Keys::layout(n, nseg, passes);
  return vb ? SegU64Pairs::layout(n, nseg, passes) : SegU64Keys::layout(n, nseg, passes);
}

cudaError_t seg_run(int kb, int vb, void* keys, void* vals, void* keys_alt, void* vals_alt,
                    size_t n, const uint64_t* d_off, size_t nseg, int begin_bit, int end_bit,
                    void* ws, cudaStream_t s, Knobs knobs) {
  if (kb == 4 && vb)
    return SegU32Pairs::run(keys, vals, keys_alt, vals_alt, n, d_off, nseg, begin_bit, end_bit,
                            ws, s, knobs);
  if (kb == 4)
    return SegU32Keys::run(keys, vals, keys_alt, vals_alt, n, d_off, nseg, begin_bit, end_bit,
                           ws, s, knobs);
  if (vb)
    return SegU64Pairs::run(keys, vals, keys_alt, vals_alt, n, d_off, nseg, begin_bit, end_bit,
                            ws, s, knobs);
  return SegU64Keys::run(keys, vals, keys_alt, vals_alt, n, d_off, nseg, begin_bit, end_bit, ws,
                         s, knobs);
}

}  // namespace

Knobs knobs_now();

}  // namespace rs

using namespace rs;

extern "C" {

rs_status rs_segmented_workspace_bytes_typed(int key_bytes, int val_bytes, size_t n, size_t n_seg,
                                             int begin_bit, int end_bit, size_t* bytes) {
  if (!bytes || !seg_types(key_bytes, val_bytes)) return RS_ERR_INVALID;
  if (begin_bit < 0 || begin_bit > end_bit || end_bit > 8 * key_bytes) return RS_ERR_INVALID;
  if (n >= (size_t(1) << 40) || n_seg >= (size_t(1) << 31)) return RS_ERR_INVALID;
  *bytes = 0;
  if (n == 0 || n_seg == 0 || begin_bit == end_bit) return RS_OK;
  const SegLayout L =
      seg_layout_for(key_bytes, val_bytes, n, n_seg, num_passes(begin_bit, end_bit, 8));
  if (L.tiles_max >= (size_t(1) << 32)) return RS_ERR_INVALID;
  *bytes = L.total;
  return RS_OK;
}

rs_status rs_segmented_sort(int key_bytes, int val_bytes, void* keys, void* vals, void* keys_alt,
                            void* vals_alt, size_t n, const uint64_t* d_offsets, size_t n_seg,
                            int begin_bit, int end_bit, void* ws, size_t ws_bytes,
                            rs_stream_t stream, int* result_in_alt) {
  if (!result_in_alt) return RS_ERR_INVALID;
  *result_in_alt = 0;
  size_t need = 0;
  rs_status st = rs_segmented_workspace_bytes_typed(key_bytes, val_bytes, n, n_seg, begin_bit,
                                                    end_bit, &need);
  if (st != RS_OK) return st;
  if (n == 0 || n_seg == 0 || begin_bit == end_bit) return RS_OK;
  if (!keys || !keys_alt || !d_offsets || keys == keys_alt) return RS_ERR_INVALID;
  if ((val_bytes != 0) != (vals != nullptr && vals_alt != nullptr)) return RS_ERR_INVALID;
  if (val_bytes == 0 && (vals || vals_alt)) return RS_ERR_INVALID;
  if (val_bytes && vals == vals_alt) return RS_ERR_INVALID;
  auto al = [](const void* p, size_t a) { return reinterpret_cast<uintptr_t>(p) % a == 0; };
  if (!al(keys, key_bytes) || !al(keys_alt, key_bytes) || !al(d_offsets, 8)) return RS_ERR_INVALID;
  if (val_bytes && (!al(vals, val_bytes) || !al(vals_alt, val_bytes))) return RS_ERR_INVALID;
  if (!ws || ws_bytes < need || !al(ws, 256)) return RS_ERR_WORKSPACE;
  const int passes = num_passes(begin_bit, end_bit, 8);
  const cudaError_t e = seg_run(key_bytes, val_bytes, keys, vals, keys_alt, vals_alt, n,
                                d_offsets, n_seg, begin_bit, end_bit, ws,
                                reinterpret_cast<cudaStream_t>(stream), knobs_now());
  if (e != cudaSuccess) return RS_ERR_CUDA;
  *result_in_alt = passes & 1;
  return RS_OK;
}


rs_status rs_segmented_workspace_bytes(size_t n, size_t n_seg, int begin_bit, int end_bit,
                                       size_t* bytes) {
  return rs_segmented_workspace_bytes_typed(4, 4, n, n_seg, begin_bit, end_bit, bytes);
}

rs_status rs_segmented_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt,
                                  uint32_t* vals_alt, size_t n, const uint64_t* d_offsets,
                                  size_t n_seg, int begin_bit, int end_bit, void* ws,
                                  size_t ws_bytes, rs_stream_t stream, int* result_in_alt) {
  if (n > 0 && n_seg > 0 && begin_bit != end_bit && (!vals || !vals_alt)) return RS_ERR_INVALID;
  return rs_segmented_sort(4, 4, keys, vals, keys_alt, vals_alt, n, d_offsets, n_seg, begin_bit,
                           end_bit, ws, ws_bytes, stream, result_in_alt);
}

}  // extern "C"
