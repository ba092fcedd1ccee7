// Sample sort (Sec. 2.7) as an MSD partition front end for 32-bit key-value
// pairs, after the regular-sampling variant of Dehne et al.:
//   1. blocks of kSampleBlock elements, each sorted stably (one batched
//      segmented sort: every block is a short segment, one CTA each);
//   2. s equidistant samples from each sorted block (k_ss_sample);
//   3. the samples sorted (rs_sort) and B - 1 equidistant splitters taken
//      (k_ss_splitters);
//   4. per block, the boundary of every bucket found by binary search in the
//      sorted block, counts[q][block] (k_ss_count); one exclusive scan of the
//      bucket-major counts gives every run's destination (k_scan_*);
//   5. each block's bucket runs copied to their destinations (k_ss_scatter),
//      so bucket q holds, block after block, every key x with
//      s[q-1] < x <= s[q];
//   6. rs_sample_sort_pairs_u32 then sorts every bucket (segmented sort).
// Everything runs on the caller's stream; nothing waits on another CTA.
#include <algorithm>

#include "../../include/rs.h"
#include "rs_host.h"
#include "rs_kernels.cuh"

namespace rs {

namespace {

constexpr int kSampleBlock = 4096;  // one short segment of the segmented sort
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanChunk = kScanThreads * kScanItems;
constexpr int kMaxBuckets = 4096;
constexpr int kMaxSamples = 4096;

// Segment offsets of the blocks: off[i] = min(i * block, n).
__global__ void k_ss_block_offsets(uint64_t* off, uint64_t nblk, uint64_t n) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i <= nblk;
       i += uint64_t(gridDim.x) * blockDim.x)
    if (dbg_ok(i, nblk + 1, kSiteSampleOff)) off[i] = min(i * kSampleBlock, n);
}

// sample[i * s + j] = block i's element floor(j * L_i / s).
__global__ void k_ss_sample(const uint32_t* __restrict__ keys, uint64_t n, uint32_t s,
                            uint64_t m, uint32_t* __restrict__ sample) {
  for (uint64_t t = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; t < m;
       t += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t blk = t / s, j = t % s;
    const uint64_t base = blk * kSampleBlock;
    const uint64_t len = min(uint64_t(kSampleBlock), n - base);
    if (dbg_ok(t, m, kSiteSampleSample)) sample[t] = keys[base + (j * len) / s];
  }
}

// splitter q = sorted_sample[floor((q + 1) * m / buckets)], q < buckets - 1.
__global__ void k_ss_splitters(const uint32_t* __restrict__ sorted, uint64_t m, uint32_t buckets,
                               uint32_t* __restrict__ spl) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q + 1 < buckets;
       q += gridDim.x * blockDim.x)
    if (dbg_ok(q, buckets - 1u, kSiteSampleSplitter)) spl[q] = sorted[((uint64_t(q) + 1) * m) / buckets];
}

// Number of elements <= x in the sorted run a[0 .. len).
__device__ __forceinline__ uint32_t upper_bound_u32(const uint32_t* a, uint32_t len, uint32_t x) {
  uint32_t lo = 0, hi = len;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Bucket boundaries of one sorted block in shared memory: e[q] = elements
// <= s[q] for q < B - 1, e[B - 1] = len; bucket q is [e[q-1], e[q]).
__device__ __forceinline__ void block_bounds(const uint32_t* s_blk, uint32_t len,
                                             const uint32_t* __restrict__ spl, uint32_t buckets,
                                             uint32_t* s_e) {
  for (uint32_t q = threadIdx.x; q < buckets; q += blockDim.x)
    s_e[q] = q + 1 < buckets ? upper_bound_u32(s_blk, len, spl[q]) : len;
}

// One CTA per block: counts[q * nblk + blk] = elements of bucket q.
__global__ void __launch_bounds__(1024) k_ss_count(const uint32_t* __restrict__ keys, uint64_t n,
                                                   uint64_t nblk,
                                                   const uint32_t* __restrict__ spl,
                                                   uint32_t buckets,
                                                   uint32_t* __restrict__ counts) {
  __shared__ uint32_t s_blk[kSampleBlock];
  __shared__ uint32_t s_e[kMaxBuckets];
  const uint64_t blk = blockIdx.x;
  const uint64_t base = blk * kSampleBlock;
  const uint32_t len = uint32_t(min(uint64_t(kSampleBlock), n - base));
  for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) s_blk[i] = keys[base + i];
  __syncthreads();
  block_bounds(s_blk, len, spl, buckets, s_e);
  __syncthreads();
  for (uint32_t q = threadIdx.x; q < buckets; q += blockDim.x)
    if (dbg_ok(uint64_t(q) * nblk + blk, uint64_t(buckets) * nblk, kSiteSampleCount))
      counts[uint64_t(q) * nblk + blk] = s_e[q] - (q ? s_e[q - 1] : 0u);
}

// One CTA per block: element i of bucket q's run goes to
// dest[q * nblk + blk] + (i - e[q-1]).
__global__ void __launch_bounds__(1024) k_ss_scatter(const uint32_t* __restrict__ keys,
                                                     const uint32_t* __restrict__ vals,
                                                     uint32_t* __restrict__ kout,
                                                     uint32_t* __restrict__ vout, uint64_t n,
                                                     uint64_t nblk,
                                                     const uint32_t* __restrict__ spl,
                                                     uint32_t buckets,
                                                     const uint32_t* __restrict__ dest) {
  __shared__ uint32_t s_blk[kSampleBlock];
  __shared__ uint32_t s_e[kMaxBuckets];
  const uint64_t blk = blockIdx.x;
  const uint64_t base = blk * kSampleBlock;
  const uint32_t len = uint32_t(min(uint64_t(kSampleBlock), n - base));
  for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) s_blk[i] = keys[base + i];
  __syncthreads();
  block_bounds(s_blk, len, spl, buckets, s_e);
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) {
    // q = the number of boundaries e[q] <= i (the bucket whose run holds i)
    uint32_t lo = 0, hi = buckets - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (s_e[mid] <= i) lo = mid + 1;
      else hi = mid;
    }
    const uint32_t q = lo;
    const uint64_t d = uint64_t(dest[uint64_t(q) * nblk + blk]) + (i - (q ? s_e[q - 1] : 0u));
    if (!dbg_ok(d, n, kSiteSampleOut)) continue;
    kout[d] = s_blk[i];
    vout[d] = vals[base + i];
  }
}

// Exclusive scan of a u32 array in place: chunk sums, a one-CTA scan of
// the chunk sums, then each chunk rescanned with its prefix.
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ a,
                                                              uint64_t m,
                                                              uint32_t* __restrict__ part) {
  __shared__ uint32_t s_tot[32];
  const uint64_t base = uint64_t(blockIdx.x) * kScanChunk;
  uint32_t sum = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const uint64_t i = base + uint64_t(j) * kScanThreads + threadIdx.x;
    if (i < m) sum += a[i];
  }
  const uint32_t ex = block_exclusive_scan<kScanThreads>(sum, s_tot);
  if (threadIdx.x == kScanThreads - 1) part[blockIdx.x] = ex + sum;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_partials(uint32_t* __restrict__ part,
                                                                uint32_t count) {
  __shared__ uint32_t s_tot[32];
  __shared__ uint32_t s_carry;
  if (threadIdx.x == 0) s_carry = 0u;
  __syncthreads();
  for (uint32_t b = 0; b < count; b += kScanThreads) {
    const uint32_t i = b + threadIdx.x;
    const uint32_t x = i < count ? part[i] : 0u;
    const uint32_t ex = block_exclusive_scan<kScanThreads>(x, s_tot);
    const uint32_t carry = s_carry;
    if (i < count) part[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) s_carry = carry + ex + x;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(uint32_t* __restrict__ a, uint64_t m,
                                                            const uint32_t* __restrict__ part) {
  __shared__ uint32_t s_tot[32];
  const uint64_t base = uint64_t(blockIdx.x) * kScanChunk + uint64_t(threadIdx.x) * kScanItems;
  uint32_t x[kScanItems];
  uint32_t sum = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const uint64_t i = base + j;
    x[j] = i < m ? a[i] : 0u;
    sum += x[j];
  }
  uint32_t run = block_exclusive_scan<kScanThreads>(sum, s_tot) + part[blockIdx.x];
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const uint64_t i = base + j;
    if (i < m) a[i] = run;
    run += x[j];
  }
}

// Bucket offsets for the caller and the bucket sort: off[q] = dest[q * nblk]
// (the first block's run of bucket q), off[B] = n.
__global__ void k_ss_bucket_offsets(const uint32_t* __restrict__ dest, uint64_t nblk,
                                    uint32_t buckets, uint64_t n, uint64_t* __restrict__ off) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q <= buckets;
       q += gridDim.x * blockDim.x)
    if (dbg_ok(q, uint64_t(buckets) + 1, kSiteSampleBucket))
      off[q] = q < buckets ? uint64_t(dest[uint64_t(q) * nblk]) : n;
}

struct SampleLayout {
  size_t blk_off, seg_ws, seg_bytes, sample, sample_alt, sort_ws, sort_bytes, spl, counts, part,
      total;
  uint64_t nblk, m, parts;
};

bool sample_layout(size_t n, int samples, int buckets, SampleLayout* L) {
  L->nblk = (n + kSampleBlock - 1) / kSampleBlock;
  L->m = L->nblk * uint64_t(samples);
  const uint64_t cells = L->nblk * uint64_t(buckets);
  L->parts = (cells + kScanChunk - 1) / kScanChunk;
  if (L->m > RS_MAX_N || cells >= (uint64_t(1) << 32)) return false;
  size_t seg_a = 0, seg_b = 0;
  if (rs_segmented_workspace_bytes(n, L->nblk, 0, 32, &seg_a) != RS_OK) return false;
  if (rs_segmented_workspace_bytes(n, size_t(buckets), 0, 32, &seg_b) != RS_OK) return false;
  L->seg_bytes = std::max(seg_a, seg_b);
  if (rs_workspace_bytes(4, 0, L->m, 0, 32, nullptr, &L->sort_bytes) != RS_OK) return false;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes, 256);
    return at;
  };
  L->blk_off = take((L->nblk + 1) * 8);
  L->seg_ws = take(L->seg_bytes);
  L->sample = take(L->m * 4);
  L->sample_alt = take(L->m * 4);
  L->sort_ws = take(L->sort_bytes);
  L->spl = take(size_t(buckets) * 4);
  L->counts = take(cells * 4);
  L->part = take(std::max<uint64_t>(L->parts, 1) * 4);
  L->total = o;
  return true;
}

unsigned grid_for(uint64_t work, int threads) {
  const uint64_t g = (work + threads - 1) / threads;
  const uint64_t cap = uint64_t(device_info().sms) * 8;
  return unsigned(std::max<uint64_t>(1, std::min(g, cap)));
}

rs_status check_args(size_t n, int samples, int buckets) {
  if (n > RS_MAX_N || samples < 1 || samples > kMaxSamples || buckets < 2 ||
      buckets > kMaxBuckets)
    return RS_ERR_INVALID;
  return RS_OK;
}

// Steps 1-5.  keys / vals are sorted block-wise in place (they are the
// segmented sort's primary buffers); the partition lands in kout / vout.
rs_status partition(uint32_t* keys, uint32_t* vals, uint32_t* kout, uint32_t* vout, size_t n,
                    int samples, int buckets, uint64_t* d_off, uint32_t* d_spl, char* w,
                    const SampleLayout& L, cudaStream_t s) {
  auto* blk_off = reinterpret_cast<uint64_t*>(w + L.blk_off);
  k_ss_block_offsets<<<grid_for(L.nblk + 1, 256), 256, 0, s>>>(blk_off, L.nblk, n);
  if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
  int in_alt = 0;
  rs_status st = rs_segmented_sort_pairs(keys, vals, kout, vout, n, blk_off, L.nblk, 0, 32,
                                         w + L.seg_ws, L.seg_bytes,
                                         reinterpret_cast<rs_stream_t>(s), &in_alt);
  if (st != RS_OK) return st;
  if (in_alt) return RS_ERR_INVALID;  // 4 passes over 32 bits: the blocks are sorted in place
  const uint32_t* bk = keys;          // the block-sorted pairs
  const uint32_t* bv = vals;
  auto* sample = reinterpret_cast<uint32_t*>(w + L.sample);
  auto* sample_alt = reinterpret_cast<uint32_t*>(w + L.sample_alt);
  k_ss_sample<<<grid_for(L.m, 256), 256, 0, s>>>(bk, n, uint32_t(samples), L.m, sample);
  if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
  int s_alt = 0;
  st = rs_sort(4, 0, sample, nullptr, sample_alt, nullptr, L.m, 0, 32, nullptr, w + L.sort_ws,
               L.sort_bytes, reinterpret_cast<rs_stream_t>(s), &s_alt);
  if (st != RS_OK) return st;
  auto* spl = reinterpret_cast<uint32_t*>(w + L.spl);
  k_ss_splitters<<<grid_for(buckets, 256), 256, 0, s>>>(s_alt ? sample_alt : sample, L.m,
                                                        uint32_t(buckets), spl);
  auto* counts = reinterpret_cast<uint32_t*>(w + L.counts);
  auto* part = reinterpret_cast<uint32_t*>(w + L.part);
  const uint64_t cells = L.nblk * uint64_t(buckets);
  prof_before(s);
  k_ss_count<<<unsigned(L.nblk), 1024, 0, s>>>(bk, n, L.nblk, spl, uint32_t(buckets), counts);
  prof_after(s, RS_KERNEL_SAMPLE, double(n) * 4.0);
  k_scan_reduce<<<unsigned(L.parts), kScanThreads, 0, s>>>(counts, cells, part);
  k_scan_partials<<<1, kScanThreads, 0, s>>>(part, uint32_t(L.parts));
  k_scan_down<<<unsigned(L.parts), kScanThreads, 0, s>>>(counts, cells, part);
  prof_before(s);
  k_ss_scatter<<<unsigned(L.nblk), 1024, 0, s>>>(bk, bv, kout, vout, n, L.nblk, spl,
                                                 uint32_t(buckets), counts);
  prof_after(s, RS_KERNEL_SAMPLE, 2.0 * double(n) * 8.0);
  k_ss_bucket_offsets<<<grid_for(uint64_t(buckets) + 1, 256), 256, 0, s>>>(
      counts, L.nblk, uint32_t(buckets), n, d_off);
  if (d_spl && cudaMemcpyAsync(d_spl, spl, size_t(buckets - 1) * 4, cudaMemcpyDeviceToDevice,
                               s) != cudaSuccess)
    return RS_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
  return RS_OK;
}

}  // namespace

}  // namespace rs

using namespace rs;

extern "C" {

rs_status rs_sample_workspace_bytes(size_t n, int samples, int buckets, size_t* bytes) {
  if (!bytes) return RS_ERR_INVALID;
  *bytes = 0;
  rs_status st = check_args(n, samples, buckets);
  if (st != RS_OK) return st;
  if (n == 0) return RS_OK;
  SampleLayout L;
  if (!sample_layout(n, samples, buckets, &L)) return RS_ERR_INVALID;
  *bytes = L.total;
  return RS_OK;
}

rs_status rs_sample_partition_pairs_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_out,
                                        uint32_t* vals_out, size_t n, int samples, int buckets,
                                        uint64_t* d_bucket_offsets, uint32_t* d_splitters,
                                        void* ws, size_t ws_bytes, rs_stream_t stream) {
  rs_status st = check_args(n, samples, buckets);
  if (st != RS_OK) return st;
  if (!d_bucket_offsets) return RS_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (n == 0) {
    if (cudaMemsetAsync(d_bucket_offsets, 0, size_t(buckets + 1) * 8, s) != cudaSuccess)
      return RS_ERR_CUDA;
    return RS_OK;
  }
  if (!keys || !vals || !keys_out || !vals_out || keys == keys_out || vals == vals_out)
    return RS_ERR_INVALID;
  auto al = [](const void* p, size_t a) { return reinterpret_cast<uintptr_t>(p) % a == 0; };
  if (!al(keys, 4) || !al(vals, 4) || !al(keys_out, 4) || !al(vals_out, 4) ||
      !al(d_bucket_offsets, 8) || (d_splitters && !al(d_splitters, 4)))
    return RS_ERR_INVALID;
  SampleLayout L;
  if (!sample_layout(n, samples, buckets, &L)) return RS_ERR_INVALID;
  if (!ws || ws_bytes < L.total || !al(ws, 256)) return RS_ERR_WORKSPACE;
  return partition(keys, vals, keys_out, vals_out, n, samples, buckets, d_bucket_offsets,
                   d_splitters, static_cast<char*>(ws), L, s);
}

rs_status rs_sample_sort_pairs_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_out,
                                   uint32_t* vals_out, size_t n, int samples, int buckets,
                                   uint64_t* d_bucket_offsets, void* ws, size_t ws_bytes,
                                   rs_stream_t stream, int* result_in_alt) {
  if (!result_in_alt) return RS_ERR_INVALID;
  *result_in_alt = 0;
  rs_status st = rs_sample_partition_pairs_u32(keys, vals, keys_out, vals_out, n, samples,
                                               buckets, d_bucket_offsets, nullptr, ws, ws_bytes,
                                               stream);
  if (st != RS_OK || n == 0) {
    if (st == RS_OK) *result_in_alt = 1;  // nothing to sort: keys_out is (empty) output
    return st;
  }
  SampleLayout L;
  sample_layout(n, samples, buckets, &L);
  char* w = static_cast<char*>(ws);
  int in_alt = 0;
  st = rs_segmented_sort_pairs(keys_out, vals_out, keys, vals, n, d_bucket_offsets,
                               size_t(buckets), 0, 32, w + L.seg_ws, L.seg_bytes, stream, &in_alt);
  if (st != RS_OK) return st;
  *result_in_alt = in_alt ? 0 : 1;  // relative to (keys, keys_out)
  return RS_OK;
}

}  // extern "C"
