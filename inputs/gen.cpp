// Seeded synthetic inputs for the sort workloads of the comparison study
// (arXiv 1511.03404, Sec. 3 and Sec. 4): six key distributions (uniform,
// Gaussian, zero, bucket, sorted, sorted descending) over 32- and 64-bit
// keys, drawn from a Mersenne Twister, plus the 16-bit-entropy keys, the
// segment-length law of the batched workload and raw engine outputs.
//
// This module holds no part of the radix-sort method.  It is shared by the
// tests, the oracle's checks and the benchmark, and by nothing else.  Only
// raw engine outputs of std::mt19937 / std::mt19937_64 are used: the C++
// standard fixes those bit for bit, whereas std::*_distribution and
// std::shuffle are implementation-defined.  The two "sorted" distributions
// order a uniform draw with std::sort, a library comparison sort.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <functional>
#include <random>

namespace {

enum Dist : int {
  DIST_UNIFORM = 0,
  DIST_GAUSSIAN = 1,
  DIST_ZERO = 2,
  DIST_SORTED = 3,
  DIST_SORTED_DESC = 4,
  DIST_BUCKET = 5,
  DIST_ENTROPY16 = 6,
  DIST_COUNT = 7
};

constexpr uint32_t kBuckets = 1u << 13;

// Chunk owning element i when n elements are split into kBuckets contiguous,
// balanced chunks (any n, including n < kBuckets).
inline uint32_t chunk_of(uint64_t i, uint64_t n) {
  return (uint32_t)((i * (uint64_t)kBuckets) / n);
}

template <class Engine>
void bucket_permutation(Engine& mt, uint32_t* perm) {
  for (uint32_t i = 0; i < kBuckets; ++i) perm[i] = i;
  // Fisher-Yates, high index first, j drawn as engine() mod (i+1).
  for (uint32_t i = kBuckets - 1; i >= 1; --i) {
    uint32_t j = (uint32_t)(mt() % (uint64_t)(i + 1));
    std::swap(perm[i], perm[j]);
  }
}

}  // namespace

extern "C" {

int rsgen_num_dists(void) { return DIST_COUNT; }

// Raw engine outputs, in draw order.
int rsgen_mt19937(uint32_t seed, uint64_t count, uint32_t* out) {
  if (!out && count) return 1;
  std::mt19937 mt(seed);
  for (uint64_t i = 0; i < count; ++i) out[i] = (uint32_t)mt();
  return 0;
}

int rsgen_mt19937_64(uint64_t seed, uint64_t count, uint64_t* out) {
  if (!out && count) return 1;
  std::mt19937_64 mt(seed);
  for (uint64_t i = 0; i < count; ++i) out[i] = (uint64_t)mt();
  return 0;
}

// 32-bit keys of distribution `dist`, seeded engine std::mt19937(seed).
int rsgen_keys_u32(int dist, uint64_t n, uint32_t seed, uint32_t* out) {
  if (!out && n) return 1;
  std::mt19937 mt(seed);
  switch (dist) {
    case DIST_UNIFORM:
      for (uint64_t i = 0; i < n; ++i) out[i] = (uint32_t)mt();
      return 0;
    case DIST_GAUSSIAN:
      // floor of the mean of four consecutive uniform draws
      for (uint64_t i = 0; i < n; ++i) {
        uint64_t a = mt(), b = mt(), c = mt(), d = mt();
        out[i] = (uint32_t)((a + b + c + d) >> 2);
      }
      return 0;
    case DIST_ZERO:
      for (uint64_t i = 0; i < n; ++i) out[i] = 0u;
      return 0;
    case DIST_SORTED:
    case DIST_SORTED_DESC:
      for (uint64_t i = 0; i < n; ++i) out[i] = (uint32_t)mt();
      if (dist == DIST_SORTED)
        std::sort(out, out + n);
      else
        std::sort(out, out + n, std::greater<uint32_t>());
      return 0;
    case DIST_BUCKET: {
      uint32_t perm[kBuckets];
      bucket_permutation(mt, perm);
      for (uint64_t i = 0; i < n; ++i) {
        uint32_t b = perm[chunk_of(i, n)];
        out[i] = (b << 19) | ((uint32_t)mt() >> 13);
      }
      return 0;
    }
    case DIST_ENTROPY16:
      for (uint64_t i = 0; i < n; ++i) out[i] = (uint32_t)mt() & 0xFFFFu;
      return 0;
    default:
      return 2;
  }
}

// 64-bit keys of distribution `dist`, seeded engine std::mt19937_64(seed).
int rsgen_keys_u64(int dist, uint64_t n, uint64_t seed, uint64_t* out) {
  if (!out && n) return 1;
  std::mt19937_64 mt(seed);
  switch (dist) {
    case DIST_UNIFORM:
      for (uint64_t i = 0; i < n; ++i) out[i] = (uint64_t)mt();
      return 0;
    case DIST_GAUSSIAN:
      // exact floor of the mean of four draws without 66-bit intermediates
      for (uint64_t i = 0; i < n; ++i) {
        uint64_t a = mt(), b = mt(), c = mt(), d = mt();
        out[i] = (a >> 2) + (b >> 2) + (c >> 2) + (d >> 2) +
                 (((a & 3) + (b & 3) + (c & 3) + (d & 3)) >> 2);
      }
      return 0;
    case DIST_ZERO:
      for (uint64_t i = 0; i < n; ++i) out[i] = 0ull;
      return 0;
    case DIST_SORTED:
    case DIST_SORTED_DESC:
      for (uint64_t i = 0; i < n; ++i) out[i] = (uint64_t)mt();
      if (dist == DIST_SORTED)
        std::sort(out, out + n);
      else
        std::sort(out, out + n, std::greater<uint64_t>());
      return 0;
    case DIST_BUCKET: {
      uint32_t perm[kBuckets];
      bucket_permutation(mt, perm);
      for (uint64_t i = 0; i < n; ++i) {
        uint64_t b = perm[chunk_of(i, n)];
        out[i] = (b << 51) | ((uint64_t)mt() >> 13);
      }
      return 0;
    }
    case DIST_ENTROPY16:
      for (uint64_t i = 0; i < n; ++i) out[i] = (uint64_t)mt() & 0xFFFFull;
      return 0;
    default:
      return 2;
  }
}

// Segment lengths of the batched workload: L = min(2^max_log2,
// floor(2^(max_log2 * u))) with u = mt() * 2^-32, so 1 <= L <= 2^max_log2 and
// log2 L is uniform.
int rsgen_segment_lengths(uint64_t nseg, uint32_t seed, uint32_t max_log2,
                          uint64_t* out) {
  if (!out && nseg) return 1;
  if (max_log2 > 40) return 2;
  std::mt19937 mt(seed);
  const uint64_t cap = 1ull << max_log2;
  for (uint64_t s = 0; s < nseg; ++s) {
    double u = (double)(uint32_t)mt() * (1.0 / 4294967296.0);
    double len = std::floor(std::exp2((double)max_log2 * u));
    uint64_t L = (uint64_t)len;
    if (L < 1) L = 1;
    if (L > cap) L = cap;
    out[s] = L;
  }
  return 0;
}

}  // extern "C"
