// Host/device shared definitions of the rs library: workspace layout, the
// control block the kernels communicate through, and kernel arguments.
#pragma once

#include <cstddef>
#include <cstdint>

namespace rs {

// Look-back status word of one (tile, digit): 2 flag bits + a 30-bit count.
constexpr uint32_t kFlagShift = 30;
constexpr uint32_t kFlagAgg = 1u << kFlagShift;  // count of this tile only
constexpr uint32_t kFlagInc = 2u << kFlagShift;  // count of all tiles up to and including this one
constexpr uint32_t kFlagErr = 3u << kFlagShift;  // this tile gave up; successors give up too
constexpr uint32_t kFlagMask = 3u << kFlagShift;
constexpr uint32_t kValueMask = (1u << kFlagShift) - 1u;

constexpr int kMaxPasses = 16;  // 64-bit keys at 4-bit digits

// Look-back groups: every kGroupTiles consecutive tiles of a pass also sum
// their digit counts into one group word per digit (count in the low 24 bits,
// number of tiles that added in the high 8), and the group's last tile
// publishes the inclusive prefix through the group's end.
constexpr int kGroupTiles = 32;
constexpr uint32_t kGroupOne = 1u << 24;
constexpr uint32_t kGroupCountMask = kGroupOne - 1u;

// Device status codes (the values of rs_status).
constexpr uint32_t kDevOk = 0;
constexpr uint32_t kDevTimeout = 4;
constexpr uint32_t kDevIndex = 7;

// The first 256 bytes of every workspace.
struct Ctrl {
  uint32_t error;       // 0, or the first device status code reported
  uint32_t error_info;  // tile (or pass) that reported it
  uint32_t hist_ticket; // upsweep CTAs that have finished
  uint32_t exec_mask;   // bit p: pass p moves the data (written by the upsweep's last CTA)
  uint32_t tile_counter[kMaxPasses];  // dynamic tile ids of each pass
  uint32_t grid_bar;    // arrivals at the grid barriers of a one-launch sort
  // Record of the call for rs_workspace_stats (zeroed with the rest of the
  // block at the start of every multi-launch sort).  Times are %globaltimer
  // nanoseconds after t0, the upsweep's start.
  uint32_t stat_n;       // elements sorted
  uint32_t stat_shape;   // key bytes | value bytes << 8 | passes << 16 | 1 << 24 (recorded)
  uint32_t t0_lo, t0_hi; // %globaltimer when the upsweep started
  uint32_t t_upsweep;    // upsweep's last CTA done
  uint32_t t_pass[kMaxPasses][2];  // per pass: first tile taken, last CTA done
  uint32_t reserved[64 - 5 - kMaxPasses - 5 - 2 * kMaxPasses];
};
static_assert(sizeof(Ctrl) == 256, "Ctrl must be 256 bytes");

// Test-only fault injection and the bound on every device-side wait.
struct Knobs {
  uint64_t timeout_ns;     // a look-back wait gives up after this long
  int32_t drop_tile;       // this tile never publishes its status (-1: off)
  int32_t drop_pass;       // ... in this pass
  uint64_t* trace;         // device [trace_tiles][16] phase timestamps (ns) and counters, or null
  uint32_t trace_tiles;    // tiles 0 .. trace_tiles-1 of trace_pass are recorded
  int32_t trace_pass;
  int32_t lb_small;        // test-only: look-back windows of 8 instead of 32 words
  int32_t dbg_bad_tile;    // debug builds only: this tile of pass 0 computes scatter
                           // indices past the array, which the bounds checks drop (-1: off)
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Order-preserving key transform for signed integers, IEEE-754 floats and
// descending order.  The digit passes order T(k) = k ^ c ^ (f & top(k)) as
// unsigned integers, where top(k) is all ones when the top bit of k is set;
// the inverse is T^-1(t) = t ^ c ^ (f & top(t ^ g)).  on == 0: identity.
//   unsigned: c = 0 (or all ones descending), f = g = 0
//   signed:   c = sign bit (descending: all bits but the sign), f = g = 0
//   float:    c as signed, f = all bits but the sign, g = sign bit ascending,
//             0 descending (negative values are reversed, positive ones get
//             the sign bit: -NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN)
template <class K>
struct KeyXf {
  K c, f, g;
  uint32_t on;
};

template <class K>
__host__ __device__ __forceinline__ K top_ones(K k) {
  return K(0) - (k >> (8 * sizeof(K) - 1));
}

template <class K>
__host__ __device__ __forceinline__ K xf_fwd(K k, const KeyXf<K>& x) {
  return k ^ x.c ^ (x.f & top_ones(k));
}

template <class K>
__host__ __device__ __forceinline__ K xf_inv(K t, const KeyXf<K>& x) {
  return t ^ x.c ^ (x.f & top_ones(K(t ^ x.g)));
}

// kind: 0 unsigned, 1 signed (two's complement), 2 IEEE-754 float.
template <class K>
inline KeyXf<K> make_key_xf(int kind, int descending) {
  const K sign = K(1) << (8 * sizeof(K) - 1);
  KeyXf<K> x{};
  if (kind == 0) {
    x.c = descending ? K(~K(0)) : K(0);
  } else {
    x.c = descending ? K(~sign) : sign;
    if (kind == 2) {
      x.f = K(~sign);
      x.g = descending ? K(0) : sign;
    }
  }
  x.on = (x.c | x.f | x.g) != K(0) ? 1u : 0u;
  return x;
}

// Word of (tile or group t, digit d) in a [t/4][radix][4] look-back array.
template <int RADIX>
__host__ __device__ __forceinline__ size_t lb_index(uint32_t t, uint32_t d) {
  return ((size_t(t >> 2) * RADIX + d) << 2) | (t & 3u);
}

// Workspace of one onesweep sort with `passes` digit passes, radix 2^r and
// `tiles` tiles per pass:
//   [0, 256)            Ctrl
//   counts   u32 [passes][radix]    digit histograms (atomics; zeroed per call)
//   offsets  u32 [passes][radix]    exclusive scans of the histograms
//   status   u32 [passes][tiles/4][radix][4]   look-back words of the tiles
//   gagg     u32 [passes][groups/4][radix][4]  group digit counts (+ tiles added)
//   ginc     u32 [passes][groups/4][radix][4]  group inclusive prefixes
// Four consecutive tiles (groups) of one digit are adjacent, so a look-back
// thread fetches four of them with one 16-byte load, and a warp's loads (32
// digits) are one contiguous 512-byte block.  status, gagg and ginc are one
// range, zeroed by the upsweep; tile and group counts are rounded up to 4.
struct Layout {
  size_t counts, offsets, status, gagg, ginc, status_bytes, total, memset_bytes;
  size_t tiles, groups;
};

inline Layout onesweep_layout(int passes, int radix_bits, size_t tiles) {
  Layout L;
  const size_t radix = size_t(1) << radix_bits;
  L.tiles = align_up(tiles, 4);
  L.groups = align_up((tiles + kGroupTiles - 1) / kGroupTiles, 4);
  L.counts = 256;
  L.offsets = align_up(L.counts + size_t(passes) * radix * 4, 256);
  L.status = align_up(L.offsets + size_t(passes) * radix * 4, 256);
  L.gagg = L.status + size_t(passes) * L.tiles * radix * 4;
  L.ginc = L.gagg + size_t(passes) * L.groups * radix * 4;
  L.status_bytes = align_up(L.ginc + size_t(passes) * L.groups * radix * 4 - L.status, 256);
  L.total = L.status + L.status_bytes;
  L.memset_bytes = L.offsets;  // Ctrl + counts
  return L;
}

}  // namespace rs
