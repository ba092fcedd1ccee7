// rs_sort_keys_u32_noalloc: the 32-bit key sort with its workspace taken
// from a fixed array in device memory that the library itself owns, for
// callers that cannot allocate device memory.
//
// The array below is static device memory of this library: the CUDA runtime
// creates it on every GPU where the library's module is loaded and keeps it
// until the process exits.  In host code its name does not denote a device
// address, so the address is fetched once per device with
// cudaGetSymbolAddress (while that device is current) and handed to the
// kernels as their workspace pointer.  All calls on a device share the one
// array; the sort clears everything in it that must start at zero, and calls
// whose work overlaps on the GPU (for example on two streams) would race on it.
#include <mutex>

#include "../../include/rs.h"
#include "rs_host.h"

namespace {

// Workspace of a sort of up to RS_NOALLOC_MAX_N keys: control block, digit
// counts and offsets, one look-back word per (pass, tile, digit) and two per
// (pass, group of tiles, digit): about 8.5 MiB at 2^23 keys with 4096-key
// tiles.  A tile shape whose workspace would not fit is not used here (see
// pick_config).
constexpr size_t kScratchBytes = RS_NOALLOC_SCRATCH_BYTES;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device (set up on first use).
rs_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RS_ERR_CUDA;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return RS_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return RS_OK;
}

// The configuration of a sort of n keys over [begin_bit, end_bit) whose
// workspace fits the array: the library's own choice when it fits, else the
// compiled variant with the smallest workspace for n (every variant gives the
// same sorted result).  RS_ERR_INVALID when none fits.
rs_status pick_config(size_t n, int begin_bit, int end_bit, rs_config* cfg) {
  *cfg = rs_config{0, -1, RS_KEY_UNSIGNED, 0};
  size_t need = 0;
  rs_status st = rs_workspace_bytes(4, 0, n, begin_bit, end_bit, nullptr, &need);
  if (st != RS_OK) return st;
  if (need <= kScratchBytes) return RS_OK;
  size_t best = ~size_t(0);
  const int count = rs_num_variants(4, 0);
  for (int i = 0; i < count; ++i) {
    rs_config c{0, i, RS_KEY_UNSIGNED, 0};
    if (rs_workspace_bytes(4, 0, n, begin_bit, end_bit, &c, &need) == RS_OK && need < best) {
      best = need;
      cfg->variant = i;
    }
  }
  return best <= kScratchBytes ? RS_OK : RS_ERR_INVALID;
}

}  // namespace

extern "C" {

rs_status rs_sort_keys_u32_noalloc(uint32_t* keys, uint32_t* keys_alt, size_t n, int begin_bit,
                                   int end_bit, rs_stream_t stream, int* result_in_alt) {
  if (!result_in_alt) return RS_ERR_INVALID;
  *result_in_alt = 0;
  if (n > RS_NOALLOC_MAX_N) return RS_ERR_INVALID;
  rs_config cfg;
  const rs_status st = pick_config(n, begin_bit, end_bit, &cfg);
  if (st != RS_OK) return st;
  void* ws = nullptr;
  const rs_status ad = scratch_address(&ws);
  if (ad != RS_OK) return ad;
  return rs_sort(4, 0, keys, nullptr, keys_alt, nullptr, n, begin_bit, end_bit, &cfg, ws,
                 kScratchBytes, stream, result_in_alt);
}

rs_status rs_sort_keys_u32_noalloc_status(rs_stream_t stream, uint32_t* info) {
  if (info) *info = 0;
  void* ws = nullptr;
  const rs_status ad = scratch_address(&ws);
  if (ad != RS_OK) return ad;
  return rs_workspace_status(ws, stream, info);
}

}  // extern "C"
