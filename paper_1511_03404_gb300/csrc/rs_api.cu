// C ABI of the rs library (declared in include/rs.h): argument checks,
// variant choice, workspace sizing, device-status readback, per-kernel
// event timing and the test-only fault-injection knobs.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/rs.h"
#include "rs_host.h"

namespace rs {

const Variant* variants_k32(int* count);
const Variant* variants_kv32(int* count);
const Variant* variants_k64(int* count);
const Variant* variants_kv64(int* count);

const Variant* variants(int key_bytes, int val_bytes, int* count) {
  *count = 0;
  if (key_bytes == 4 && val_bytes == 0) return variants_k32(count);
  if (key_bytes == 4 && val_bytes == 4) return variants_kv32(count);
  if (key_bytes == 8 && val_bytes == 0) return variants_k64(count);
  if (key_bytes == 8 && val_bytes == 8) return variants_kv64(count);
  return nullptr;
}

// ---------------------------------------------------------------- device

const DeviceInfo& device_info() {
  static std::mutex mu;
  static std::map<int, DeviceInfo> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(mu);
  auto it = cache.find(dev);
  if (it == cache.end()) {
    DeviceInfo d{dev, 1, 48 * 1024};
    cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    it = cache.emplace(dev, d).first;
  }
  return it->second;
}

int prepare_kernel(const void* func, int threads, int smem_bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> cache;  // (func, device) -> CTAs/SM
  const DeviceInfo& di = device_info();
  std::lock_guard<std::mutex> g(mu);
  auto key = std::make_pair(func, di.device * 4096 + threads);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  if (smem_bytes > di.smem_optin) return 0;
  if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, func, threads, smem_bytes) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cache[key] = blocks;
  return blocks;
}

// ------------------------------------------------- debug bounds checks

namespace {
std::mutex& dbg_mu() {
  static std::mutex m;
  return m;
}
std::vector<DbgReader>& dbg_readers() {
  static std::vector<DbgReader> v;
  return v;
}
}  // namespace

void register_dbg_reader(DbgReader reader) {
  std::lock_guard<std::mutex> g(dbg_mu());
  dbg_readers().push_back(reader);
}

// ----------------------------------------------------------------- knobs

static std::atomic<long long> g_timeout_ns{1000000000LL};
static std::atomic<long long> g_drop_tile{-1};
static std::atomic<long long> g_drop_pass{-1};
static std::atomic<long long> g_trace_ptr{0};
static std::atomic<long long> g_trace_tiles{0};
static std::atomic<long long> g_trace_pass{0};
static std::atomic<long long> g_lb_small{0};
static std::atomic<long long> g_dbg_bad_tile{-1};

bool pdl_enabled() {
  static const bool on = std::getenv("RS_NO_PDL") == nullptr;
  return on;
}

bool nvtx_enabled() {
  static const bool on = std::getenv("RS_NVTX") != nullptr;
  return on;
}

void nvtx_push(const char* name) {
  if (nvtx_enabled()) nvtxRangePushA(name);
}

void nvtx_pop() {
  if (nvtx_enabled()) nvtxRangePop();
}

const char* const kPassNames[kMaxPasses] = {
    "rs pass 0",  "rs pass 1",  "rs pass 2",  "rs pass 3",  "rs pass 4",  "rs pass 5",
    "rs pass 6",  "rs pass 7",  "rs pass 8",  "rs pass 9",  "rs pass 10", "rs pass 11",
    "rs pass 12", "rs pass 13", "rs pass 14", "rs pass 15"};

Knobs knobs_now() {
  Knobs k;
  k.timeout_ns = uint64_t(g_timeout_ns.load());
  k.drop_tile = int32_t(g_drop_tile.load());
  k.drop_pass = int32_t(g_drop_pass.load());
  k.trace = reinterpret_cast<uint64_t*>(g_trace_ptr.load());
  k.trace_tiles = uint32_t(g_trace_tiles.load());
  k.trace_pass = int32_t(g_trace_pass.load());
  k.lb_small = int32_t(g_lb_small.load());
  k.dbg_bad_tile = int32_t(g_dbg_bad_tile.load());
  return k;
}

// -------------------------------------------------------------- profiler

namespace {
struct ProfRec {
  int kind;
  double bytes;
  int slot;
  int pass;
};
struct Prof {
  bool on = false;
  int cap = 0;
  int device = -1;
  std::vector<cudaEvent_t> ev;
  std::vector<ProfRec> recs;
  uint32_t* h_masks = nullptr;
  int next_mask = 0;
  void release() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    ev.clear();
    recs.clear();
    if (h_masks) cudaFreeHost(h_masks);
    h_masks = nullptr;
    next_mask = 0;
    cap = 0;
    on = false;
  }
};
thread_local Prof g_prof;
}  // namespace

void prof_before(cudaStream_t s) {
  Prof& p = g_prof;
  if (!p.on || int(p.recs.size()) >= p.cap) return;
  cudaEventRecord(p.ev[2 * p.recs.size()], s);
}

int prof_note_mask(cudaStream_t s, const uint32_t* d_mask) {
  Prof& p = g_prof;
  if (!p.on || p.next_mask >= p.cap) return -1;
  const int slot = p.next_mask++;
  cudaMemcpyAsync(p.h_masks + slot, d_mask, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  return slot;
}

void prof_after(cudaStream_t s, int kind, double bytes, int slot, int pass) {
  Prof& p = g_prof;
  if (!p.on || int(p.recs.size()) >= p.cap) return;
  cudaEventRecord(p.ev[2 * p.recs.size() + 1], s);
  p.recs.push_back(ProfRec{kind, bytes, slot, pass});
}

// ------------------------------------------------------------ tuned table

namespace {
struct TuneEntry {
  size_t n_max;
  int variant;
};
std::mutex g_tune_mu;
std::map<int, std::vector<TuneEntry>> g_tune;  // key: key_bytes * 16 + val_bytes
std::once_flag g_tune_defaults;

// The package's tuned table as it stood when the library was built (the
// build step writes it from tuned.json), so that C callers get the tuned
// choices without the Python binding.
struct TunedDefault {
  int key_bytes, val_bytes;
  unsigned long long n_max;
  int variant;
};
const TunedDefault kTunedDefault[] = {
#include "rs_tuned_table.inc"
    {0, 0, 0ull, -1}};

// caller holds g_tune_mu
bool tune_set_locked(int key_bytes, int val_bytes, size_t n_max, int variant) {
  int count = 0;
  const Variant* v = variants(key_bytes, val_bytes, &count);
  if (!v || variant < 0 || variant >= count) return false;
  auto& list = g_tune[key_bytes * 16 + val_bytes];
  bool replaced = false;
  for (TuneEntry& e : list)
    if (e.n_max == n_max) {
      e.variant = variant;
      replaced = true;
    }
  if (!replaced) list.push_back(TuneEntry{n_max, variant});
  std::sort(list.begin(), list.end(),
            [](const TuneEntry& a, const TuneEntry& b) { return a.n_max < b.n_max; });
  return true;
}

// Install the built-in table once, before the table is first read or
// changed (not when the environment sets RS_NO_TUNED_TABLE).
void tune_defaults_once() {
  std::call_once(g_tune_defaults, [] {
    if (std::getenv("RS_NO_TUNED_TABLE")) return;
    std::lock_guard<std::mutex> g(g_tune_mu);
    for (const TunedDefault& d : kTunedDefault)
      if (d.variant >= 0) tune_set_locked(d.key_bytes, d.val_bytes, size_t(d.n_max), d.variant);
  });
}
}  // namespace

// The tuned variant for n elements of (kb, vb), or -1.
static int tuned_variant(int kb, int vb, size_t n) {
  tune_defaults_once();
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto it = g_tune.find(kb * 16 + vb);
  if (it == g_tune.end()) return -1;
  for (const TuneEntry& e : it->second)
    if (n <= e.n_max) return e.variant;
  return -1;
}

// -------------------------------------------------------------- choosing

static const Variant* choose(int kb, int vb, size_t n, const rs_config* cfg) {
  int count = 0;
  const Variant* v = variants(kb, vb, &count);
  if (!v) return nullptr;
  const int want_r = (cfg && cfg->radix_bits > 0) ? cfg->radix_bits : 0;
  if (cfg && cfg->variant >= 0) {
    if (cfg->variant >= count) return nullptr;
    const Variant* c = &v[cfg->variant];
    if (want_r && c->radix_bits != want_r) return nullptr;
    return n <= c->max_n ? c : nullptr;
  }
  if (!want_r) {
    const int tv = tuned_variant(kb, vb, n);
    if (tv >= 0 && tv < count && n <= v[tv].max_n) return &v[tv];
  }
  // default: one CTA when the array fits a small-sort tile, else onesweep
  const Variant* best = nullptr;
  for (int i = 0; i < count; ++i) {
    const Variant* c = &v[i];
    if (want_r && c->radix_bits != want_r) continue;
    if (n > c->max_n) continue;
    if (c->kind == kSmall && (!best || best->kind != kSmall)) best = c;
    if ((c->kind == kOnesweep || c->kind == kOnesweepPersist) && !best) best = c;
  }
  return best;
}

static bool valid_types(int kb, int vb) {
  return (kb == 4 || kb == 8) && (vb == 0 || vb == kb);
}

static bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace rs

using namespace rs;

extern "C" {

const char* rs_status_string(rs_status s) {
  switch (s) {
    case RS_OK: return "RS_OK";
    case RS_ERR_INVALID: return "RS_ERR_INVALID: invalid argument";
    case RS_ERR_NOMEM: return "RS_ERR_NOMEM: allocation failed";
    case RS_ERR_CUDA: return "RS_ERR_CUDA: CUDA runtime error";
    case RS_ERR_TIMEOUT: return "RS_ERR_TIMEOUT: bounded device wait ran out";
    case RS_ERR_BUSY: return "RS_ERR_BUSY: not admitted now";
    case RS_ERR_WORKSPACE: return "RS_ERR_WORKSPACE: workspace missing, too small or misaligned";
    case RS_ERR_DEVICE: return "RS_ERR_DEVICE: device-side index check failed";
    case RS_ERR_CANCELLED: return "RS_ERR_CANCELLED: request cancelled";
    case RS_ERR_NOT_FOUND: return "RS_ERR_NOT_FOUND: unknown handle";
  }
  return "unknown rs_status";
}

const char* rs_version(void) { return "0.1.0"; }

int rs_num_variants(int key_bytes, int val_bytes) {
  int count = 0;
  variants(key_bytes, val_bytes, &count);
  return count;
}

rs_status rs_variant_info(int key_bytes, int val_bytes, int index, int* radix_bits, int* threads,
                          int* items_per_thread, int* kind, size_t* max_n) {
  int count = 0;
  const Variant* v = variants(key_bytes, val_bytes, &count);
  if (!v || index < 0 || index >= count) return RS_ERR_INVALID;
  const Variant& c = v[index];
  if (radix_bits) *radix_bits = c.radix_bits;
  if (threads) *threads = c.threads;
  if (items_per_thread) *items_per_thread = c.items;
  if (kind) *kind = c.kind;
  if (max_n) *max_n = c.max_n;
  return RS_OK;
}

rs_status rs_workspace_bytes(int key_bytes, int val_bytes, size_t n, int begin_bit, int end_bit,
                             const rs_config* cfg, size_t* bytes) {
  if (!bytes || !valid_types(key_bytes, val_bytes)) return RS_ERR_INVALID;
  if (n > RS_MAX_N || begin_bit < 0 || begin_bit > end_bit || end_bit > 8 * key_bytes)
    return RS_ERR_INVALID;
  *bytes = 0;
  if (n <= 1 || begin_bit == end_bit) return RS_OK;
  const Variant* v = choose(key_bytes, val_bytes, n, cfg);
  if (!v) return RS_ERR_INVALID;
  *bytes = v->workspace(uint32_t(n), num_passes(begin_bit, end_bit, v->radix_bits));
  return RS_OK;
}

rs_status rs_sort(int key_bytes, int val_bytes, void* keys, void* vals, void* keys_alt,
                  void* vals_alt, size_t n, int begin_bit, int end_bit, const rs_config* cfg,
                  void* ws, size_t ws_bytes, rs_stream_t stream, int* result_in_alt) {
  if (!result_in_alt || !valid_types(key_bytes, val_bytes)) return RS_ERR_INVALID;
  if (n > RS_MAX_N || begin_bit < 0 || begin_bit > end_bit || end_bit > 8 * key_bytes)
    return RS_ERR_INVALID;
  const int key_kind = cfg ? cfg->key_kind : RS_KEY_UNSIGNED;
  const int descending = cfg ? cfg->descending : 0;
  if (key_kind < RS_KEY_UNSIGNED || key_kind > RS_KEY_FLOAT || (descending & ~1))
    return RS_ERR_INVALID;
  *result_in_alt = 0;
  if (n <= 1 || begin_bit == end_bit) {  // already sorted, nothing moves
    // clear the status word and the per-call record (no record: form 0)
    if (ws && ws_bytes >= sizeof(Ctrl) &&
        cudaMemsetAsync(ws, 0, sizeof(Ctrl), reinterpret_cast<cudaStream_t>(stream)) !=
            cudaSuccess)
      return RS_ERR_CUDA;
    return RS_OK;
  }
  if ((val_bytes == 0) != (vals == nullptr && vals_alt == nullptr)) return RS_ERR_INVALID;
  if (!keys || !keys_alt || keys == keys_alt) return RS_ERR_INVALID;
  if (!aligned(keys, key_bytes) || !aligned(keys_alt, key_bytes)) return RS_ERR_INVALID;
  if (val_bytes) {
    if (!vals || !vals_alt || vals == vals_alt) return RS_ERR_INVALID;
    if (!aligned(vals, val_bytes) || !aligned(vals_alt, val_bytes)) return RS_ERR_INVALID;
  }
  const Variant* v = choose(key_bytes, val_bytes, n, cfg);
  if (!v) return RS_ERR_INVALID;
  const int passes = num_passes(begin_bit, end_bit, v->radix_bits);
  const size_t need = v->workspace(uint32_t(n), passes);
  if (need > 0 && (!ws || ws_bytes < need || !aligned(ws, 256))) return RS_ERR_WORKSPACE;
  SortArgs a{keys, vals, keys_alt, vals_alt, uint32_t(n), begin_bit, end_bit, ws, ws_bytes,
             reinterpret_cast<cudaStream_t>(stream), knobs_now()};
  a.key_kind = key_kind;
  a.descending = descending;
  int in_alt = 0;
  nvtx_push("rs_sort");
  const cudaError_t e = v->run(a, &in_alt);
  nvtx_pop();
  if (e != cudaSuccess) return RS_ERR_CUDA;
  *result_in_alt = in_alt;
  return RS_OK;
}

rs_status rs_sort_host(int key_bytes, int val_bytes, const void* h_keys, const void* h_vals,
                       void* h_out_keys, void* h_out_vals, size_t n, int begin_bit, int end_bit,
                       const rs_config* cfg, void* keys, void* vals, void* keys_alt,
                       void* vals_alt, void* ws, size_t ws_bytes, rs_stream_t stream,
                       int* result_in_alt) {
  if (!result_in_alt || !valid_types(key_bytes, val_bytes)) return RS_ERR_INVALID;
  *result_in_alt = 0;
  if (n > RS_MAX_N) return RS_ERR_INVALID;
  if (n > 0 && (!h_keys || !h_out_keys || !keys)) return RS_ERR_INVALID;
  if (n > 0 && (val_bytes != 0) != (h_vals != nullptr && h_out_vals != nullptr && vals != nullptr))
    return RS_ERR_INVALID;
  if (val_bytes == 0 && (h_vals || h_out_vals)) return RS_ERR_INVALID;
  // every argument the sort checks is checked before anything is enqueued
  size_t need = 0;
  rs_status st = rs_workspace_bytes(key_bytes, val_bytes, n, begin_bit, end_bit, cfg, &need);
  if (st != RS_OK) return st;
  if (n <= 1 || begin_bit == end_bit) {  // nothing moves: the input is the output
    if (n == 0) return rs_sort(key_bytes, val_bytes, keys, vals, keys_alt, vals_alt, n,
                               begin_bit, end_bit, cfg, ws, ws_bytes, stream, result_in_alt);
  } else {
    if ((val_bytes == 0) != (vals_alt == nullptr) || !keys_alt || keys == keys_alt)
      return RS_ERR_INVALID;
    if (!aligned(keys, key_bytes) || !aligned(keys_alt, key_bytes)) return RS_ERR_INVALID;
    if (val_bytes && (vals == vals_alt || !aligned(vals, val_bytes) || !aligned(vals_alt, val_bytes)))
      return RS_ERR_INVALID;
    if (cfg && (cfg->key_kind < RS_KEY_UNSIGNED || cfg->key_kind > RS_KEY_FLOAT ||
                (cfg->descending & ~1)))
      return RS_ERR_INVALID;
    if (need > 0 && (!ws || ws_bytes < need || !aligned(ws, 256))) return RS_ERR_WORKSPACE;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t kbytes = n * size_t(key_bytes), vbytes = n * size_t(val_bytes);
  nvtx_push("rs_sort_host");
  if (cudaMemcpyAsync(keys, h_keys, kbytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      (vbytes && cudaMemcpyAsync(vals, h_vals, vbytes, cudaMemcpyHostToDevice, s) != cudaSuccess)) {
    nvtx_pop();
    return RS_ERR_CUDA;
  }
  int in_alt = 0;
  st = rs_sort(key_bytes, val_bytes, keys, vals, keys_alt, vals_alt, n, begin_bit, end_bit, cfg,
               ws, ws_bytes, stream, &in_alt);
  if (st != RS_OK) {
    nvtx_pop();
    return st;
  }
  const void* rk = in_alt ? keys_alt : keys;
  const void* rv = in_alt ? vals_alt : vals;
  if (cudaMemcpyAsync(h_out_keys, rk, kbytes, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      (vbytes && cudaMemcpyAsync(h_out_vals, rv, vbytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)) {
    nvtx_pop();
    return RS_ERR_CUDA;
  }
  nvtx_pop();
  *result_in_alt = in_alt;
  return RS_OK;
}

rs_status rs_sort_keys_u32(uint32_t* keys, uint32_t* keys_alt, size_t n, int begin_bit,
                           int end_bit, void* ws, size_t ws_bytes, rs_stream_t stream,
                           int* result_in_alt) {
  return rs_sort(4, 0, keys, nullptr, keys_alt, nullptr, n, begin_bit, end_bit, nullptr, ws,
                 ws_bytes, stream, result_in_alt);
}

rs_status rs_sort_keys_u64(uint64_t* keys, uint64_t* keys_alt, size_t n, int begin_bit,
                           int end_bit, void* ws, size_t ws_bytes, rs_stream_t stream,
                           int* result_in_alt) {
  return rs_sort(8, 0, keys, nullptr, keys_alt, nullptr, n, begin_bit, end_bit, nullptr, ws,
                 ws_bytes, stream, result_in_alt);
}

rs_status rs_sort_pairs_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt,
                            uint32_t* vals_alt, size_t n, int begin_bit, int end_bit, void* ws,
                            size_t ws_bytes, rs_stream_t stream, int* result_in_alt) {
  return rs_sort(4, 4, keys, vals, keys_alt, vals_alt, n, begin_bit, end_bit, nullptr, ws,
                 ws_bytes, stream, result_in_alt);
}

rs_status rs_sort_pairs_u64(uint64_t* keys, uint64_t* vals, uint64_t* keys_alt,
                            uint64_t* vals_alt, size_t n, int begin_bit, int end_bit, void* ws,
                            size_t ws_bytes, rs_stream_t stream, int* result_in_alt) {
  return rs_sort(8, 8, keys, vals, keys_alt, vals_alt, n, begin_bit, end_bit, nullptr, ws,
                 ws_bytes, stream, result_in_alt);
}

rs_status rs_digit_counts(int key_bytes, const void* keys, size_t n, int begin_bit, int end_bit,
                          int radix_bits, uint32_t* d_counts, uint32_t* d_offsets,
                          uint32_t* d_exec_mask, void* ws, size_t ws_bytes, rs_stream_t stream) {
  if (!valid_types(key_bytes, 0) || n > RS_MAX_N || begin_bit < 0 || begin_bit >= end_bit ||
      end_bit > 8 * key_bytes)
    return RS_ERR_INVALID;
  if (!d_counts || !d_offsets || !d_exec_mask || (n && !keys) || !aligned(keys, key_bytes))
    return RS_ERR_INVALID;
  int count = 0;
  const Variant* all = variants(key_bytes, 0, &count);
  const Variant* v = nullptr;
  for (int i = 0; i < count && !v; ++i)
    if (all[i].count != nullptr && all[i].radix_bits == radix_bits) v = &all[i];
  if (!v) return RS_ERR_INVALID;
  const int passes = num_passes(begin_bit, end_bit, radix_bits);
  const Layout L = onesweep_layout(passes, radix_bits, 0);
  if (!ws || ws_bytes < L.status || !aligned(ws, 256)) return RS_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  SortArgs a{const_cast<void*>(keys), nullptr, nullptr, nullptr, uint32_t(n), begin_bit,
             end_bit, ws, ws_bytes, s, knobs_now()};
  if (v->count(a) != cudaSuccess) return RS_ERR_CUDA;
  const size_t table = size_t(passes) << radix_bits;
  char* w = static_cast<char*>(ws);
  if (cudaMemcpyAsync(d_counts, w + L.counts, table * 4, cudaMemcpyDeviceToDevice, s) ||
      cudaMemcpyAsync(d_offsets, w + L.offsets, table * 4, cudaMemcpyDeviceToDevice, s) ||
      cudaMemcpyAsync(d_exec_mask, &reinterpret_cast<Ctrl*>(w)->exec_mask, 4,
                      cudaMemcpyDeviceToDevice, s))
    return RS_ERR_CUDA;
  return RS_OK;
}

rs_status rs_workspace_status(const void* ws, rs_stream_t stream, uint32_t* info) {
  if (info) *info = 0;
  if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
    return RS_ERR_CUDA;
  if (!ws) return RS_OK;
  uint32_t head[2] = {0, 0};
  if (cudaMemcpy(head, ws, sizeof(head), cudaMemcpyDeviceToHost) != cudaSuccess)
    return RS_ERR_CUDA;
  if (info) *info = head[1];
  switch (head[0]) {
    case kDevOk: return RS_OK;
    case kDevTimeout: return RS_ERR_TIMEOUT;
    case 1u: return RS_ERR_INVALID;  // e.g. segment offsets that do not describe the array
    default: return RS_ERR_DEVICE;
  }
}

rs_status rs_workspace_stats(const void* ws, rs_stream_t stream, rs_sort_stats* out) {
  if (!out) return RS_ERR_INVALID;
  std::memset(out, 0, sizeof(*out));
  out->status = rs_workspace_status(ws, stream, &out->info);
  if (out->status == RS_ERR_CUDA || !ws) return out->status == RS_ERR_CUDA ? RS_ERR_CUDA : RS_OK;
  Ctrl c;
  if (cudaMemcpy(&c, ws, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess) return RS_ERR_CUDA;
  const int form = int(c.stat_shape >> 24);
  if (form < 1 || form > 3) return RS_OK;  // this call left no record (see the header)
  out->form = form;
  out->key_bytes = int(c.stat_shape & 0xffu);
  out->val_bytes = int((c.stat_shape >> 8) & 0xffu);
  out->passes = int((c.stat_shape >> 16) & 0xffu);
  out->n = c.stat_n;
  if (out->passes < 1 || out->passes > kMaxPasses) {
    out->form = 0;
    return RS_OK;
  }
  const uint32_t all = out->passes >= 32 ? ~0u : ((1u << out->passes) - 1u);
  out->moved_mask = c.exec_mask & all;
  out->skipped_mask = all & ~out->moved_mask;
  const double kb = out->key_bytes, vb = out->val_bytes, n = double(out->n);
  out->upsweep_ms = c.t_upsweep * 1e-6;
  uint32_t last = c.t_upsweep;
  for (int p = 0; p < out->passes; ++p) {
    if (c.t_pass[p][1] > c.t_pass[p][0] && c.t_pass[p][0] > 0)
      out->pass_ms[p] = (c.t_pass[p][1] - c.t_pass[p][0]) * 1e-6;
    last = std::max(last, c.t_pass[p][1]);
  }
  out->total_ms = last * 1e-6;
  if (form == 3)
    out->bytes = 2.0 * n * (kb + vb);  // one read and one write; the passes stay on chip
  else
    out->bytes = n * kb + double(__builtin_popcount(out->moved_mask)) * 2.0 * n * (kb + vb);
  return RS_OK;
}

rs_status rs_debug_status(int* debug_build, uint32_t* site, uint64_t* index) {
#ifdef RS_DEBUG
  const int is_debug = 1;
#else
  const int is_debug = 0;
#endif
  if (debug_build) *debug_build = is_debug;
  if (site) *site = 0;
  if (index) *index = 0;
  if (!is_debug) return RS_OK;
  if (cudaDeviceSynchronize() != cudaSuccess) return RS_ERR_CUDA;
  std::vector<DbgReader> readers;
  {
    std::lock_guard<std::mutex> g(dbg_mu());
    readers = dbg_readers();
  }
  rs_status st = RS_OK;
  for (DbgReader r : readers) {
    uint64_t w = 0;
    if (!r(&w)) return RS_ERR_CUDA;
    if ((w >> 63) && st == RS_OK) {
      st = RS_ERR_DEVICE;
      if (site) *site = uint32_t((w >> 48) & 0x7fffu);
      if (index) *index = w & ((uint64_t(1) << 48) - 1);
    }
  }
  return st;
}

rs_status rs_profile_begin(int capacity) {
  if (capacity <= 0 || capacity > (1 << 20)) return RS_ERR_INVALID;
  Prof& p = g_prof;
  p.release();
  p.ev.resize(size_t(2) * capacity);
  for (auto& e : p.ev) {
    if (cudaEventCreate(&e) != cudaSuccess) {
      e = nullptr;
      p.release();
      return RS_ERR_CUDA;
    }
  }
  if (cudaHostAlloc(reinterpret_cast<void**>(&p.h_masks), sizeof(uint32_t) * capacity,
                    cudaHostAllocDefault) != cudaSuccess) {
    p.h_masks = nullptr;
    p.release();
    return RS_ERR_NOMEM;
  }
  p.cap = capacity;
  p.recs.reserve(capacity);
  p.on = true;
  return RS_OK;
}

rs_status rs_profile_end(int* launches, double* ms, double* bytes) {
  Prof& p = g_prof;
  if (!p.on) return RS_ERR_INVALID;
  p.on = false;
  int l[RS_KERNEL_KINDS] = {0};
  double t[RS_KERNEL_KINDS] = {0}, b[RS_KERNEL_KINDS] = {0};
  rs_status st = RS_OK;
  for (size_t i = 0; i < p.recs.size(); ++i) {
    const ProfRec& r = p.recs[i];
    float e = 0.f;
    if (cudaEventSynchronize(p.ev[2 * i + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&e, p.ev[2 * i], p.ev[2 * i + 1]) != cudaSuccess) {
      st = RS_ERR_CUDA;
      continue;
    }
    double by = r.bytes;
    if (r.slot >= 0 && !((p.h_masks[r.slot] >> r.pass) & 1u)) by = 0.0;  // pass did not move data
    if (r.kind >= 0 && r.kind < RS_KERNEL_KINDS) {
      l[r.kind] += 1;
      t[r.kind] += e;
      b[r.kind] += by;
    }
  }
  for (int k = 0; k < RS_KERNEL_KINDS; ++k) {
    if (launches) launches[k] = l[k];
    if (ms) ms[k] = t[k];
    if (bytes) bytes[k] = b[k];
  }
  p.release();
  return st;
}

rs_status rs_tune_set(int key_bytes, int val_bytes, size_t n_max, int variant) {
  tune_defaults_once();
  std::lock_guard<std::mutex> g(g_tune_mu);
  return tune_set_locked(key_bytes, val_bytes, n_max, variant) ? RS_OK : RS_ERR_INVALID;
}

rs_status rs_tune_clear(void) {
  tune_defaults_once();
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune.clear();
  return RS_OK;
}

rs_status rs_debug_set(rs_debug_knob knob, long long value) {
  switch (knob) {
    case RS_DEBUG_TIMEOUT_NS:
      if (value <= 0) return RS_ERR_INVALID;
      g_timeout_ns.store(value);
      return RS_OK;
    case RS_DEBUG_DROP_PUBLISH_TILE:
      g_drop_tile.store(value);
      return RS_OK;
    case RS_DEBUG_DROP_PUBLISH_PASS:
      g_drop_pass.store(value);
      return RS_OK;
    case RS_DEBUG_TRACE_PTR:
      g_trace_ptr.store(value);
      return RS_OK;
    case RS_DEBUG_TRACE_TILES:
      if (value < 0 || value > (1ll << 30)) return RS_ERR_INVALID;
      g_trace_tiles.store(value);
      return RS_OK;
    case RS_DEBUG_TRACE_PASS:
      g_trace_pass.store(value);
      return RS_OK;
    case RS_DEBUG_LB_SMALL:
      g_lb_small.store(value);
      return RS_OK;
    case RS_DEBUG_BAD_INDEX_TILE:
#ifdef RS_DEBUG
      g_dbg_bad_tile.store(value < 0 ? -1 : value);
      return RS_OK;
#else
      return RS_ERR_INVALID;  // only a build that checks every store index takes it
#endif
  }
  return RS_ERR_INVALID;
}

}  // extern "C"
