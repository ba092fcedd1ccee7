// Sort server: continuous batching of sort requests on one GPU.
//
// A scheduler thread admits queued requests while their device footprint
// fits the memory budget (one resident device pool, carved by a first-fit
// allocator) and while stream slots are free.  Admitted short requests of one
// type and bit range are packed into one batched segmented sort; every other
// request runs as its own sort.  Each admitted unit goes to one of several CUDA
// streams, so copies and sorts of different requests overlap on the device,
// and requests that arrive while others run are admitted as memory and slots
// free up.  A host callback at the end of each unit's stream work marks its
// requests done; rs_poll reports that without blocking.
//
// Copies: by default a unit's copies run on its own stream.  With shared copy
// queues (a policy option) every unit's host-to-device copies go through one
// FIFO copy stream per size class (short / large) and its device-to-host
// copies through another, ordered against the unit's sort by events: one
// copy then has the host link to itself and its sort starts as soon as it
// lands.  On the mixed serving trace the two measured the same capacity and
// the option gave short requests a longer median (their copies wait behind
// larger ones in the FIFO), so it is off by default.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/rs.h"
#include "rs_common.h"
#include "rs_host.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_s() {
  return std::chrono::duration<double>(Clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) with coalescing free blocks.
class Pool {
 public:
  explicit Pool(size_t size) : size_(size) { free_[0] = size; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = rs::align_up(std::max<size_t>(bytes, 256), 256);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t noff = it->first + bytes;
        free_.erase(it);
        if (rest) free_[noff] = rest;
        used_ += bytes;
        peak_ = std::max(peak_, used_);
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = rs::align_up(std::max<size_t>(bytes, 256), 256);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }

 private:
  size_t size_, used_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_;
};

struct Request {
  uint64_t id = 0;
  rs_request req{};
  int state = 0;  // 0 queued, 1 running, 2 done
  rs_status status = RS_OK;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int stream = -1;
  bool batched = false;
};

struct Unit;  // one admitted sort or batch

constexpr size_t kMaxBatchMembers = 1024;

}  // namespace

struct rs_server {
  int device = 0;
  size_t budget = 0;
  char* pool_base = nullptr;
  std::unique_ptr<Pool> pool;
  std::vector<cudaStream_t> streams;     // high priority: short requests and batches
  std::vector<cudaStream_t> streams_lo;  // low priority, same slots: large requests
  std::vector<int> stream_busy;
  size_t batch_max_n = 1u << 14;  // requests up to this size share a segmented launch
  size_t max_batch_keys = 1u << 22;
  // Large requests (at least large_n keys) are admitted at most max_large at a
  // time, oldest first: running many at once only splits the copy bandwidth
  // between them and stretches every one (the tail of the latency), while
  // shorter requests keep the other streams.
  size_t large_n = size_t(1) << 21;
  int max_large = 3;
  int large_low_priority = 1;
  int shared_copy_queues = 0;
  int large_running = 0;
  cudaStream_t copy_in[2] = {nullptr, nullptr};   // FIFO host-to-device: [0] short, [1] large
  cudaStream_t copy_out[2] = {nullptr, nullptr};  // FIFO device-to-host, same classes
  std::vector<cudaEvent_t> ev_in, ev_sorted;      // per stream slot: input landed, sort done
  std::mutex mu;
  std::condition_variable cv;
  std::deque<uint64_t> pending;
  std::unordered_map<uint64_t, std::shared_ptr<Request>> reqs;
  std::vector<Unit*> finished;  // completed units, handed over by the host callbacks
  uint64_t changes = 0;         // bumped by every submit, cancel and completion
  uint32_t* status_slab = nullptr;  // pinned, one device-status word per stream
  // pinned, per stream: the segment offsets of a batch (a copy from pageable
  // memory would wait for the stream's earlier copies and stall the scheduler)
  uint64_t* off_slab = nullptr;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread sched;
  // statistics
  std::vector<rs_trace_record> trace;  // completed requests; times absolute (now_s)
  std::deque<uint64_t> completed_ids;  // finished, not yet taken by rs_server_completed
  uint64_t completed = 0, failed = 0, keys_done = 0, batches = 0, batched_requests = 0;
  double first_submit = 0, last_done = 0;
  size_t max_queue = 0;
};

namespace {

struct Unit {
  rs_server* srv = nullptr;
  std::vector<std::shared_ptr<Request>> members;
  size_t pool_off = 0, pool_bytes = 0;
  int stream = 0;
  bool large = false;
  bool low_priority = false;     // sorts on the slot's low-priority stream
  bool shared_copies = false;    // copies through the server's copy queues
  uint32_t* h_status = nullptr;  // pinned: device status word of the sort
};

// The streams of one unit's copies in, sort and copies out (one stream for
// all three unless the unit uses the shared copy queues).
struct Lanes {
  cudaStream_t in, cs, out;
};

Lanes lanes_of(const rs_server* s, const Unit* u) {
  // (the unit's fields are set at admission, under the server's lock; the
  // streams do not change after creation)
  const cudaStream_t cs = u->low_priority ? s->streams_lo[u->stream] : s->streams[u->stream];
  if (!u->shared_copies) return Lanes{cs, cs, cs};
  const int c = u->large ? 1 : 0;
  return Lanes{s->copy_in[c], cs, s->copy_out[c]};
}

// Order `to` after the work enqueued so far on `from` (nothing when they are
// the same stream).
bool order_after(cudaStream_t from, cudaStream_t to, cudaEvent_t ev) {
  if (from == to) return true;
  return cudaEventRecord(ev, from) == cudaSuccess && cudaStreamWaitEvent(to, ev, 0) == cudaSuccess;
}


bool valid_request(const rs_request& r) {
  if (!((r.key_bytes == 4 || r.key_bytes == 8) && (r.val_bytes == 0 || r.val_bytes == r.key_bytes)))
    return false;
  if (r.n > RS_MAX_N || r.begin_bit < 0 || r.begin_bit > r.end_bit || r.end_bit > 8 * r.key_bytes)
    return false;
  if (r.n && (!r.h_keys || !r.h_out_keys)) return false;
  if (r.n && r.val_bytes && (!r.h_vals || !r.h_out_vals)) return false;
  return true;
}

// Device layout of one request's unit: keys, values, their alternates, workspace.
struct SingleLayout {
  size_t k, v, ka, va, ws, ws_bytes, total;
};

SingleLayout single_layout(const rs_request& r) {
  SingleLayout L;
  size_t ws = 0;
  rs_workspace_bytes(r.key_bytes, r.val_bytes, r.n, r.begin_bit, r.end_bit, nullptr, &ws);
  const size_t kb = rs::align_up(r.n * size_t(r.key_bytes), 256);
  const size_t vb = rs::align_up(r.n * size_t(r.val_bytes), 256);
  L.k = 0;
  L.v = L.k + kb;
  L.ka = L.v + vb;
  L.va = L.ka + kb;
  L.ws = L.va + vb;
  L.ws_bytes = rs::align_up(std::max<size_t>(ws, 256), 256);
  L.total = L.ws + L.ws_bytes;
  return L;
}

size_t single_footprint(const rs_request& r) { return single_layout(r).total; }

bool batchable(const rs_server* s, const rs_request& r) {
  return r.n <= s->batch_max_n && r.n > 1 && r.begin_bit < r.end_bit;
}

// Requests that can share one batched segmented sort: same types and bits.
bool same_batch(const rs_request& a, const rs_request& b) {
  return a.key_bytes == b.key_bytes && a.val_bytes == b.val_bytes &&
         a.begin_bit == b.begin_bit && a.end_bit == b.end_bit;
}

void CUDART_CB on_unit_done(void* p) {
  Unit* u = static_cast<Unit*>(p);
  rs_server* s = u->srv;
  const double t = now_s();
  {
    std::lock_guard<std::mutex> g(s->mu);
    for (auto& m : u->members) m->t_done = t;
    s->finished.push_back(u);
    s->changes += 1;
  }
  s->cv.notify_all();
}

// Enqueue copies in, the sort, copies out and the completion callback.
rs_status launch_single(rs_server* s, Unit* u) {
  Request& r = *u->members[0];
  const rs_request& q = r.req;
  const Lanes ln = lanes_of(s, u);
  char* base = s->pool_base + u->pool_off;
  const size_t kbytes = q.n * q.key_bytes, vbytes = q.n * q.val_bytes;
  const SingleLayout L = single_layout(q);
  char* k = base + L.k;
  char* v = base + L.v;
  char* ka = base + L.ka;
  char* va = base + L.va;
  char* ws = base + L.ws;
  const size_t ws_bytes = L.ws_bytes;
  if (cudaMemcpyAsync(k, q.h_keys, kbytes, cudaMemcpyHostToDevice, ln.in) != cudaSuccess)
    return RS_ERR_CUDA;
  if (vbytes && cudaMemcpyAsync(v, q.h_vals, vbytes, cudaMemcpyHostToDevice, ln.in) != cudaSuccess)
    return RS_ERR_CUDA;
  if (!order_after(ln.in, ln.cs, s->ev_in[u->stream])) return RS_ERR_CUDA;
  int in_alt = 0;
  rs_status rs_st = rs_sort(q.key_bytes, q.val_bytes, k, vbytes ? v : nullptr, ka,
                            vbytes ? va : nullptr, q.n, q.begin_bit, q.end_bit, nullptr, ws,
                            ws_bytes, reinterpret_cast<rs_stream_t>(ln.cs), &in_alt);
  if (rs_st != RS_OK) return rs_st;
  if (!order_after(ln.cs, ln.out, s->ev_sorted[u->stream])) return RS_ERR_CUDA;
  if (cudaMemcpyAsync(u->h_status, ws, sizeof(uint32_t), cudaMemcpyDeviceToHost, ln.out) !=
      cudaSuccess)
    return RS_ERR_CUDA;
  if (cudaMemcpyAsync(q.h_out_keys, in_alt ? ka : k, kbytes, cudaMemcpyDeviceToHost, ln.out) !=
      cudaSuccess)
    return RS_ERR_CUDA;
  if (vbytes && cudaMemcpyAsync(q.h_out_vals, in_alt ? va : v, vbytes, cudaMemcpyDeviceToHost,
                                ln.out) != cudaSuccess)
    return RS_ERR_CUDA;
  if (cudaLaunchHostFunc(ln.out, on_unit_done, u) != cudaSuccess) return RS_ERR_CUDA;
  return RS_OK;
}

struct BatchPlan {
  size_t total = 0, seg_ws = 0;
  size_t k, v, ka, va, off, ws, bytes;
};

// Device layout of a batch of nseg requests of the type of q, total keys.
BatchPlan plan_batch(const rs_request& q, size_t total, size_t nseg) {
  BatchPlan b;
  b.total = total;
  rs_segmented_workspace_bytes_typed(q.key_bytes, q.val_bytes, total, nseg, q.begin_bit,
                                     q.end_bit, &b.seg_ws);
  const size_t karr = rs::align_up(total * size_t(q.key_bytes), 256);
  const size_t varr = rs::align_up(total * size_t(q.val_bytes), 256);
  b.k = 0;
  b.v = b.k + karr;
  b.ka = b.v + varr;
  b.va = b.ka + karr;
  b.off = b.va + varr;
  b.ws = b.off + rs::align_up((nseg + 1) * 8, 256);
  b.bytes = b.ws + rs::align_up(std::max<size_t>(b.seg_ws, 256), 256);
  return b;
}

rs_status launch_batch(rs_server* s, Unit* u, const BatchPlan& b) {
  const Lanes ln = lanes_of(s, u);
  char* base = s->pool_base + u->pool_off;
  const size_t nseg = u->members.size();
  uint64_t* off = s->off_slab + size_t(u->stream) * (kMaxBatchMembers + 1);
  off[0] = 0;
  for (size_t i = 0; i < nseg; ++i) off[i + 1] = off[i] + u->members[i]->req.n;
  // every member in a batch has the same types and bit range (the scheduler
  // groups them)
  const rs_request& q0 = u->members[0]->req;
  const size_t kb = size_t(q0.key_bytes), vb = size_t(q0.val_bytes);
  for (size_t i = 0; i < nseg; ++i) {
    const rs_request& q = u->members[i]->req;
    if (cudaMemcpyAsync(base + b.k + off[i] * kb, q.h_keys, q.n * kb, cudaMemcpyHostToDevice,
                        ln.in) ||
        (vb && cudaMemcpyAsync(base + b.v + off[i] * vb, q.h_vals, q.n * vb,
                               cudaMemcpyHostToDevice, ln.in)))
      return RS_ERR_CUDA;
  }
  if (cudaMemcpyAsync(base + b.off, off, (nseg + 1) * 8, cudaMemcpyHostToDevice, ln.in))
    return RS_ERR_CUDA;
  if (!order_after(ln.in, ln.cs, s->ev_in[u->stream])) return RS_ERR_CUDA;
  int in_alt = 0;
  rs_status rs_st = rs_segmented_sort(
      q0.key_bytes, q0.val_bytes, base + b.k, vb ? base + b.v : nullptr, base + b.ka,
      vb ? base + b.va : nullptr, b.total, reinterpret_cast<const uint64_t*>(base + b.off), nseg,
      q0.begin_bit, q0.end_bit, base + b.ws, b.bytes - b.ws,
      reinterpret_cast<rs_stream_t>(ln.cs), &in_alt);
  if (rs_st != RS_OK) return rs_st;
  if (!order_after(ln.cs, ln.out, s->ev_sorted[u->stream])) return RS_ERR_CUDA;
  if (cudaMemcpyAsync(u->h_status, base + b.ws, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                      ln.out))
    return RS_ERR_CUDA;
  const size_t ko = in_alt ? b.ka : b.k, vo = in_alt ? b.va : b.v;
  for (size_t i = 0; i < nseg; ++i) {
    const rs_request& q = u->members[i]->req;
    if (cudaMemcpyAsync(q.h_out_keys, base + ko + off[i] * kb, q.n * kb, cudaMemcpyDeviceToHost,
                        ln.out) ||
        (vb && cudaMemcpyAsync(q.h_out_vals, base + vo + off[i] * vb, q.n * vb,
                               cudaMemcpyDeviceToHost, ln.out)))
      return RS_ERR_CUDA;
  }
  if (cudaLaunchHostFunc(ln.out, on_unit_done, u) != cudaSuccess) return RS_ERR_CUDA;
  return RS_OK;
}

int free_stream(rs_server* s) {
  for (size_t i = 0; i < s->streams.size(); ++i)
    if (!s->stream_busy[i]) return int(i);
  return -1;
}

constexpr size_t kMaxCompletedQueue = size_t(1) << 20;

void note_completed(rs_server* s, uint64_t id) {
  // caller holds s->mu
  if (s->completed_ids.size() >= kMaxCompletedQueue) s->completed_ids.pop_front();
  s->completed_ids.push_back(id);
}

void finish_unit(rs_server* s, Unit* u, rs_status st) {
  // caller holds s->mu
  s->pool->release(u->pool_off, u->pool_bytes);
  s->stream_busy[u->stream] = 0;
  if (u->large) s->large_running -= 1;
  rs_status dev = RS_OK;
  if (st == RS_OK && u->h_status && *u->h_status != 0u)
    dev = (*u->h_status == rs::kDevTimeout) ? RS_ERR_TIMEOUT
          : (*u->h_status == 1u)            ? RS_ERR_INVALID
                                            : RS_ERR_DEVICE;
  for (auto& m : u->members) {
    m->state = 2;
    m->status = st != RS_OK ? st : dev;
    note_completed(s, m->id);
    if (m->t_done == 0) m->t_done = now_s();
    if (m->status == RS_OK) {
      s->completed += 1;
      s->keys_done += m->req.n;
      rs_trace_record rec{};
      rec.submit_s = m->t_submit;
      rec.admit_s = m->t_admit;
      rec.done_s = m->t_done;
      rec.n = m->req.n;
      rec.key_bytes = m->req.key_bytes;
      rec.val_bytes = m->req.val_bytes;
      rec.stream = m->stream;
      rec.batched = m->batched ? 1 : 0;
      s->trace.push_back(rec);
      s->last_done = std::max(s->last_done, m->t_done);
    } else {
      s->failed += 1;
    }
  }
  delete u;
}

void scheduler(rs_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  uint64_t seen = ~0ull;
  while (true) {
    // sleep until something changed: a submission, a cancel or a completion
    s->cv.wait(lk, [&] { return s->stop || s->changes != seen; });
    seen = s->changes;
    for (Unit* u : s->finished) finish_unit(s, u, RS_OK);
    s->finished.clear();
    if (s->stop && s->pending.empty()) {
      bool busy = false;
      for (int b : s->stream_busy) busy |= (b != 0);
      if (!busy) break;
      continue;
    }
    // Admission, oldest first; a request that does not fit yet does not block
    // younger ones (bounded look-ahead).  Every decision is taken under the
    // lock and no iterator into the queue survives it: rs_submit may append
    // to the queue as soon as the lock is released.
    struct Launch {
      Unit* u;
      bool batch;
      BatchPlan plan;
    };
    std::vector<Launch> launches;
    std::vector<uint64_t> keep;  // looked at, still queued
    std::vector<std::shared_ptr<Request>> seen;  // taken off the queue front, in order
    while (!s->pending.empty() && seen.size() < 256) {
      const uint64_t id = s->pending.front();
      s->pending.pop_front();
      auto found = s->reqs.find(id);
      if (found != s->reqs.end()) seen.push_back(found->second);
    }
    // 1. Short requests first: the oldest batchable ones form one batch,
    //    which takes a free stream before any single request does.  Taken
    //    after the singles, it found every freed stream gone to the steady
    //    flow of medium requests, and short requests waited tens of ms.
    std::vector<std::shared_ptr<Request>> batch;
    size_t batch_keys = 0;
    for (auto& r : seen) {
      if (!batchable(s, r->req)) continue;
      const bool same = batch.empty() || same_batch(batch[0]->req, r->req);
      // a batch never outgrows the pool, so that it is admitted once enough
      // of the pool is free
      if (same && batch_keys + r->req.n <= s->max_batch_keys &&
          batch.size() < kMaxBatchMembers &&
          plan_batch(r->req, batch_keys + r->req.n, batch.size() + 1).bytes <= s->budget) {
        batch.push_back(r);
        batch_keys += r->req.n;
      }
    }
    // a batch of one request runs as that request's own sort (one launch for
    // a short array instead of the segmented sort's sequence)
    std::shared_ptr<Request> solo;
    if (batch.size() == 1) {
      solo = batch[0];
      batch.clear();
    }
    if (!batch.empty()) {
      const int si = free_stream(s);
      const BatchPlan b = plan_batch(batch[0]->req, batch_keys, batch.size());
      size_t off = 0;
      if (si >= 0 && s->pool->alloc(b.bytes, &off)) {
        Unit* u = new Unit;
        u->srv = s;
        u->members = batch;
        u->pool_off = off;
        u->pool_bytes = rs::align_up(b.bytes, 256);
        u->stream = si;
        u->shared_copies = s->shared_copy_queues != 0;
        u->h_status = s->status_slab + si;
        *u->h_status = 0u;
        s->stream_busy[si] = 1;
        const double t = now_s();
        for (auto& m : batch) {
          m->state = 1;
          m->t_admit = t;
          m->stream = si;
          m->batched = true;
        }
        s->batches += 1;
        s->batched_requests += batch.size();
        launches.push_back(Launch{u, true, b});
      }
    }
    // 2. Single requests in submission order.
    bool large_blocked = false;  // large requests are admitted in submission order
    for (auto& r : seen) {
      if (r->state != 0) continue;  // in the batch just formed
      if (batchable(s, r->req) && r != solo) {  // waits for a later batch
        keep.push_back(r->id);
        continue;
      }
      const bool large = r->req.n >= s->large_n;
      if (large && (large_blocked || s->large_running >= s->max_large)) {
        large_blocked = true;  // later large requests wait behind this one
        keep.push_back(r->id);
        continue;
      }
      const int si = free_stream(s);
      size_t off = 0;
      const size_t need = single_footprint(r->req);
      if (si < 0 || !s->pool->alloc(need, &off)) {
        if (large) large_blocked = true;
        keep.push_back(r->id);
        continue;
      }
      Unit* u = new Unit;
      u->srv = s;
      u->large = large;
      if (large) s->large_running += 1;
      u->members.push_back(r);
      u->pool_off = off;
      u->pool_bytes = rs::align_up(std::max<size_t>(need, 256), 256);
      u->stream = si;
      u->low_priority = large && s->large_low_priority != 0;
      u->shared_copies = s->shared_copy_queues != 0;
      u->h_status = s->status_slab + si;
      *u->h_status = 0u;
      s->stream_busy[si] = 1;
      r->state = 1;
      r->t_admit = now_s();
      r->stream = si;
      launches.push_back(Launch{u, false, BatchPlan{}});
    }
    if (keep.size() > 1)
      std::sort(keep.begin(), keep.end());  // ids grow with submission order
    for (auto it = keep.rbegin(); it != keep.rend(); ++it) s->pending.push_front(*it);
    if (launches.empty()) continue;
    lk.unlock();
    std::vector<rs_status> res(launches.size());
    for (size_t i = 0; i < launches.size(); ++i)
      res[i] = launches[i].batch ? launch_batch(s, launches[i].u, launches[i].plan)
                                 : launch_single(s, launches[i].u);
    for (size_t i = 0; i < launches.size(); ++i)
      if (res[i] != RS_OK) {
        // copies or kernels of the unit may already be queued: let them
        // finish before its pool range and slot are handed out again
        const Lanes ln = lanes_of(s, launches[i].u);
        cudaStreamSynchronize(ln.in);
        cudaStreamSynchronize(ln.cs);
        cudaStreamSynchronize(ln.out);
        cudaGetLastError();
      }
    lk.lock();
    for (size_t i = 0; i < launches.size(); ++i)
      if (res[i] != RS_OK) finish_unit(s, launches[i].u, res[i]);
  }
}

// Streams, events, the pool and the pinned slabs of a server (whichever exist).
void release_cuda(rs_server* s) {
  for (auto* v : {&s->streams, &s->streams_lo})
    for (auto& t : *v)
      if (t) cudaStreamDestroy(t);
  for (auto* v : {&s->ev_in, &s->ev_sorted})
    for (auto& e : *v)
      if (e) cudaEventDestroy(e);
  for (int c = 0; c < 2; ++c) {
    if (s->copy_in[c]) cudaStreamDestroy(s->copy_in[c]);
    if (s->copy_out[c]) cudaStreamDestroy(s->copy_out[c]);
  }
  if (s->pool_base) cudaFree(s->pool_base);
  if (s->status_slab) cudaFreeHost(s->status_slab);
  if (s->off_slab) cudaFreeHost(s->off_slab);
}

}  // namespace

extern "C" {

rs_status rs_server_create(size_t budget_bytes, int streams, rs_server** out) {
  if (!out || budget_bytes < (1u << 20) || streams < 1 || streams > 64) return RS_ERR_INVALID;
  *out = nullptr;
  auto* s = new rs_server;
  cudaGetDevice(&s->device);
  s->budget = budget_bytes;
  if (cudaMalloc(reinterpret_cast<void**>(&s->pool_base), budget_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return RS_ERR_NOMEM;
  }
  s->pool.reset(new Pool(budget_bytes));
  if (cudaHostAlloc(reinterpret_cast<void**>(&s->status_slab), sizeof(uint32_t) * streams,
                    cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(s->pool_base);
    delete s;
    return RS_ERR_NOMEM;
  }
  if (cudaHostAlloc(reinterpret_cast<void**>(&s->off_slab),
                    sizeof(uint64_t) * (kMaxBatchMembers + 1) * streams,
                    cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(s->status_slab);
    cudaFree(s->pool_base);
    delete s;
    return RS_ERR_NOMEM;
  }
  s->streams.assign(streams, nullptr);
  s->streams_lo.assign(streams, nullptr);
  s->stream_busy.assign(streams, 0);
  s->ev_in.assign(streams, nullptr);
  s->ev_sorted.assign(streams, nullptr);
  int least = 0, greatest = 0;  // numerically: greatest < least
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
    cudaGetLastError();
    least = greatest = 0;
  }
  bool ok = true;
  for (int i = 0; i < streams && ok; ++i)
    ok = cudaStreamCreateWithPriority(&s->streams[i], cudaStreamNonBlocking, greatest) ==
             cudaSuccess &&
         cudaStreamCreateWithPriority(&s->streams_lo[i], cudaStreamNonBlocking, least) ==
             cudaSuccess &&
         cudaEventCreateWithFlags(&s->ev_in[i], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&s->ev_sorted[i], cudaEventDisableTiming) == cudaSuccess;
  for (int c = 0; c < 2 && ok; ++c)
    ok = cudaStreamCreateWithFlags(&s->copy_in[c], cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithFlags(&s->copy_out[c], cudaStreamNonBlocking) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    release_cuda(s);
    delete s;
    return RS_ERR_CUDA;
  }
  s->sched = std::thread(scheduler, s);
  *out = s;
  return RS_OK;
}

rs_status rs_server_destroy(rs_server* s) {
  if (!s) return RS_ERR_INVALID;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
    for (uint64_t id : s->pending) {  // never started: cancelled
      auto it = s->reqs.find(id);
      if (it != s->reqs.end()) {
        it->second->state = 2;
        it->second->status = RS_ERR_CANCELLED;
      }
    }
    s->pending.clear();
    s->changes += 1;
  }
  s->cv.notify_all();
  if (s->sched.joinable()) s->sched.join();
  release_cuda(s);
  delete s;
  return RS_OK;
}

rs_status rs_server_get_config(rs_server* s, rs_server_config* out) {
  if (!s || !out) return RS_ERR_INVALID;
  std::lock_guard<std::mutex> g(s->mu);
  out->batch_max_n = s->batch_max_n;
  out->max_batch_keys = s->max_batch_keys;
  out->large_n = s->large_n;
  out->max_large = s->max_large;
  out->large_low_priority = s->large_low_priority;
  out->shared_copy_queues = s->shared_copy_queues;
  return RS_OK;
}

rs_status rs_server_set_config(rs_server* s, const rs_server_config* c) {
  if (!s || !c) return RS_ERR_INVALID;
  if (c->batch_max_n > c->max_batch_keys || c->max_batch_keys > RS_MAX_N || c->large_n == 0 ||
      c->max_large < 1 || c->max_large > 64 ||
      (c->large_low_priority != 0 && c->large_low_priority != 1) ||
      (c->shared_copy_queues != 0 && c->shared_copy_queues != 1))
    return RS_ERR_INVALID;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->batch_max_n = c->batch_max_n;
    s->max_batch_keys = c->max_batch_keys;
    s->large_n = c->large_n;
    s->max_large = c->max_large;
    s->large_low_priority = c->large_low_priority;
    s->shared_copy_queues = c->shared_copy_queues;
    s->changes += 1;  // the scheduler looks at the queue again
  }
  s->cv.notify_all();
  return RS_OK;
}

rs_status rs_submit(rs_server* s, const rs_request* req, rs_handle* out) {
  if (!s || !req || !out || !valid_request(*req)) return RS_ERR_INVALID;
  // whichever way the policy at admission runs it, it must fit the pool
  const size_t need = std::max(single_footprint(*req), plan_batch(*req, req->n, 1).bytes);
  if (need > s->budget) return RS_ERR_INVALID;  // could never be admitted
  auto r = std::make_shared<Request>();
  r->req = *req;
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop) return RS_ERR_BUSY;
    if (s->pending.size() >= (1u << 20)) return RS_ERR_BUSY;
    r->id = s->next_id++;
    if (s->first_submit == 0) s->first_submit = r->t_submit;
    s->reqs[r->id] = r;
    s->pending.push_back(r->id);
    s->changes += 1;
    s->max_queue = std::max(s->max_queue, s->pending.size());
    *out = r->id;
  }
  s->cv.notify_all();
  return RS_OK;
}

rs_status rs_poll(rs_server* s, rs_handle h, int* done) {
  if (!s || !done) return RS_ERR_INVALID;
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(h);
  if (it == s->reqs.end()) return RS_ERR_NOT_FOUND;
  *done = it->second->state == 2;
  if (!*done) return RS_OK;
  const rs_status st = it->second->status;
  s->reqs.erase(it);  // a handle is retired once its completion is reported
  return st;
}

rs_status rs_cancel(rs_server* s, rs_handle h) {
  if (!s) return RS_ERR_INVALID;
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(h);
  if (it == s->reqs.end()) return RS_ERR_NOT_FOUND;
  if (it->second->state != 0) return RS_ERR_BUSY;  // already on the GPU
  auto q = std::find(s->pending.begin(), s->pending.end(), h);
  if (q != s->pending.end()) s->pending.erase(q);
  it->second->state = 2;
  it->second->status = RS_ERR_CANCELLED;
  note_completed(s, h);
  s->changes += 1;
  return RS_OK;
}

rs_status rs_server_completed(rs_server* s, rs_handle* out, size_t cap, size_t* count) {
  if (!s || !count || (cap && !out)) return RS_ERR_INVALID;
  std::lock_guard<std::mutex> g(s->mu);
  size_t k = 0;
  while (k < cap && !s->completed_ids.empty()) {
    out[k++] = s->completed_ids.front();
    s->completed_ids.pop_front();
  }
  *count = k;
  return RS_OK;
}

rs_status rs_server_stats(rs_server* s, rs_server_stats_t* out) {
  if (!s || !out) return RS_ERR_INVALID;
  std::lock_guard<std::mutex> g(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->completed = s->completed;
  out->failed = s->failed;
  out->keys = s->keys_done;
  out->batches = s->batches;
  out->batched_requests = s->batched_requests;
  out->queued = s->pending.size();
  out->max_queued = s->max_queue;
  out->pool_peak_bytes = s->pool->peak();
  out->pool_used_bytes = s->pool->used();
  if (!s->trace.empty()) {
    // percentile p of the interval b - a over the records, in ms
    auto pct = [&](double rs_trace_record::*a, double rs_trace_record::*b, double p) {
      std::vector<double> l;
      l.reserve(s->trace.size());
      for (const auto& r : s->trace) l.push_back(r.*b - r.*a);
      std::sort(l.begin(), l.end());
      const size_t i = std::min(l.size() - 1, size_t(p * double(l.size() - 1) + 0.5));
      return l[i] * 1e3;
    };
    using T = rs_trace_record;
    out->p50_ms = pct(&T::submit_s, &T::done_s, 0.50);
    out->p99_ms = pct(&T::submit_s, &T::done_s, 0.99);
    out->max_ms = pct(&T::submit_s, &T::done_s, 1.0);
    out->wait_p50_ms = pct(&T::submit_s, &T::admit_s, 0.50);
    out->wait_p99_ms = pct(&T::submit_s, &T::admit_s, 0.99);
    out->service_p50_ms = pct(&T::admit_s, &T::done_s, 0.50);
    out->service_p99_ms = pct(&T::admit_s, &T::done_s, 0.99);
  }
  const double span = s->last_done - s->first_submit;
  out->wall_s = span > 0 ? span : 0;
  out->gkeys_per_s = span > 0 ? double(s->keys_done) / span / 1e9 : 0;
  return RS_OK;
}

rs_status rs_server_trace(rs_server* s, rs_trace_record* out, size_t cap, size_t* total) {
  if (!s || !total || (cap && !out)) return RS_ERR_INVALID;
  std::lock_guard<std::mutex> g(s->mu);
  *total = s->trace.size();
  double t0 = s->first_submit;
  if (t0 == 0)
    for (const auto& r : s->trace) t0 = (t0 == 0 || r.submit_s < t0) ? r.submit_s : t0;
  const size_t m = std::min(cap, s->trace.size());
  for (size_t i = 0; i < m; ++i) {
    out[i] = s->trace[i];
    out[i].submit_s -= t0;
    out[i].admit_s -= t0;
    out[i].done_s -= t0;
  }
  return RS_OK;
}

rs_status rs_server_reset_stats(rs_server* s) {
  if (!s) return RS_ERR_INVALID;
  std::lock_guard<std::mutex> g(s->mu);
  s->trace.clear();
  s->completed = s->failed = s->keys_done = s->batches = s->batched_requests = 0;
  s->first_submit = s->last_done = 0;
  s->max_queue = s->pending.size();
  return RS_OK;
}

}  // extern "C"
