// Serving loop: hologram requests admitted by a device-memory budget and
// continuously batched over several streams.
//
// One scheduler thread owns the GPU side.  Requests wait in FIFO order; when
// a stream is free, the scheduler takes requests from the head of the queue
// for as long as their buffers (points, outputs) and the launch's binning
// scratch fit in the free part of one resident device arena, uploads their
// points, runs them as one batch (binning + superposition with the fused
// inverse transform and binarisation, replayed from a CUDA graph per stream)
// and copies their outputs back.  A host callback after the copies marks the
// launch finished; the scheduler then releases its memory, completes its
// requests and starts the next launch.  Requests that arrive while others
// run join the next launch on a free stream, so launches of different
// requests overlap on the device.  Each request's result depends only on its
// own points (per-job amplitude bound, fixed super-tile configuration), so
// it is the same alone and in any mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.cuh"
#include "lut_object.h"

using namespace wsb;

namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over the offsets of one device allocation; free blocks
// are kept sorted by offset and merged with their neighbours on release.
class Arena {
 public:
  explicit Arena(size_t size) : size_(size) { free_[0] = size; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = granule(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t o = it->first, rest = it->second - bytes;
      free_.erase(it);
      if (rest) free_[o + bytes] = rest;
      *off = o;
      used_ += bytes;
      peak_ = std::max(peak_, used_);
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = granule(bytes);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  static size_t granule(size_t b) { return align_up(std::max<size_t>(b, 1), 256); }
  size_t size() const { return size_; }
  size_t peak() const { return peak_; }

 private:
  size_t size_, used_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_;
};

struct Request {
  int64_t id = 0;
  wasabi_request r{};
  double t_submit = 0, t_launch = -1, t_done = -1;
  int batch_jobs = 0;
  int status = WASABI_OK;
  bool done = false;
  size_t off_pts = 0, off_bits = 0, off_u = 0;
  size_t sz_pts = 0, sz_bits = 0, sz_u = 0;
};

struct Launch {
  wasabi_server* server = nullptr;
  std::vector<Request*> reqs;
  size_t off_scratch = 0, sz_scratch = 0;
  bool busy = false;
  bool finished = false;  // set by the host callback
  double t_done = 0;
};

}  // namespace

struct wasabi_server {
  const wasabi_lut* lut = nullptr;
  int device = 0;
  char* arena_base = nullptr;
  Arena* arena = nullptr;
  int max_batch = 1;
  std::vector<cudaStream_t> streams;
  std::vector<wasabi_batch*> batches;
  std::vector<Launch> launches;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<Request*> pending;
  std::map<int64_t, Request*> reqs;
  int64_t next_id = 1;
  int64_t completed = 0, nlaunch = 0;
  bool stop = false;
  bool blocked = false;  // the queue head waits for memory: retry after a launch retires
  std::thread th;
  Clock::time_point epoch;

  double now() const { return std::chrono::duration<double>(Clock::now() - epoch).count(); }
  void run();
  bool fits_alone(const Request& q) const;
  void release(Request* q);
};

namespace {

void CUDART_CB on_launch_done(void* p) {
  Launch* L = static_cast<Launch*>(p);
  wasabi_server* s = L->server;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    L->t_done = s->now();
    L->finished = true;
  }
  s->cv_sched.notify_one();
}

size_t bits_bytes(const wasabi_request& r) { return ((size_t)r.holo_w * r.holo_h + 7) / 8; }
size_t u_bytes(const wasabi_request& r) { return (size_t)r.holo_w * r.holo_h * sizeof(float2); }

}  // namespace

// Scratch of one job in a batch (the batch API's own sizing).
static size_t job_scratch_bytes(const wasabi_batch* b, const wasabi_request& r, char* dummy_pts) {
  wasabi_job j{};
  j.points_dev = reinterpret_cast<const wasabi_point*>(dummy_pts);
  j.n = r.n;
  j.holo_w = r.holo_w;
  j.holo_h = r.holo_h;
  size_t bytes = 0;
  wasabi_batch_scratch_bytes(b, &j, 1, &bytes);
  return bytes;
}

bool wasabi_server::fits_alone(const Request& q) const {
  const size_t need = Arena::granule(q.sz_pts) + Arena::granule(q.sz_bits) + Arena::granule(q.sz_u) +
                      Arena::granule(job_scratch_bytes(batches[0], q.r, arena_base));
  return need <= arena->size();
}

void wasabi_server::release(Request* q) {
  if (q->sz_pts) arena->release(q->off_pts, q->sz_pts);
  if (q->sz_bits) arena->release(q->off_bits, q->sz_bits);
  if (q->sz_u) arena->release(q->off_u, q->sz_u);
}

void wasabi_server::run() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    // Retire finished launches.
    for (Launch& L : launches) {
      if (!L.busy || !L.finished) continue;
      for (Request* q : L.reqs) {
        release(q);
        q->t_done = L.t_done;
        q->done = true;
        ++completed;
      }
      arena->release(L.off_scratch, L.sz_scratch);
      blocked = false;
      L.reqs.clear();
      L.busy = false;
      L.finished = false;
      cv_done.notify_all();
    }
    bool any_busy = false;
    for (const Launch& L : launches) any_busy = any_busy || L.busy;
    if (stop && !any_busy) break;

    // Start launches on free streams.
    for (size_t si = 0; si < launches.size() && !pending.empty() && !stop && !blocked; ++si) {
      Launch& L = launches[si];
      if (L.busy) continue;
      // Admit from the head of the queue while buffers and scratch fit.
      std::vector<Request*> take;
      size_t scratch = 0;
      while (!pending.empty() && (int)take.size() < max_batch) {
        Request* q = pending.front();
        const size_t js = job_scratch_bytes(batches[si], q->r, arena_base);
        bool ok = q->sz_pts == 0 || arena->alloc(q->sz_pts, &q->off_pts);
        bool okb = ok && (q->sz_bits == 0 || arena->alloc(q->sz_bits, &q->off_bits));
        bool oku = okb && (q->sz_u == 0 || arena->alloc(q->sz_u, &q->off_u));
        // The launch's scratch is allocated last; keep room for it.
        size_t probe = 0;
        const bool oks = oku && arena->alloc(scratch + js, &probe);
        if (oks) arena->release(probe, scratch + js);
        if (!oks) {
          if (oku && q->sz_u) arena->release(q->off_u, q->sz_u);
          if (okb && q->sz_bits) arena->release(q->off_bits, q->sz_bits);
          if (ok && q->sz_pts) arena->release(q->off_pts, q->sz_pts);
          break;
        }
        take.push_back(q);
        scratch += js;
        pending.pop_front();
      }
      if (take.empty()) {  // the head waits for memory to free up
        blocked = true;
        break;
      }
      const bool got = arena->alloc(scratch, &L.off_scratch);
      if (!got) {  // cannot happen after the probe above; fail safe
        for (auto it = take.rbegin(); it != take.rend(); ++it) {
          release(*it);
          pending.push_front(*it);
        }
        break;
      }
      L.sz_scratch = scratch;
      L.reqs = take;
      L.busy = true;
      L.finished = false;
      const double t = now();
      for (Request* q : take) {
        q->t_launch = t;
        q->batch_jobs = (int)take.size();
      }
      ++nlaunch;
      // Enqueue without the lock: uploads, the batch, downloads, callback.
      lk.unlock();
      const cudaStream_t s = streams[si];
      std::vector<wasabi_job> jobs(take.size());
      cudaError_t e = cudaSuccess;
      for (size_t i = 0; i < take.size() && e == cudaSuccess; ++i) {
        const Request* q = take[i];
        wasabi_job& j = jobs[i];
        j.points_dev = reinterpret_cast<const wasabi_point*>(arena_base + q->off_pts);
        j.n = q->r.n;
        j.holo_w = q->r.holo_w;
        j.holo_h = q->r.holo_h;
        j.rule = q->r.rule;
        j.wbuf_dev = nullptr;
        j.u_dev = q->sz_u ? arena_base + q->off_u : nullptr;
        j.bits_dev = q->sz_bits ? reinterpret_cast<uint8_t*>(arena_base + q->off_bits) : nullptr;
        j.frame = q->r.frame;
        if (q->r.n > 0)
          e = cudaMemcpyAsync(arena_base + q->off_pts, q->r.points_host, q->sz_pts, cudaMemcpyHostToDevice, s);
      }
      wasabi_status st = WASABI_OK;
      if (e == cudaSuccess)
        st = wasabi_batch_run(batches[si], jobs.data(), (int)jobs.size(), arena_base + L.off_scratch, scratch, s);
      for (size_t i = 0; i < take.size() && e == cudaSuccess && st == WASABI_OK; ++i) {
        const Request* q = take[i];
        if (q->sz_bits)
          e = cudaMemcpyAsync(q->r.bits_host, arena_base + q->off_bits, q->sz_bits, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && q->sz_u)
          e = cudaMemcpyAsync(q->r.u_host, arena_base + q->off_u, q->sz_u, cudaMemcpyDeviceToHost, s);
      }
      if (e == cudaSuccess && st == WASABI_OK) e = cudaLaunchHostFunc(s, on_launch_done, &L);
      lk.lock();
      if (e != cudaSuccess || st != WASABI_OK) {
        // Nothing was left waiting on the callback: finish the launch here
        // once the stream has drained.
        lk.unlock();
        cudaStreamSynchronize(s);
        lk.lock();
        for (Request* q : take) q->status = st != WASABI_OK ? st : WASABI_E_CUDA;
        L.t_done = now();
        L.finished = true;
      }
    }
    // Sleep until a callback, a submission or shutdown.
    cv_sched.wait_for(lk, std::chrono::milliseconds(2), [&] {
      if (stop) return true;
      for (const Launch& L : launches)
        if (L.busy && L.finished) return true;
      if (pending.empty() || blocked) return false;
      for (const Launch& L : launches)
        if (!L.busy) return true;
      return false;
    });
  }
  // Shutdown: requests still queued are cancelled.
  for (Request* q : pending) {
    q->status = WASABI_E_INVALID;
    q->done = true;
  }
  pending.clear();
  cv_done.notify_all();
}

extern "C" {

wasabi_status wasabi_server_create(const wasabi_lut* lut, size_t hbm_budget_bytes, int streams, int max_batch,
                                   int holo_side_hint, wasabi_server** out) {
  if (!lut || !out || streams < 1 || streams > 16 || max_batch < 1 || max_batch > kMaxJobs ||
      hbm_budget_bytes < (1u << 20)) {
    set_error("server_create: need a LUT, 1..16 streams, 1..%d jobs per launch and a budget >= 1 MiB", kMaxJobs);
    return WASABI_E_INVALID;
  }
  if (lut->L < 2) { set_error("server_create: the fused inverse needs levels >= 2"); return WASABI_E_INVALID; }
  if (lut->wavelet != WASABI_HAAR) { set_error("server_create: the fused inverse is Haar's"); return WASABI_E_INVALID; }
  *out = nullptr;
  int* status;
  int sms;
  if (!device_info(&status, &sms)) return WASABI_E_CUDA;
  wasabi_server* s = new wasabi_server;
  s->lut = lut;
  cudaGetDevice(&s->device);
  s->max_batch = max_batch;
  cudaError_t e = cudaMalloc(&s->arena_base, hbm_budget_bytes);
  if (e != cudaSuccess) {
    delete s;
    set_error("server_create: cannot reserve %zu bytes: %s", hbm_budget_bytes, cudaGetErrorString(e));
    return WASABI_E_NOMEM;
  }
  s->arena = new Arena(hbm_budget_bytes);
  s->launches = std::vector<Launch>(streams);
  for (int i = 0; i < streams; ++i) {
    cudaStream_t st = nullptr;
    wasabi_batch* b = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    wasabi_status bs = e == cudaSuccess ? wasabi_batch_create(lut, max_batch, holo_side_hint, 1, &b) : WASABI_E_CUDA;
    if (e != cudaSuccess || bs != WASABI_OK) {
      if (st) cudaStreamDestroy(st);
      for (size_t k = 0; k < s->streams.size(); ++k) {
        wasabi_batch_destroy(s->batches[k]);
        cudaStreamDestroy(s->streams[k]);
      }
      cudaFree(s->arena_base);
      delete s->arena;
      delete s;
      if (e != cudaSuccess) return cuda_fail("server_create: stream", e);
      return bs;
    }
    s->streams.push_back(st);
    s->batches.push_back(b);
    s->launches[i].server = s;
  }
  s->epoch = Clock::now();
  s->th = std::thread([s] { s->run(); });
  *out = s;
  return WASABI_OK;
}

wasabi_status wasabi_server_submit(wasabi_server* s, const wasabi_request* r, int64_t* id_out) {
  if (!s || !r || !id_out || r->n < 0 || (r->n > 0 && !r->points_host) || (!r->bits_host && !r->u_host)) {
    set_error("server_submit: need points (if n > 0) and at least one output");
    return WASABI_E_INVALID;
  }
  const int ts = 1 << s->lut->L;
  if (r->holo_w < ts || r->holo_h < ts || r->holo_w % ts || r->holo_h % ts || (r->bits_host && r->holo_w % 8) ||
      (r->rule != WASABI_SHIFT_FLOOR && r->rule != WASABI_SHIFT_NEAREST)) {
    set_error("server_submit: holo_w, holo_h must be multiples of 2^L = %d (holo_w %% 8 == 0 for bits)", ts);
    return WASABI_E_INVALID;
  }
  {
    int ox, oy;
    RefDev ref;
    const char* why = "";
    if (!frame_to_dev(&r->frame, &ox, &oy, &ref, &why)) {
      set_error("server_submit: %s", why);
      return WASABI_E_INVALID;
    }
  }
  // Depth indices are checked here, on the host, so that a bad request is
  // refused on its own instead of flagging the shared device status word.
  for (int64_t i = 0; i < r->n; ++i) {
    if (r->points_host[i].d >= (uint32_t)s->lut->D) {
      set_error("server_submit: point %lld has depth index %u >= %d", (long long)i, r->points_host[i].d, s->lut->D);
      return WASABI_E_RANGE;
    }
  }
  Request* q = new Request;
  q->r = *r;
  q->sz_pts = (size_t)r->n * sizeof(wasabi_point);
  q->sz_bits = r->bits_host ? bits_bytes(*r) : 0;
  q->sz_u = r->u_host ? u_bytes(*r) : 0;
  if (!s->fits_alone(*q)) {
    delete q;
    set_error("server_submit: the request alone needs more than the server's device-memory budget");
    return WASABI_E_NOMEM;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      delete q;
      set_error("server_submit: server is shutting down");
      return WASABI_E_INVALID;
    }
    q->id = s->next_id++;
    q->t_submit = s->now();
    s->reqs[q->id] = q;
    s->pending.push_back(q);
    *id_out = q->id;
  }
  s->cv_sched.notify_one();
  return WASABI_OK;
}

wasabi_status wasabi_server_wait(wasabi_server* s, int64_t id, double timeout_s, wasabi_request_info* info) {
  if (!s) { set_error("server_wait: NULL server"); return WASABI_E_INVALID; }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) { set_error("server_wait: unknown request %lld", (long long)id); return WASABI_E_INVALID; }
  Request* q = it->second;
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9));
  if (!s->cv_done.wait_until(lk, deadline, [&] { return q->done; })) {
    set_error("server_wait: request %lld not finished in time", (long long)id);
    return WASABI_E_TIMEOUT;
  }
  if (info) {
    info->submit_s = q->t_submit;
    info->launch_s = q->t_launch;
    info->done_s = q->t_done;
    info->batch_jobs = q->batch_jobs;
    info->status = q->status;
  }
  const int st = q->status;
  s->reqs.erase(it);
  delete q;
  if (st != WASABI_OK) set_error("server_wait: request %lld failed", (long long)id);
  return (wasabi_status)st;
}

wasabi_status wasabi_server_stats(wasabi_server* s, size_t* peak_bytes, int64_t* completed, int64_t* launches) {
  if (!s) { set_error("server_stats: NULL server"); return WASABI_E_INVALID; }
  std::lock_guard<std::mutex> lk(s->mu);
  if (peak_bytes) *peak_bytes = s->arena->peak();
  if (completed) *completed = s->completed;
  if (launches) *launches = s->nlaunch;
  return WASABI_OK;
}

wasabi_status wasabi_server_destroy(wasabi_server* s) {
  if (!s) return WASABI_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_sched.notify_one();
  if (s->th.joinable()) s->th.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  for (size_t k = 0; k < s->streams.size(); ++k) {
    cudaStreamSynchronize(s->streams[k]);
    wasabi_batch_destroy(s->batches[k]);
    cudaStreamDestroy(s->streams[k]);
  }
  cudaFree(s->arena_base);
  cudaSetDevice(prev);
  cudaGetLastError();
  for (auto& kv : s->reqs) delete kv.second;
  delete s->arena;
  delete s;
  return WASABI_OK;
}

}  // extern "C"
