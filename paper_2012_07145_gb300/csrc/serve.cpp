// Serving loop: continuous batching of pipeline requests on one GPU.
//
// Requests (a pipeline, input buffers, an output buffer) arrive at any time
// through hp_server_submit (host buffers) or hp_server_submit_device (device
// buffers).  A worker thread admits them in arrival order as soon as a slot (a
// CUDA stream) and device memory are free.  Admitted work runs concurrently on
// the slots' streams, so a request that arrives while others are on the GPU
// overlaps with them.
//
// Batching: up to max_batch queued requests for the same pipeline, image size
// and buffer kind are served by one realize of a batched copy of the pipeline,
// which launches each kernel once for the whole batch: their images are
// stacked as planes of one buffer.  Pipelines whose stages all act on each
// channel separately (stencils, per-channel point-wise ops, resampling) simply
// see more channels; the fused Harris and histogram-equalization kernels take
// the batch as an image index (each image keeps its own planes, and for the
// histogram its own counters and table).  The kernels of a batch are
// persistent: one grid sized to the GPU walks every image's work units.
//
// Residency: each slot keeps, per (pipeline, batch size, image size), a
// staging region in the HBM arena reserved at creation, and keeps it after
// the request completes, so later requests of that shape reuse the same device
// addresses.  That makes every slot's realize of a shape a CUDA graph after its
// second use (the slots' pipeline copies replay their launch sequence as a
// graph per set of buffer addresses).  Admission is by HBM footprint: a region
// is taken from the arena first-fit; when the arena is full, the least
// recently used regions of idle slots are given back first.  A device request
// served alone needs no staging at all: the realize runs on the caller's
// buffers.  Each slot keeps its own copies of the pipelines it runs, so
// concurrent requests never share a pipeline's scratch.  Latency is measured
// from submit to the completion the worker observes.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "arena.h"
#include "hp_internal.h"

namespace hp {
// Provided by pipeline.cpp.
hp_pipeline* clone_pipeline(const hp_pipeline* p, int batch);
bool pipeline_batch_ok(const hp_pipeline* p, const int* widths, const int* heights, int n_inputs, int batch);
unsigned long long pipeline_graph_replays(const hp_pipeline* p);
hp_status pipeline_output_shape(hp_pipeline* p, const int* widths, const int* heights, int n_inputs, int* w, int* h,
                                int* channels, int* dtype);
}  // namespace hp

namespace {

using Clock = std::chrono::steady_clock;

constexpr long long kBatchBytesMax = 32LL << 20;  // largest batch (inputs + outputs of all its requests)

int dtype_size(int d) { return d == HP_U8 ? 1 : (d == HP_U16 || d == HP_F16 || d == HP_BF16) ? 2 : 4; }
using hp::Arena;
long long r256(long long v) { return hp::round256(v); }

struct Request {
  unsigned long long ticket = 0;
  hp_pipeline* p = nullptr;
  std::vector<hp_buffer> in;
  hp_buffer out{};
  bool device = false;  // buffers in device memory (no host copies)
  Clock::time_point t_submit;
};

// A slot's staging region for one request shape and batch size.
struct Resident {
  long long off = 0, bytes = 0;
  unsigned long long last = 0;  // admission counter at its last use
};

typedef std::vector<long long> ShapeKey;  // pipeline, batch, buffer kind, every buffer's size / type / channels

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  std::vector<Request*> batch;
  Resident* cur = nullptr;  // staging of the batch in flight (null: a device request served in place)
  std::map<ShapeKey, Resident> resident;
  std::map<std::pair<hp_pipeline*, int>, hp_pipeline*> clones;
};

struct Result {
  hp_status status;
  double latency_us;
};

}  // namespace

struct hp_server {
  Arena arena;
  std::vector<Slot> slots;
  int max_batch = 1;
  std::deque<Request*> queue;
  std::map<unsigned long long, Result> results;
  std::vector<double> latencies;
  std::map<std::vector<long long>, bool> batch_ok;  // (pipeline, input sizes) -> batchable
  std::mutex mu;
  std::mutex clone_mu;  // the slots' pipeline copies (the worker and hp_server_prepare)
  std::condition_variable cv_done, cv_work;
  std::thread worker;
  bool stop = false;
  unsigned long long next_ticket = 1, submitted = 0, completed = 0, failed = 0, batched = 0, admissions = 0;
  unsigned long long device_requests = 0, evictions = 0;
  double mpix = 0;
  Clock::time_point t_first, t_last;
  bool any = false;
  int device = 0;
};

namespace {

long long buffer_bytes(const hp_buffer& x) { return r256((long long)x.width * dtype_size(x.dtype)) * x.height * x.channels; }

// Staging footprint of `batch` requests of r's shape: every input and the
// output, packed.
long long staging_bytes(const Request& r, int batch) {
  long long b = 0;
  for (const hp_buffer& x : r.in) b += r256(buffer_bytes(x) * batch);
  return b + r256(buffer_bytes(r.out) * batch);
}

bool same_shape(const Request& a, const Request& b) {
  if (a.p != b.p || a.device != b.device || a.in.size() != b.in.size()) return false;
  for (size_t i = 0; i < a.in.size(); ++i)
    if (a.in[i].width != b.in[i].width || a.in[i].height != b.in[i].height || a.in[i].dtype != b.in[i].dtype ||
        a.in[i].channels != b.in[i].channels)
      return false;
  return a.out.width == b.out.width && a.out.height == b.out.height && a.out.channels == b.out.channels &&
         a.out.dtype == b.out.dtype;
}

ShapeKey shape_key(const Request& r, int batch) {
  ShapeKey k{(long long)(uintptr_t)r.p, batch, r.device ? 1 : 0};
  for (const hp_buffer& b : r.in) k.insert(k.end(), {b.width, b.height, b.channels, b.dtype});
  k.insert(k.end(), {r.out.width, r.out.height, r.out.channels, r.out.dtype});
  return k;
}

// The slot's copy of p for batches of `batch` (made on first use); the caller
// holds clone_mu.
hp_pipeline* slot_clone(Slot& sl, hp_pipeline* p, int batch) {
  auto key = std::make_pair(p, batch);
  auto it = sl.clones.find(key);
  if (it != sl.clones.end()) return it->second;
  hp_pipeline* c = hp::clone_pipeline(p, batch);
  if (c) hp_set_option(c, HP_OPT_CUDA_GRAPH, 1);  // a slot's realize of a shape replays as a graph
  sl.clones[key] = c;
  return c;
}

// Whether requests of r's pipeline and input sizes may share a realize
// (computed once per pipeline and sizes; called with the server lock held).
bool batchable(hp_server* s, const Request& r) {
  std::vector<long long> k{(long long)(uintptr_t)r.p};
  std::vector<int> ws, hs;
  for (const hp_buffer& b : r.in) {
    k.push_back(b.width);
    k.push_back(b.height);
    ws.push_back(b.width);
    hs.push_back(b.height);
  }
  auto it = s->batch_ok.find(k);
  if (it != s->batch_ok.end()) return it->second;
  const bool ok = hp::pipeline_batch_ok(r.p, ws.data(), hs.data(), (int)ws.size(), 2);
  s->batch_ok[k] = ok;
  return ok;
}

// Gives back the least recently used staging region of an idle slot; false
// when there is none.
bool evict_one(hp_server* s) {
  Slot* best_slot = nullptr;
  std::map<ShapeKey, Resident>::iterator best;
  for (Slot& sl : s->slots) {
    if (sl.busy) continue;
    for (auto it = sl.resident.begin(); it != sl.resident.end(); ++it)
      if (!best_slot || it->second.last < best->second.last) {
        best_slot = &sl;
        best = it;
      }
  }
  if (!best_slot) return false;
  s->arena.release(best->second.off, best->second.bytes);
  best_slot->resident.erase(best);
  ++s->evictions;
  return true;
}

// Device layout of a batch in its staging region: for each input i, B stacked
// images of C_i planes; then the output, B stacked images.  Row stride is the
// packed width rounded to 16 bytes.
void staging_layout(char* dev, const Request& r0, int B, std::vector<hp_buffer>& din, hp_buffer& dout) {
  din.resize(r0.in.size());
  long long pos = 0;
  for (size_t i = 0; i < r0.in.size(); ++i) {
    const hp_buffer& h = r0.in[i];
    hp_buffer d = h;
    d.data = dev + pos;
    d.row_stride_bytes = (((long long)h.width * dtype_size(h.dtype)) + 15) / 16 * 16;
    d.plane_stride_bytes = d.row_stride_bytes * h.height;
    d.channels = h.channels * B;
    din[i] = d;
    pos += r256(d.plane_stride_bytes * d.channels);
  }
  dout = r0.out;
  dout.data = dev + pos;
  dout.row_stride_bytes = (((long long)r0.out.width * dtype_size(r0.out.dtype)) + 15) / 16 * 16;
  dout.plane_stride_bytes = dout.row_stride_bytes * r0.out.height;
  dout.channels = r0.out.channels * B;
}

// Runs a staged batch: copies in, the realize, copies out.  A device request
// served alone runs in place.
hp_status launch_batch(hp_server* s, Slot& sl) {
  const int B = (int)sl.batch.size();
  const Request& r0 = *sl.batch[0];
  cudaStream_t st = sl.stream;
  std::lock_guard<std::mutex> ck(s->clone_mu);  // hp_server_prepare may touch this slot's copies
  hp_pipeline* p = slot_clone(sl, r0.p, B);
  if (!p) return hp::report_error(HP_ERR_INVALID_ARG, "server: pipeline cannot be copied");
  if (!sl.cur) {  // a device request alone: its own buffers
    hp_status rs = hp_realize(p, r0.in.data(), (int)r0.in.size(), &r0.out, st);
    if (rs) return rs;
    if (cudaEventRecord(sl.done, st)) return hp::report_error(HP_ERR_CUDA, "server: event record failed");
    return HP_OK;
  }
  const cudaMemcpyKind to_dev = r0.device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind from_dev = r0.device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  std::vector<hp_buffer> din;
  hp_buffer dout;
  staging_layout(s->arena.base + sl.cur->off, r0, B, din, dout);
  for (int j = 0; j < B; ++j) {
    const Request& r = *sl.batch[j];
    for (size_t i = 0; i < r.in.size(); ++i) {
      const hp_buffer& h = r.in[i];
      for (int c = 0; c < h.channels; ++c) {
        char* dst = (char*)din[i].data + (long long)(j * h.channels + c) * din[i].plane_stride_bytes;
        const char* src = (const char*)h.data + (long long)c * h.plane_stride_bytes;
        if (cudaMemcpy2DAsync(dst, din[i].row_stride_bytes, src, h.row_stride_bytes,
                              (size_t)h.width * dtype_size(h.dtype), h.height, to_dev, st))
          return hp::report_error(HP_ERR_CUDA, "server: copy of an input into staging failed");
      }
    }
  }
  hp_status rs = hp_realize(p, din.data(), (int)din.size(), &dout, st);
  if (rs) return rs;
  for (int j = 0; j < B; ++j) {
    const hp_buffer& h = sl.batch[j]->out;
    for (int c = 0; c < h.channels; ++c) {
      const char* src = (const char*)dout.data + (long long)(j * h.channels + c) * dout.plane_stride_bytes;
      char* dst = (char*)h.data + (long long)c * h.plane_stride_bytes;
      if (cudaMemcpy2DAsync(dst, h.row_stride_bytes, src, dout.row_stride_bytes, (size_t)h.width * dtype_size(h.dtype),
                            h.height, from_dev, st))
        return hp::report_error(HP_ERR_CUDA, "server: copy of an output from staging failed");
    }
  }
  if (cudaEventRecord(sl.done, st)) return hp::report_error(HP_ERR_CUDA, "server: event record failed");
  return HP_OK;
}

void finish_slot(hp_server* s, Slot& sl, hp_status st) {
  const auto now = Clock::now();
  for (Request* r : sl.batch) {
    double us = std::chrono::duration<double, std::micro>(now - r->t_submit).count();
    s->results[r->ticket] = Result{st, us};
    if (st == HP_OK) {
      ++s->completed;
      s->latencies.push_back(us);
      s->mpix += (double)r->out.width * r->out.height / 1e6;
    } else {
      ++s->failed;
    }
    delete r;
  }
  if (sl.batch.size() > 1) ++s->batched;
  sl.batch.clear();
  sl.cur = nullptr;  // the staging region stays resident for the next request of its shape
  sl.busy = false;
  s->t_last = now;
}

// Admits the request at the head of the queue (with the same-shape requests
// that may join it) onto a free slot; returns the slot, or null when no slot
// or memory is free (the request stays queued).  Called with the lock held.
Slot* admit(hp_server* s) {
  Request* head = s->queue.front();
  std::vector<size_t> pick{0};
  // only requests of modest size are batched, and a batch holds at most
  // kBatchBytesMax: a large request already fills the GPU on its own, and a
  // batch makes each request wait for every other one's copies
  if (s->max_batch > 1 && staging_bytes(*head, 2) <= kBatchBytesMax && batchable(s, *head)) {
    for (size_t i = 1; i < s->queue.size() && (int)pick.size() < s->max_batch && i < 64 &&
                       staging_bytes(*head, (int)pick.size() + 1) <= kBatchBytesMax;
         ++i)
      if (same_shape(*head, *s->queue[i])) pick.push_back(i);
  }
  while (true) {
    const int B = (int)pick.size();
    const ShapeKey key = shape_key(*head, B);
    const bool staged = !(head->device && B == 1);
    // a free slot, preferably one that keeps this shape resident
    Slot* slot = nullptr;
    for (Slot& sl : s->slots) {
      if (sl.busy) continue;
      if (!slot) slot = &sl;
      if (staged && sl.resident.count(key)) {
        slot = &sl;
        break;
      }
    }
    if (!slot) return nullptr;
    Resident* region = nullptr;
    if (staged) {
      auto it = slot->resident.find(key);
      if (it != slot->resident.end()) {
        region = &it->second;
      } else {
        const long long bytes = staging_bytes(*head, B);
        long long off = 0;
        bool ok = s->arena.alloc(bytes, &off);
        while (!ok && evict_one(s)) ok = s->arena.alloc(bytes, &off);
        if (!ok) {
          if (B > 1) {  // the head alone may still fit
            pick.resize(1);
            continue;
          }
          return nullptr;
        }
        Resident& r = slot->resident[key];
        r.off = off;
        r.bytes = bytes;
        region = &r;
      }
      region->last = ++s->admissions;
    }
    slot->batch.clear();
    for (size_t i : pick) slot->batch.push_back(s->queue[i]);
    for (size_t k = pick.size(); k-- > 0;) s->queue.erase(s->queue.begin() + pick[k]);
    slot->cur = region;
    slot->busy = true;
    return slot;
  }
}

void worker_loop(hp_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    bool progress = false;
    // completions
    for (Slot& sl : s->slots) {
      if (!sl.busy || sl.batch.empty()) continue;
      cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      finish_slot(s, sl, q == cudaSuccess ? HP_OK : HP_ERR_CUDA);
      progress = true;
    }
    if (progress) s->cv_done.notify_all();
    // admissions, in arrival order; the copies and launches are enqueued
    // without the lock, so submitters and waiters are not held up
    while (!s->queue.empty()) {
      Slot* sl = admit(s);
      if (!sl) break;
      lk.unlock();
      hp_status st = launch_batch(s, *sl);
      if (st) {
        cudaStreamSynchronize(sl->stream);
        cudaGetLastError();
      }
      lk.lock();
      if (st) {
        finish_slot(s, *sl, st);
        s->cv_done.notify_all();
      }
      progress = true;
    }
    bool idle = s->queue.empty();
    for (Slot& sl : s->slots) idle &= !sl.busy;
    if (s->stop && idle) break;
    if (!progress) {
      // nothing to do right now: sleep briefly (new work wakes us at once)
      s->cv_work.wait_for(lk, std::chrono::microseconds(idle ? 2000 : 20));
    }
  }
}

hp_status submit(hp_server* s, hp_pipeline* p, const hp_buffer* inputs, int n_inputs, const hp_buffer* output,
                 unsigned long long* ticket, bool device) {
  if (!s || !p || !inputs || n_inputs < 1 || n_inputs > 16 || !output || !ticket)
    return hp::report_error(HP_ERR_INVALID_ARG, "hp_server_submit: bad arguments");
  auto* r = new Request();
  r->p = p;
  r->device = device;
  r->in.assign(inputs, inputs + n_inputs);
  r->out = *output;
  for (const hp_buffer& b : r->in)
    if (!b.data || b.width < 1 || b.height < 1 || b.channels < 1) {
      delete r;
      return hp::report_error(HP_ERR_INVALID_ARG, "hp_server_submit: empty input buffer");
    }
  if (!r->out.data || r->out.width < 1 || r->out.height < 1 || r->out.channels < 1) {
    delete r;
    return hp::report_error(HP_ERR_INVALID_ARG, "hp_server_submit: empty output buffer");
  }
  if (staging_bytes(*r, 1) > s->arena.size) {
    delete r;
    return hp::report_error(HP_ERR_OOM, "hp_server_submit: request larger than the whole HBM budget");
  }
  std::lock_guard<std::mutex> lk(s->mu);
  r->t_submit = Clock::now();
  if (!s->any) {
    s->t_first = r->t_submit;
    s->any = true;
  }
  r->ticket = s->next_ticket++;
  *ticket = r->ticket;
  ++s->submitted;
  if (device) ++s->device_requests;
  s->queue.push_back(r);
  s->cv_work.notify_one();
  return HP_OK;
}

}  // namespace

extern "C" {

hp_status hp_server_create(hp_server** out, long long hbm_budget_bytes, int slots, int max_batch) {
  if (!out || hbm_budget_bytes < (1 << 20) || slots < 1 || slots > 64 || max_batch < 1 || max_batch > 64)
    return hp::report_error(HP_ERR_INVALID_ARG, "hp_server_create: bad arguments");
  auto* s = new hp_server();
  cudaGetDevice(&s->device);
  void* base = nullptr;
  if (cudaMalloc(&base, (size_t)hbm_budget_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return hp::report_error(HP_ERR_OOM, "hp_server_create: cannot reserve the HBM budget");
  }
  s->arena.init((char*)base, hbm_budget_bytes);
  s->slots.resize(slots);
  for (Slot& sl : s->slots) {
    const cudaError_t e1 = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    const cudaError_t e2 = e1 == cudaSuccess ? cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) : e1;
    if (e2 != cudaSuccess) {  // undo what was created so far
      cudaGetLastError();
      for (Slot& o : s->slots) {
        if (o.stream) cudaStreamDestroy(o.stream);
        if (o.done) cudaEventDestroy(o.done);
      }
      cudaFree(base);
      delete s;
      char msg[160];
      snprintf(msg, sizeof msg, "hp_server_create: stream or event creation failed: %s", cudaGetErrorString(e2));
      return hp::report_error(HP_ERR_CUDA, msg);
    }
  }
  s->max_batch = max_batch;
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return HP_OK;
}

hp_status hp_server_submit(hp_server* s, hp_pipeline* p, const hp_buffer* inputs, int n_inputs,
                           const hp_buffer* output, unsigned long long* ticket) {
  return submit(s, p, inputs, n_inputs, output, ticket, false);
}

hp_status hp_server_submit_device(hp_server* s, hp_pipeline* p, const hp_buffer* inputs, int n_inputs,
                                  const hp_buffer* output, unsigned long long* ticket) {
  return submit(s, p, inputs, n_inputs, output, ticket, true);
}

hp_status hp_server_wait(hp_server* s, unsigned long long ticket, int timeout_ms, double* latency_us) {
  if (!s) return hp::report_error(HP_ERR_INVALID_ARG, "hp_server_wait: null server");
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
  while (s->results.find(ticket) == s->results.end()) {
    if (ticket == 0 || ticket >= s->next_ticket) return hp::report_error(HP_ERR_INVALID_ARG, "unknown ticket");
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout &&
        s->results.find(ticket) == s->results.end())
      return hp::report_error(HP_ERR_TIMEOUT, "hp_server_wait: request not complete within the timeout");
  }
  Result r = s->results[ticket];
  if (latency_us) *latency_us = r.latency_us;
  return r.status;
}

hp_status hp_server_stats_get(hp_server* s, hp_server_stats* st) {
  if (!s || !st) return hp::report_error(HP_ERR_INVALID_ARG, "hp_server_stats_get: null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  memset(st, 0, sizeof *st);
  st->submitted = s->submitted;
  st->completed = s->completed;
  st->failed = s->failed;
  st->batched_launches = s->batched;
  st->peak_bytes = (unsigned long long)s->arena.peak;
  st->mpix = s->mpix;
  st->device_requests = s->device_requests;
  st->evictions = s->evictions;
  {
    std::lock_guard<std::mutex> ck(s->clone_mu);
    for (Slot& sl : s->slots) {
      for (auto& kv : sl.clones) st->graph_replays += hp::pipeline_graph_replays(kv.second);
      for (auto& kv : sl.resident) st->resident_bytes += (unsigned long long)kv.second.bytes;
    }
  }
  if (s->any) st->busy_s = std::chrono::duration<double>(s->t_last - s->t_first).count();
  if (!s->latencies.empty()) {
    std::vector<double> v = s->latencies;
    std::sort(v.begin(), v.end());
    auto q = [&](double f) { return v[std::min(v.size() - 1, (size_t)(f * (v.size() - 1) + 0.5))]; };
    st->p50_us = q(0.50);
    st->p99_us = q(0.99);
    st->max_us = v.back();
    double sum = 0;
    for (double x : v) sum += x;
    st->mean_us = sum / v.size();
  }
  return HP_OK;
}

hp_status hp_server_prepare(hp_server* s, hp_pipeline* p, const hp_buffer* inputs, int n_inputs) {
  if (!s || !p || !inputs || n_inputs < 1 || n_inputs > 16)
    return hp::report_error(HP_ERR_INVALID_ARG, "hp_server_prepare: bad arguments");
  std::vector<int> ws(n_inputs), hs(n_inputs);
  for (int i = 0; i < n_inputs; ++i) {
    ws[i] = inputs[i].width;
    hs[i] = inputs[i].height;
  }
  // the shape of a single host request with these inputs
  Request r;
  r.p = p;
  r.in.assign(inputs, inputs + n_inputs);
  int ow = 0, oh = 0, oc = 0, odt = 0;
  hp_status st = hp::pipeline_output_shape(p, ws.data(), hs.data(), n_inputs, &ow, &oh, &oc, &odt);
  if (st) return st;
  r.out = hp_buffer{nullptr, (hp_dtype)odt, oc, ow, oh, 0, 0};
  // the batches of this shape the server may form (2 .. max_batch requests of
  // at most kBatchBytesMax in all, host or device buffers) are made ready too,
  // so that no batch size is lowered, allocated or captured while requests
  // are in flight
  bool batches;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    batches = s->max_batch > 1 && staging_bytes(r, 2) <= kBatchBytesMax && batchable(s, r);
  }
  int bmax = 1;
  if (batches)
    while (bmax < s->max_batch && staging_bytes(r, bmax + 1) <= kBatchBytesMax) ++bmax;
  std::lock_guard<std::mutex> ck(s->clone_mu);  // the worker realizes the slots' copies under this lock
  for (int B = 1; B <= bmax; ++B)
    for (int dev = 0; dev < (B > 1 ? 2 : 1); ++dev) {
      r.device = dev != 0;
      const ShapeKey key = shape_key(r, B);
      for (Slot& sl : s->slots) {
        hp_pipeline* c = slot_clone(sl, p, B);
        if (!c) return hp::report_error(HP_ERR_INVALID_ARG, "hp_server_prepare: pipeline cannot be copied");
        if ((st = hp_prepare(c, ws.data(), hs.data(), n_inputs, sl.stream))) return st;
        // the slot's staging region for this shape, resident from now on, and
        // the graph of its realize on it (two realizes: the first runs, the
        // second captures), so the first request of the shape already replays
        // a graph; an idle slot only (a busy one may be using its regions)
        Resident* region = nullptr;
        {
          std::lock_guard<std::mutex> lk(s->mu);
          if (sl.busy) continue;
          auto it = sl.resident.find(key);
          if (it == sl.resident.end()) {
            long long off = 0;
            const long long bytes = staging_bytes(r, B);
            if (!s->arena.alloc(bytes, &off)) continue;  // no room: the shape becomes resident on first use
            Resident& nr = sl.resident[key];
            nr.off = off;
            nr.bytes = bytes;
            it = sl.resident.find(key);
          }
          it->second.last = ++s->admissions;
          region = &it->second;
          sl.busy = true;  // the worker leaves the slot alone meanwhile
        }
        std::vector<hp_buffer> din;
        hp_buffer dout;
        staging_layout(s->arena.base + region->off, r, B, din, dout);
        for (int k = 0; k < 2 && !st; ++k) st = hp_realize(c, din.data(), n_inputs, &dout, sl.stream);
        if (!st && cudaStreamSynchronize(sl.stream) != cudaSuccess) {
          cudaGetLastError();
          st = hp::report_error(HP_ERR_CUDA, "hp_server_prepare: realize on the staging region failed");
        }
        {
          std::lock_guard<std::mutex> lk(s->mu);
          sl.busy = false;
        }
        if (st) return st;
      }
    }
  return HP_OK;
}

hp_status hp_server_destroy(hp_server* s) {
  if (!s) return hp::report_error(HP_ERR_INVALID_ARG, "null server");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_one();
  }
  s->worker.join();
  for (Slot& sl : s->slots) {
    cudaStreamSynchronize(sl.stream);
    for (auto& kv : sl.clones) hp_pipeline_destroy(kv.second);
    cudaStreamDestroy(sl.stream);
    cudaEventDestroy(sl.done);
  }
  for (Request* r : s->queue) delete r;
  cudaFree(s->arena.base);
  delete s;
  return HP_OK;
}

}  // extern "C"
