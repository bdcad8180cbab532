// Serving loop: continuous batching of pipeline requests on one GPU.
//
// Requests (a pipeline, host input buffers, a host output buffer) arrive at
// any time through hp_server_submit.  A worker thread admits them in arrival
// order as soon as a slot (a CUDA stream) and device memory are free: request
// buffers come from one arena reserved at creation, so admission is by HBM
// footprint (a slot's pipeline copies allocate their own small scratch the
// first time they run an image size).  Admitted work runs
// concurrently on the slots' streams (copies in, realize, copies out), so a
// request that arrives while others are on the GPU overlaps with them.
// Requests for the same pipeline and image size whose stages all act on each
// channel separately (stencils, point-wise per-channel ops, resampling) are
// batched: their planes are stacked into one image and served by one realize,
// which launches each kernel once for the whole batch.  Each slot keeps its
// own copies of the pipelines it runs, so concurrent requests never share a
// pipeline's scratch.  Latency is measured from submit to the completion the
// worker observes.
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
bool pipeline_stackable(const hp_pipeline* p);
}  // namespace hp

namespace {

using Clock = std::chrono::steady_clock;

int dtype_size(int d) { return d == HP_U8 ? 1 : (d == HP_U16 || d == HP_F16 || d == HP_BF16) ? 2 : 4; }
using hp::Arena;
long long r256(long long v) { return hp::round256(v); }

struct Request {
  unsigned long long ticket = 0;
  hp_pipeline* p = nullptr;
  std::vector<hp_buffer> in;
  hp_buffer out{};
  Clock::time_point t_submit;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  std::vector<Request*> batch;
  long long off = 0, bytes = 0;
  hp_status status = HP_OK;
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
  std::mutex mu;
  std::condition_variable cv_done, cv_work;
  std::thread worker;
  bool stop = false;
  unsigned long long next_ticket = 1, submitted = 0, completed = 0, failed = 0, batched = 0;
  double mpix = 0;
  Clock::time_point t_first, t_last;
  bool any = false;
  int device = 0;
};

namespace {

// Footprint of one request: every input and the output, packed.
long long request_bytes(const Request& r) {
  long long b = 0;
  for (const hp_buffer& x : r.in) b += r256((long long)x.width * dtype_size(x.dtype)) * x.height * x.channels;
  b += r256((long long)r.out.width * dtype_size(r.out.dtype)) * r.out.height * r.out.channels;
  return b + 256 * (long long)(r.in.size() + 1);
}

bool same_shape(const Request& a, const Request& b) {
  if (a.p != b.p || a.in.size() != b.in.size()) return false;
  for (size_t i = 0; i < a.in.size(); ++i)
    if (a.in[i].width != b.in[i].width || a.in[i].height != b.in[i].height || a.in[i].dtype != b.in[i].dtype)
      return false;
  return a.out.width == b.out.width && a.out.height == b.out.height;
}

hp_pipeline* slot_clone(Slot& sl, hp_pipeline* p, int batch) {
  auto key = std::make_pair(p, batch);
  auto it = sl.clones.find(key);
  if (it != sl.clones.end()) return it->second;
  hp_pipeline* c = hp::clone_pipeline(p, batch);
  sl.clones[key] = c;
  return c;
}

// Device layout of a batch: for each input i, B stacked images of C_i planes;
// then the output, B stacked images.  Row stride is the packed width rounded
// to 16 bytes.
hp_status launch_batch(hp_server* s, Slot& sl) {
  const int B = (int)sl.batch.size();
  const Request& r0 = *sl.batch[0];
  char* dev = s->arena.base + sl.off;
  std::vector<hp_buffer> din(r0.in.size());
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
  hp_buffer dout = r0.out;
  dout.data = dev + pos;
  dout.row_stride_bytes = (((long long)r0.out.width * dtype_size(r0.out.dtype)) + 15) / 16 * 16;
  dout.plane_stride_bytes = dout.row_stride_bytes * r0.out.height;
  dout.channels = r0.out.channels * B;
  cudaStream_t st = sl.stream;
  for (int j = 0; j < B; ++j) {
    const Request& r = *sl.batch[j];
    for (size_t i = 0; i < r.in.size(); ++i) {
      const hp_buffer& h = r.in[i];
      for (int c = 0; c < h.channels; ++c) {
        char* dst = (char*)din[i].data + (long long)(j * h.channels + c) * din[i].plane_stride_bytes;
        const char* src = (const char*)h.data + (long long)c * h.plane_stride_bytes;
        if (cudaMemcpy2DAsync(dst, din[i].row_stride_bytes, src, h.row_stride_bytes,
                              (size_t)h.width * dtype_size(h.dtype), h.height, cudaMemcpyHostToDevice, st))
          return hp::report_error(HP_ERR_CUDA, "server: host-to-device copy failed");
      }
    }
  }
  hp_pipeline* p = slot_clone(sl, r0.p, B);
  if (!p) return hp::report_error(HP_ERR_INVALID_ARG, "server: pipeline cannot be batched");
  hp_status rs = hp_realize(p, din.data(), (int)din.size(), &dout, st);
  if (rs) return rs;
  for (int j = 0; j < B; ++j) {
    const hp_buffer& h = sl.batch[j]->out;
    for (int c = 0; c < h.channels; ++c) {
      const char* src = (const char*)dout.data + (long long)(j * h.channels + c) * dout.plane_stride_bytes;
      char* dst = (char*)h.data + (long long)c * h.plane_stride_bytes;
      if (cudaMemcpy2DAsync(dst, h.row_stride_bytes, src, dout.row_stride_bytes, (size_t)h.width * dtype_size(h.dtype),
                            h.height, cudaMemcpyDeviceToHost, st))
        return hp::report_error(HP_ERR_CUDA, "server: device-to-host copy failed");
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
  s->arena.release(sl.off, sl.bytes);
  sl.busy = false;
  s->t_last = now;
}

void worker_loop(hp_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    bool progress = false;
    // completions
    for (Slot& sl : s->slots) {
      if (!sl.busy) continue;
      cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      finish_slot(s, sl, q == cudaSuccess ? HP_OK : HP_ERR_CUDA);
      progress = true;
    }
    if (progress) s->cv_done.notify_all();
    // admissions, in arrival order
    while (!s->queue.empty()) {
      Slot* free_slot = nullptr;
      for (Slot& sl : s->slots)
        if (!sl.busy) {
          free_slot = &sl;
          break;
        }
      if (!free_slot) break;
      Request* head = s->queue.front();
      std::vector<size_t> pick{0};
      if (s->max_batch > 1 && hp::pipeline_stackable(head->p)) {
        for (size_t i = 1; i < s->queue.size() && (int)pick.size() < s->max_batch && i < 64; ++i)
          if (same_shape(*head, *s->queue[i])) pick.push_back(i);
      }
      long long bytes = 0;
      for (size_t i : pick) bytes += request_bytes(*s->queue[i]);
      long long off = 0;
      if (!s->arena.alloc(bytes, &off)) {
        if (pick.size() > 1) {  // try the head alone before waiting for memory
          pick.resize(1);
          bytes = request_bytes(*head);
          if (!s->arena.alloc(bytes, &off)) break;
        } else {
          break;
        }
      }
      Slot& sl = *free_slot;
      sl.batch.clear();
      for (size_t i : pick) sl.batch.push_back(s->queue[i]);
      for (size_t k = pick.size(); k-- > 0;) s->queue.erase(s->queue.begin() + pick[k]);
      sl.off = off;
      sl.bytes = bytes;
      sl.busy = true;
      hp_status st = launch_batch(s, sl);
      if (st) {
        cudaStreamSynchronize(sl.stream);
        cudaGetLastError();
        finish_slot(s, sl, st);
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
  if (!s || !p || !inputs || n_inputs < 1 || n_inputs > 16 || !output || !ticket)
    return hp::report_error(HP_ERR_INVALID_ARG, "hp_server_submit: bad arguments");
  auto* r = new Request();
  r->p = p;
  r->in.assign(inputs, inputs + n_inputs);
  r->out = *output;
  for (const hp_buffer& b : r->in)
    if (!b.data || b.width < 1 || b.height < 1) {
      delete r;
      return hp::report_error(HP_ERR_INVALID_ARG, "hp_server_submit: empty input buffer");
    }
  if (!r->out.data || r->out.width < 1 || r->out.height < 1 || r->out.channels < 1) {
    delete r;
    return hp::report_error(HP_ERR_INVALID_ARG, "hp_server_submit: empty output buffer");
  }
  if (request_bytes(*r) > s->arena.size) {
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
  s->queue.push_back(r);
  s->cv_work.notify_one();
  return HP_OK;
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
  std::lock_guard<std::mutex> lk(s->mu);  // the worker touches slot copies only under the lock
  for (Slot& sl : s->slots) {
    hp_pipeline* c = slot_clone(sl, p, 1);
    if (!c) return hp::report_error(HP_ERR_INVALID_ARG, "hp_server_prepare: pipeline cannot be copied");
    hp_status st = hp_prepare(c, ws.data(), hs.data(), n_inputs, sl.stream);
    if (st) return st;
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
