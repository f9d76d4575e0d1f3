// Serving many streams on one GPU: admission by device-memory footprint,
// per-stream frame queues on the device, and ticks that take the oldest
// queued frame of every active stream and push them all with one batched
// Gram-row launch (sdmd_push_many). Streams that do not fit wait in arrival
// order and are admitted as memory is released (sdmd_server_close). Each
// stream's G is bit-identical to pushing its frames alone (the batched
// kernel keeps every handle's chunking and reduction order). Latency of a
// frame = completion of its tick minus its arrival (host clock, or the time
// given at submit); p50 / p99 over all completed frames.
//
// A tick's work for up to 64 streams (the ingest copies of their queued
// frames and one batched Gram-row kernel) is a CUDA graph once the same set
// of streams comes back tick after tick: built once per set (copy nodes,
// then the kernel node after them), instantiated, and on later ticks updated
// in place (new slots, sources and kernel arguments) and launched with one
// cudaGraphLaunch. Sets that change every tick launch directly.
//
// A server is driven by one host thread; all its GPU work runs on its own
// stream (sdmd_server_stream).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <deque>
#include <new>
#include <vector>

#include "sdmd.h"
#include "sdmd_internal.cuh"

namespace {

constexpr int kQueue = 4;            // frames queued per stream

struct ServedStream {
  int state = 0;                     // SDMD_STREAM_*
  int64_t n = 0;
  int32_t m = 0, dtype = 0;
  int64_t footprint = 0;
  sdmd_t h = nullptr;
  uint8_t* fifo = nullptr;           // kQueue frames
  int64_t frame_bytes = 0;
  int head = 0, len = 0;
  double arrival[kQueue] = {};
};

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

int err(int code, const char* msg) { return sdmd::set_last_error(code, msg); }

}  // namespace

// Instantiated graph of one batch position (streams hs, in order).
struct TickGraph {
  std::vector<sdmd_t> key;
  std::vector<size_t> bytes;           // frame bytes of each copy (part of the key)
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaGraphNode_t> copies;
  cudaGraphNode_t kernel = nullptr;
  std::vector<sdmd_t> last;            // streams of the previous tick at this position
};

struct sdmd_server_s {
  int device = 0;
  int num_sms = 1;
  int64_t budget = 0, used = 0;
  cudaStream_t st = nullptr;
  std::vector<ServedStream> streams;
  std::deque<int32_t> waiting;
  std::vector<double> lat;
  int64_t frames = 0;
  bool graphs = true;
  std::vector<TickGraph> tg;          // per batch position
  int64_t graph_builds = 0, graph_updates = 0;
};

namespace {

int activate(sdmd_server_s* s, int32_t sid) {
  ServedStream& q = s->streams[sid];
  int rc = sdmd_create(q.n, q.m, q.dtype, &q.h);
  if (rc != SDMD_OK) return rc;
  q.frame_bytes = q.n * ((q.dtype == SDMD_U8) ? 1 : (q.dtype == SDMD_C64 ? 8 : 4));
  if (cudaMalloc(&q.fifo, (size_t)kQueue * (size_t)q.frame_bytes) != cudaSuccess) {
    cudaGetLastError();
    sdmd_destroy(q.h);
    q.h = nullptr;
    return err(SDMD_ERR_OOM, "sdmd_server: frame queue allocation failed");
  }
  q.state = SDMD_STREAM_ACTIVE;
  s->used += q.footprint;
  return SDMD_OK;
}

void drop_graph(TickGraph& t) {
  if (t.exec) cudaGraphExecDestroy(t.exec);
  if (t.g) cudaGraphDestroy(t.g);
  std::vector<sdmd_t> last;
  last.swap(t.last);
  t = TickGraph();
  t.last.swap(last);
}

// `copied` / `launched` report how far the batch got (the copies that were
// enqueued, whether the batched kernel was), for sdmd::push_many_finish.
int run_direct(sdmd_server_s* s, const sdmd::BatchPlan& plan, int* copied, bool* launched) {
  for (int i = 0; i < plan.ncopies; ++i) {
    if (cudaMemcpyAsync(plan.dst[i], plan.src[i], plan.bytes[i], cudaMemcpyDefault, s->st) != cudaSuccess) {
      cudaGetLastError();
      return err(SDMD_ERR_CUDA, "sdmd_server_tick: copy failed");
    }
    *copied = i + 1;
  }
  if (sdmd::launch_gram_rows_batched(plan.args, s->st) != cudaSuccess) {
    cudaGetLastError();
    return err(SDMD_ERR_CUDA, "sdmd_server_tick: batched launch failed");
  }
  *launched = true;
  return SDMD_OK;
}

// Issue one planned batch on the server stream: as a graph (built or
// updated) or, with graphs off, as copies plus a kernel launch.
// A set of streams gets a graph once it has come twice in a row at a batch
// position (a steady set); sets that change every tick launch directly.
int run_batch(sdmd_server_s* s, size_t b, const std::vector<sdmd_t>& hs, const sdmd::BatchPlan& plan, int* copied,
              bool* launched) {
  *copied = 0;
  *launched = false;
  if (!s->graphs) return run_direct(s, plan, copied, launched);
  if (s->tg.size() <= b) s->tg.resize(b + 1);
  TickGraph& t = s->tg[b];
  const bool steady = (t.exec && t.key == hs) || t.last == hs;
  t.last = hs;
  if (!steady) return run_direct(s, plan, copied, launched);
  cudaKernelNodeParams kp;
  if (sdmd::batched_kernel_config(plan.args, &kp) != cudaSuccess) {
    cudaGetLastError();
    return err(SDMD_ERR_CUDA, "sdmd_server_tick: kernel configuration failed");
  }
  sdmd::BatchArgs args = plan.args;
  void* kargs[1] = {&args};
  kp.kernelParams = kargs;
  cudaError_t e = cudaSuccess;
  const std::vector<size_t> bytes(plan.bytes, plan.bytes + plan.ncopies);
  if (t.exec && t.key == hs && t.bytes == bytes) {   // same streams: update in place
    for (int i = 0; i < plan.ncopies && e == cudaSuccess; ++i)
      e = cudaGraphExecMemcpyNodeSetParams1D(t.exec, t.copies[i], plan.dst[i], plan.src[i], plan.bytes[i],
                                             cudaMemcpyDefault);
    if (e == cudaSuccess) e = cudaGraphExecKernelNodeSetParams(t.exec, t.kernel, &kp);
    if (e == cudaSuccess) s->graph_updates += 1;
  } else {
    drop_graph(t);
    e = cudaGraphCreate(&t.g, 0);
    t.copies.resize(plan.ncopies);
    for (int i = 0; i < plan.ncopies && e == cudaSuccess; ++i)
      e = cudaGraphAddMemcpyNode1D(&t.copies[i], t.g, nullptr, 0, plan.dst[i], plan.src[i], plan.bytes[i],
                                   cudaMemcpyDefault);
    if (e == cudaSuccess) e = cudaGraphAddKernelNode(&t.kernel, t.g, t.copies.data(), t.copies.size(), &kp);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&t.exec, t.g, 0);
    if (e == cudaSuccess) {
      t.key = hs;
      t.bytes = bytes;
      s->graph_builds += 1;
    }
  }
  if (e == cudaSuccess) e = cudaGraphLaunch(t.exec, s->st);
  if (e != cudaSuccess) {         // nothing of the graph ran
    cudaGetLastError();
    drop_graph(t);
    return err(SDMD_ERR_CUDA, "sdmd_server_tick: graph build, update or launch failed");
  }
  *copied = plan.ncopies;
  *launched = true;
  return SDMD_OK;
}

// Admit waiting streams, in arrival order, while the head of the line fits.
int admit_waiting(sdmd_server_s* s) {
  while (!s->waiting.empty()) {
    const int32_t sid = s->waiting.front();
    if (s->used + s->streams[sid].footprint > s->budget) break;
    s->waiting.pop_front();
    const int rc = activate(s, sid);
    if (rc != SDMD_OK) return rc;
  }
  return SDMD_OK;
}

}  // namespace

extern "C" {

int sdmd_server_create(int64_t hbm_budget, sdmd_server_t* out) {
  if (!out || hbm_budget <= 0) return err(SDMD_ERR_ARG, "sdmd_server_create: bad argument");
  sdmd_server_s* s = new (std::nothrow) sdmd_server_s();
  if (!s) return err(SDMD_ERR_OOM, "sdmd_server_create: host allocation failed");
  cudaGetDevice(&s->device);
  cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
  s->budget = hbm_budget;
  if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return err(SDMD_ERR_CUDA, "sdmd_server_create: stream creation failed");
  }
  *out = s;
  return SDMD_OK;
}

int sdmd_server_destroy(sdmd_server_t s) {
  if (!s) return err(SDMD_ERR_ARG, "sdmd_server_destroy: NULL server");
  cudaStreamSynchronize(s->st);
  for (TickGraph& t : s->tg) drop_graph(t);
  for (ServedStream& q : s->streams) {
    if (q.h) sdmd_destroy(q.h);
    cudaFree(q.fifo);
  }
  cudaStreamDestroy(s->st);
  delete s;
  return SDMD_OK;
}

int sdmd_server_stream(sdmd_server_t s, void** stream) {
  if (!s || !stream) return err(SDMD_ERR_ARG, "sdmd_server_stream: bad argument");
  *stream = s->st;
  return SDMD_OK;
}

int sdmd_server_open(sdmd_server_t s, int64_t n, int32_t m, int32_t dtype, int32_t* sid) {
  if (!s || !sid) return err(SDMD_ERR_ARG, "sdmd_server_open: bad argument");
  if (dtype != SDMD_U8 && dtype != SDMD_F32 && dtype != SDMD_C64)
    return err(SDMD_ERR_ARG, "sdmd_server_open: dense dtypes only");
  if (n < 1 || m < 2 || m > SDMD_MAX_M) return err(SDMD_ERR_ARG, "sdmd_server_open: n or m out of range");
  ServedStream q;
  q.n = n;
  q.m = m;
  q.dtype = dtype;
  const int64_t elem = (dtype == SDMD_U8) ? 1 : (dtype == SDMD_C64 ? 8 : 4);
  q.footprint = sdmd::handle_device_bytes(n, m, dtype, s->num_sms) + kQueue * n * elem;
  if (q.footprint > s->budget) return err(SDMD_ERR_ARG, "sdmd_server_open: the stream alone exceeds the budget");
  s->streams.push_back(q);
  *sid = (int32_t)s->streams.size() - 1;
  s->waiting.push_back(*sid);
  return admit_waiting(s);
}

int sdmd_server_state(sdmd_server_t s, int32_t sid) {
  if (!s || sid < 0 || sid >= (int32_t)s->streams.size()) return err(SDMD_ERR_ARG, "sdmd_server_state: bad stream");
  return s->streams[sid].state;
}

int sdmd_server_handle(sdmd_server_t s, int32_t sid, sdmd_t* h) {
  if (!s || !h || sid < 0 || sid >= (int32_t)s->streams.size()) return err(SDMD_ERR_ARG, "sdmd_server_handle: bad stream");
  if (s->streams[sid].state != SDMD_STREAM_ACTIVE) return err(SDMD_ERR_NOT_READY, "sdmd_server_handle: stream not active");
  *h = s->streams[sid].h;
  return SDMD_OK;
}

int sdmd_server_submit(sdmd_server_t s, int32_t sid, const void* x, double arrival_ms) {
  if (!s || !x || sid < 0 || sid >= (int32_t)s->streams.size()) return err(SDMD_ERR_ARG, "sdmd_server_submit: bad argument");
  ServedStream& q = s->streams[sid];
  if (q.state != SDMD_STREAM_ACTIVE) return err(SDMD_ERR_NOT_READY, "sdmd_server_submit: stream not active");
  if (q.len == kQueue) return err(SDMD_ERR_NOT_READY, "sdmd_server_submit: frame queue full");
  const int slot = (q.head + q.len) % kQueue;
  if (cudaMemcpyAsync(q.fifo + (int64_t)slot * q.frame_bytes, x, (size_t)q.frame_bytes, cudaMemcpyDefault, s->st) !=
      cudaSuccess) {
    cudaGetLastError();
    return err(SDMD_ERR_CUDA, "sdmd_server_submit: copy failed");
  }
  q.arrival[slot] = arrival_ms >= 0.0 ? arrival_ms : now_ms();
  q.len += 1;
  return SDMD_OK;
}

int sdmd_server_tick(sdmd_server_t s, int32_t* frames_done) {
  if (!s) return err(SDMD_ERR_ARG, "sdmd_server_tick: NULL server");
  std::vector<int32_t> ids;
  for (int32_t i = 0; i < (int32_t)s->streams.size(); ++i)
    if (s->streams[i].state == SDMD_STREAM_ACTIVE && s->streams[i].len > 0) ids.push_back(i);
  for (size_t b = 0; b < ids.size(); b += SDMD_MAX_BATCH) {
    const size_t e = std::min(ids.size(), b + (size_t)SDMD_MAX_BATCH);
    std::vector<sdmd_t> hs;
    std::vector<const void*> xs;
    for (size_t i = b; i < e; ++i) {
      ServedStream& q = s->streams[ids[i]];
      hs.push_back(q.h);
      xs.push_back(q.fifo + (int64_t)q.head * q.frame_bytes);
    }
    sdmd::BatchPlan plan;
    int rc = sdmd::push_many_plan(hs.data(), xs.data(), (int32_t)hs.size(), s->st, &plan);
    if (rc != SDMD_OK) return rc;
    int copied = 0;
    bool launched = false;
    rc = run_batch(s, b / SDMD_MAX_BATCH, hs, plan, &copied, &launched);
    const int rf = sdmd::push_many_finish(hs.data(), (int)hs.size(), copied, launched, s->st);
    if (rc == SDMD_OK) rc = rf;
    if (rc != SDMD_OK) return rc;
  }
  if (cudaStreamSynchronize(s->st) != cudaSuccess) {
    cudaGetLastError();
    return err(SDMD_ERR_CUDA, "sdmd_server_tick: stream synchronisation failed");
  }
  const double t = now_ms();
  for (int32_t sid : ids) {
    ServedStream& q = s->streams[sid];
    s->lat.push_back(t - q.arrival[q.head]);
    q.head = (q.head + 1) % kQueue;
    q.len -= 1;
  }
  s->frames += (int64_t)ids.size();
  if (frames_done) *frames_done = (int32_t)ids.size();
  return SDMD_OK;
}

int sdmd_server_close(sdmd_server_t s, int32_t sid) {
  if (!s || sid < 0 || sid >= (int32_t)s->streams.size()) return err(SDMD_ERR_ARG, "sdmd_server_close: bad stream");
  ServedStream& q = s->streams[sid];
  if (q.state == SDMD_STREAM_WAITING) {
    s->waiting.erase(std::find(s->waiting.begin(), s->waiting.end(), sid));
  } else if (q.state == SDMD_STREAM_ACTIVE) {
    cudaStreamSynchronize(s->st);
    sdmd_destroy(q.h);
    q.h = nullptr;
    cudaFree(q.fifo);
    q.fifo = nullptr;
    s->used -= q.footprint;
  }
  q.state = SDMD_STREAM_CLOSED;
  return admit_waiting(s);
}

int sdmd_server_stats(sdmd_server_t s, double* p50_ms, double* p99_ms, int64_t* frames) {
  if (!s) return err(SDMD_ERR_ARG, "sdmd_server_stats: NULL server");
  std::vector<double> v = s->lat;
  std::sort(v.begin(), v.end());
  auto pct = [&](double p) { return v.empty() ? 0.0 : v[(size_t)std::min<double>(v.size() - 1, p * (v.size() - 1) + 0.5)]; };
  if (p50_ms) *p50_ms = pct(0.50);
  if (p99_ms) *p99_ms = pct(0.99);
  if (frames) *frames = s->frames;
  return SDMD_OK;
}

int64_t sdmd_server_used_bytes(sdmd_server_t s) { return s ? s->used : -1; }

int sdmd_server_set_graphs(sdmd_server_t s, int32_t on) {
  if (!s) return err(SDMD_ERR_ARG, "sdmd_server_set_graphs: NULL server");
  cudaStreamSynchronize(s->st);
  for (TickGraph& t : s->tg) drop_graph(t);
  s->tg.clear();
  s->graphs = on != 0;
  return SDMD_OK;
}

int sdmd_server_graph_stats(sdmd_server_t s, int64_t* builds, int64_t* updates) {
  if (!s) return err(SDMD_ERR_ARG, "sdmd_server_graph_stats: NULL server");
  if (builds) *builds = s->graph_builds;
  if (updates) *updates = s->graph_updates;
  return SDMD_OK;
}

int sdmd_server_autotune(sdmd_server_t s) {
  if (!s) return err(SDMD_ERR_ARG, "sdmd_server_autotune: NULL server");
  for (ServedStream& q : s->streams) {
    if (q.state != SDMD_STREAM_ACTIVE) continue;
    int64_t cnt = 0;
    sdmd_count(q.h, &cnt);
    if (cnt < 1) continue;
    const int rc = sdmd_autotune(q.h, nullptr, nullptr, s->st);
    if (rc != SDMD_OK) return rc;
  }
  // schedules changed: the graphs' kernel arguments are rebuilt on the next tick
  for (TickGraph& t : s->tg) drop_graph(t);
  return SDMD_OK;
}

int sdmd_server_reset_stats(sdmd_server_t s) {
  if (!s) return err(SDMD_ERR_ARG, "sdmd_server_reset_stats: NULL server");
  s->lat.clear();
  s->frames = 0;
  return SDMD_OK;
}

double sdmd_server_clock_ms(void) { return now_ms(); }

}  // extern "C"
