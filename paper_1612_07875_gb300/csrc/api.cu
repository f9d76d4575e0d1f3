// C ABI of libsdmd: handle lifetime, argument checks, pointer-kind handling,
// and the launch sequences of sdmd_push / sdmd_modes (see include/sdmd.h).
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>
#include <deque>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "sdmd.h"
#include "sdmd_internal.cuh"

using namespace sdmd;

namespace sdmd {

cudaError_t smem_optin(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> level;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = level[std::make_pair(func, dev)];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

}  // namespace sdmd

// One in-flight DMD of the pipelined step (sdmd_step): its own workspace and
// stream, and events ordering it against the push stream. Its eigensolver
// reads the frame's window of G in place: the pushes that follow write only
// the rows and columns of their own slots, and a slot of the window is
// rewritten only after the push stream has waited for the frame
// (wait_ring_readers).
struct PipeCtx {
  double* ws = nullptr;       // modes workspace (window m)
  int* r_dev = nullptr;
  unsigned* phi_sched = nullptr;  // Phi tile-scheduling words (zero between launches)
  cudaStream_t st = nullptr;
  cudaEvent_t ev_g = nullptr;     // the frame's G row written (push stream)
  cudaEvent_t ev_done = nullptr;  // modes, Phi and output copies done (ctx stream, or the push
                                  // stream when Phi ran fused with a later Gram row)
  cudaEvent_t ev_modes = nullptr; // modes and output copies done (ctx stream)
  bool busy = false;
  int64_t frame = -1;         // push count of the frame being processed
  // Phi deferred to a later step (fused with that step's Gram row)
  bool phi_pending = false;
  float* phi = nullptr;
  int32_t r = 0, start = 0, p = 0;
  cudaEvent_t fr1 = nullptr;  // frame-trace end, recorded when the deferred Phi completes
};

struct sdmd_s {
  int device = 0;
  int num_sms = 0;
  int64_t n = 0;
  int32_t m = 0;              // window length (resident snapshots)
  int32_t cap = 0;            // ring slots (m, or m + depth when pipelined)
  int32_t depth = 1;          // DMD frames in flight (sdmd_step)
  std::vector<PipeCtx> ctx;
  std::deque<int> pending;    // contexts whose Phi is deferred, oldest first
  long long* fgpart = nullptr;  // fused Gram row: per-CTA sums (allocated on first use)
  int32_t nblk_alloc = 0;       // chunks the partials array holds
  int64_t steps = 0;
  int32_t dtype = 0;
  int64_t elem = 0;
  int64_t slot_bytes = 0;
  uint8_t* ring = nullptr;
  void* G = nullptr;          // m x m physical, 8-byte entries
  void* gtmp = nullptr;       // m x m gather scratch for sdmd_gram
  void* partials = nullptr;   // [m][nblk] 8-byte entries
  unsigned int* ticket = nullptr;
  int64_t chunk = 0;
  int32_t nblk = 0;
  double* ws = nullptr;       // modes workspace
  int* status = nullptr;      // device status word
  int* r_dev = nullptr;       // device int: kept rank of the last modes call
  unsigned* phi_sched = nullptr;  // Phi tile-scheduling words (zero between launches)
  int64_t count = 0;
  int32_t head = 0;
  int32_t last_r = 0;         // r of the last sdmd_modes call (0 = none)
  int32_t last_p = 0;
  int64_t modes_count = -1;   // push count when sdmd_modes last ran (reconstruction window)
  int64_t gsz = 8;            // bytes per G entry (16 for complex handles)
  int32_t phi_tensor = 1;     // SDMD_OPT_PHI_TENSOR
  int32_t rebuild_tensor = 1; // SDMD_OPT_REBUILD_TENSOR
  int32_t f32_bf16x3 = 0;     // SDMD_OPT_F32_BF16X3 (0 off, 1 three terms, 2 two terms)
  int32_t f32_fp64 = 0;       // SDMD_OPT_F32_FP64
  int32_t host_early = 0;     // SDMD_OPT_HOST_EARLY_READ
  cudaStream_t cst = nullptr; // its copy stream, two staging slots and events (made on first use)
  uint8_t* stage = nullptr;
  cudaEvent_t ev_h2d = nullptr;
  cudaEvent_t ev_stage_free[2] = {nullptr, nullptr};
  int64_t stage_i = 0;
  long long* gf_partials = nullptr;  // tensor-core rebuild: per-CTA sums (allocated on first use)
  unsigned* gf_sched = nullptr;      // tensor-core rebuild: chunk counter
  // sparse handles
  int32_t nnz_max = 0;
  int* idx_ring = nullptr;    // m x nnz_max indices
  float2* val_ring = nullptr; // m x nnz_max complex64 values
  int* tag = nullptr;         // n lookup tags
  unsigned* fbits = nullptr;  // Fourier modes: support bitmap (allocated on first use)
  unsigned long long* fprefix = nullptr;  // its popcount prefix, then the union size
  float2* tval = nullptr;     // n lookup values
  int stamp = 0;
  std::vector<int> nnz;       // entries per physical slot
  // tracing: per kernel class, event pairs recorded since the last read
  bool trace = false;
  std::vector<cudaEvent_t> tr_ev[SDMD_K_COUNT];
  size_t tr_used[SDMD_K_COUNT] = {0, 0, 0, 0, 0, 0};
};

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(SDMD_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

#define CK(call)                                   \
  do {                                             \
    cudaError_t _e = (call);                       \
    if (_e != cudaSuccess) return cuda_fail(_e, #call); \
  } while (0)

// Makes the handle's device current for the scope of a call.
struct DeviceScope {
  int prev = -1;
  bool changed = false;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
      if (cudaSetDevice(dev) == cudaSuccess) changed = true;
    }
  }
  ~DeviceScope() {
    if (changed) cudaSetDevice(prev);
  }
};

enum PtrKind { kPageable = 0, kPinned = 1, kDevice = 2 };

PtrKind ptr_kind(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return kPageable;
  }
  switch (at.type) {
    case cudaMemoryTypeDevice:
    case cudaMemoryTypeManaged:
      return kDevice;
    case cudaMemoryTypeHost:
      return kPinned;
    default:
      return kPageable;
  }
}

// Copy `bytes` from device memory to a caller buffer of any kind; pageable
// destinations make the call wait for the stream.
int copy_out(void* dst, const void* src_dev, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return SDMD_OK;
  const PtrKind k = ptr_kind(dst);
  CK(cudaMemcpyAsync(dst, src_dev, bytes, cudaMemcpyDefault, st));
  if (k == kPageable) CK(cudaStreamSynchronize(st));
  return SDMD_OK;
}

// Snapshot ingest on the SMs: 16-byte loads and stores, four per thread in
// flight, the last bytes (n mod 16) by the first threads of block 0. A
// device-to-device cudaMemcpyAsync of one HD frame (6.2 MB) measured about
// 13 us between two kernels of the push stream, this kernel a few us.
__global__ void __launch_bounds__(256) ingest_copy_kernel(const uint4* __restrict__ src, uint4* __restrict__ dst,
                                                          int64_t n16, int tail) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n16; i += 4 * stride) {
    const uint4 a = src[i], b = src[i + stride], c = src[i + 2 * stride], d = src[i + 3 * stride];
    dst[i] = a;
    dst[i + stride] = b;
    dst[i + 2 * stride] = c;
    dst[i + 3 * stride] = d;
  }
  for (; i < n16; i += stride) dst[i] = src[i];
  if (blockIdx.x == 0 && (int)threadIdx.x < tail)
    reinterpret_cast<uint8_t*>(dst + n16)[threadIdx.x] = reinterpret_cast<const uint8_t*>(src + n16)[threadIdx.x];
}

// Copy one snapshot (`bytes`) into a ring slot on `st`: the SM kernel above
// for device sources with both addresses 16-byte aligned, else
// cudaMemcpyAsync (host sources, unaligned device pointers).
cudaError_t copy_snapshot(void* dst, const void* src, size_t bytes, int num_sms, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  const bool aligned = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0;
  if (!aligned || ptr_kind(src) != kDevice) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st);
  const int64_t n16 = (int64_t)(bytes / 16);
  const int tail = (int)(bytes - (size_t)n16 * 16);
  int64_t blocks = (n16 + 4 * 256 - 1) / (4 * 256);
  const int64_t cap = 4 * (int64_t)(num_sms > 0 ? num_sms : 1);
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  ingest_copy_kernel<<<(unsigned)blocks, 256, 0, st>>>(static_cast<const uint4*>(src), static_cast<uint4*>(dst), n16,
                                                       tail);
  return cudaGetLastError();
}

// Time-ordered copy of the physical G; `words` 8-byte words per entry.
__global__ void gather_gram_kernel(const uint64_t* G, int m, int c, int start, int words, uint64_t* out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= c * c) return;
  const int i = idx / c, j = idx - i * c;
  const int64_t src = (int64_t)((start + i) % m) * m + (start + j) % m;
  for (int q = 0; q < words; ++q) out[(int64_t)idx * words + q] = G[src * words + q];
}

// The newest snapshot's row of the physical G (slot s_new) in time order.
__global__ void newest_row_kernel(const uint64_t* G, int m, int c, int start, int s_new, int words, uint64_t* out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= c) return;
  const int64_t src = (int64_t)s_new * m + (start + q) % m;
  for (int w = 0; w < words; ++w) out[(int64_t)q * words + w] = G[src * words + w];
}

// Row and column s_new of the physical G from a time-ordered row; the column
// gets the conjugate (complex entries: the sign bit of the imaginary part
// flips), the diagonal entry is written once.
__global__ void set_newest_row_kernel(uint64_t* G, int m, int c, int start, int s_new, int words,
                                      const uint64_t* row) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= c) return;
  const int j = (start + q) % m;
  for (int w = 0; w < words; ++w) G[((int64_t)s_new * m + j) * words + w] = row[(int64_t)q * words + w];
  if (j == s_new) return;
  for (int w = 0; w < words; ++w) {
    uint64_t v = row[(int64_t)q * words + w];
    if (w == 1) v ^= 0x8000000000000000ull;
    G[((int64_t)j * m + s_new) * words + w] = v;
  }
}

// Event pair for class k (created on first use); false if tracing is off.
bool trace_pair(sdmd_s* h, int k, cudaEvent_t* a, cudaEvent_t* b) {
  if (!h->trace) return false;
  auto& v = h->tr_ev[k];
  while (v.size() < 2 * (h->tr_used[k] + 1)) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return false;
    v.push_back(e);
  }
  *a = v[2 * h->tr_used[k]];
  *b = v[2 * h->tr_used[k] + 1];
  h->tr_used[k] += 1;
  return true;
}

// Brackets one enqueued operation with a pair of events when tracing is on.
struct TraceScope {
  sdmd_s* h;
  int k;
  cudaStream_t st;
  bool on;
  TraceScope(sdmd_s* h_, int k_, cudaStream_t st_) : h(h_), k(k_), st(st_), on(h_->trace) {
    if (!on) return;
    auto& v = h->tr_ev[k];
    while (v.size() < 2 * (h->tr_used[k] + 1)) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) {
        on = false;
        return;
      }
      v.push_back(e);
    }
    cudaEventRecord(v[2 * h->tr_used[k]], st);
  }
  ~TraceScope() {
    if (!on) return;
    cudaEventRecord(h->tr_ev[k][2 * h->tr_used[k] + 1], st);
    h->tr_used[k] += 1;
  }
};

void free_sparse(sdmd_s* h) {
  cudaFree(h->idx_ring);
  cudaFree(h->val_ring);
  cudaFree(h->tag);
  cudaFree(h->fbits);
  cudaFree(h->fprefix);
  cudaFree(h->tval);
}

void free_ctx(sdmd_s* h) {
  for (PipeCtx& c : h->ctx) {
    if (c.st) cudaStreamSynchronize(c.st);
    cudaFree(c.ws);
    cudaFree(c.r_dev);
    cudaFree(c.phi_sched);
    if (c.ev_g) cudaEventDestroy(c.ev_g);
    if (c.ev_done) cudaEventDestroy(c.ev_done);
    if (c.ev_modes) cudaEventDestroy(c.ev_modes);
    if (c.st) cudaStreamDestroy(c.st);
  }
  h->ctx.clear();
}

void free_all(sdmd_s* h) {
  free_ctx(h);
  free_sparse(h);
  for (int k = 0; k < SDMD_K_COUNT; ++k)
    for (cudaEvent_t e : h->tr_ev[k]) cudaEventDestroy(e);
  cudaFree(h->ring);
  cudaFree(h->G);
  cudaFree(h->gtmp);
  cudaFree(h->partials);
  cudaFree(h->ticket);
  cudaFree(h->ws);
  cudaFree(h->status);
  cudaFree(h->r_dev);
  cudaFree(h->phi_sched);
  cudaFree(h->gf_partials);
  cudaFree(h->gf_sched);
  cudaFree(h->fgpart);
  cudaFree(h->stage);
  if (h->ev_h2d) cudaEventDestroy(h->ev_h2d);
  for (cudaEvent_t e : h->ev_stage_free)
    if (e) cudaEventDestroy(e);
  if (h->cst) cudaStreamDestroy(h->cst);
}

inline int32_t resident(const sdmd_s* h) { return (int32_t)(h->count < h->m ? h->count : h->m); }
inline int32_t oldest_slot(const sdmd_s* h) { return (int32_t)((h->count - resident(h)) % h->cap); }

// Before push number t overwrites slot t % cap (the snapshot pushed cap
// earlier), wait for every in-flight DMD whose X' still contains it.
int flush_pending(sdmd_s* h, cudaStream_t st);

// Make `st` wait for every in-flight frame that still reads the ring slot
// push number t (default: the next push) is about to overwrite, or that
// slot's row and column of G: a frame's Phi reads its pushes frame - p + 1 ..
// frame, its eigensolver the G entries of pushes frame - p .. frame.
int wait_ring_readers(sdmd_s* h, cudaStream_t st, int64_t t = -1) {
  if (t < 0) t = h->count;
  for (PipeCtx& c : h->ctx) {
    if (c.busy && c.frame - c.p <= t - h->cap) {
      if (c.phi_pending) {                     // its Phi must run before the slot is reused
        const int rc = flush_pending(h, st);
        if (rc != SDMD_OK) return rc;
      }
      CK(cudaStreamWaitEvent(st, c.ev_done, 0));
      c.busy = false;
    }
  }
  return SDMD_OK;
}

// Phi arguments of a pipelined frame (its window, its modes workspace).
PhiArgs ctx_phi_args(const sdmd_s* h, const PipeCtx& k) {
  const ModesLayout L = modes_layout(h->m);
  PhiArgs pa;
  pa.ring = h->ring;
  pa.slot_bytes = h->slot_bytes;
  pa.n = h->n;
  pa.dtype = h->dtype;
  pa.m = h->cap;
  pa.start = k.start;
  pa.p = k.p;
  pa.r = k.r;
  pa.Mf = reinterpret_cast<const float*>(k.ws + L.Mf);
  pa.r_dev = k.r_dev;
  pa.phi = k.phi;
  pa.status = h->status;
  pa.tensor = h->phi_tensor != 0;
  pa.fit_modes = h->phi_tensor == 1;
  pa.sched = k.phi_sched;
  return pa;
}

// The deferred Phi of the oldest pending frame, on its own, on `st`.
int flush_one(sdmd_s* h, cudaStream_t st) {
  const int ci = h->pending.front();
  h->pending.pop_front();
  PipeCtx& k = h->ctx[ci];
  CK(cudaStreamWaitEvent(st, k.ev_modes, 0));
  {
    TraceScope ts(h, SDMD_K_PHI, st);
    CK(launch_phi(ctx_phi_args(h, k), st));
  }
  CK(cudaEventRecord(k.ev_done, st));
  if (k.fr1) CK(cudaEventRecord(k.fr1, st));
  k.fr1 = nullptr;
  k.phi_pending = false;
  return SDMD_OK;
}

// Make `st` wait for every in-flight frame's eigensolver and output copies
// (they read G in place), before G is rewritten inside resident windows.
int wait_modes_readers(sdmd_s* h, cudaStream_t st) {
  for (PipeCtx& c : h->ctx)
    if (c.busy) CK(cudaStreamWaitEvent(st, c.ev_modes, 0));
  return SDMD_OK;
}

// Every deferred Phi, before anything else may touch the ring or read results.
int flush_pending(sdmd_s* h, cudaStream_t st) {
  while (!h->pending.empty()) {
    const int rc = flush_one(h, st);
    if (rc != SDMD_OK) return rc;
  }
  return SDMD_OK;
}

}  // namespace

int sdmd::set_last_error(int code, const char* msg) {
  g_err = msg;
  return code;
}

// Device bytes a depth-1 dense handle allocates (as sdmd_create does), for
// admission by footprint; the tensor-core scratch of a first rebuild or
// catch-up is not included.
int64_t sdmd::handle_device_bytes(int64_t n, int32_t m, int32_t dtype, int num_sms) {
  const int64_t elem = (dtype == SDMD_U8) ? 1 : (dtype == SDMD_C64 ? 8 : 4);
  const int64_t gsz = (dtype == SDMD_C64) ? 16 : 8;
  const int64_t slot = ((n * elem + kSlotAlign - 1) / kSlotAlign) * kSlotAlign;
  int64_t chunk = 0;
  int32_t nblk = 0;
  gram_row_schedule(slot, num_sms, &chunk, &nblk);
  return (int64_t)m * slot + 2 * (int64_t)m * m * gsz + (int64_t)m * nblk * gsz + 16 +
         modes_ws_doubles(m) * (int64_t)sizeof(double) + 8 + kPhiSchedWords * 4;
}

extern "C" {

const char* sdmd_last_error(void) { return g_err.c_str(); }

int sdmd_create(int64_t n, int32_t m, int32_t dtype, sdmd_t* out) { return sdmd_create_ex(n, m, dtype, 1, out); }

int sdmd_create_ex(int64_t n, int32_t m, int32_t dtype, int32_t depth, sdmd_t* out) {
  if (!out) return fail(SDMD_ERR_ARG, "sdmd_create: out is NULL");
  if (depth < 1 || depth > SDMD_MAX_DEPTH) return fail(SDMD_ERR_ARG, "sdmd_create_ex: depth=%d not in [1, %d]", depth, SDMD_MAX_DEPTH);
  *out = nullptr;
  if (n < 1 || n > (int64_t(1) << 34)) return fail(SDMD_ERR_ARG, "sdmd_create: n=%lld out of range", (long long)n);
  if (m < 2 || m > SDMD_MAX_M) return fail(SDMD_ERR_ARG, "sdmd_create: m=%d not in [2, %d]", m, SDMD_MAX_M);
  if (dtype != SDMD_F32 && dtype != SDMD_U8 && dtype != SDMD_C64)
    return fail(SDMD_ERR_ARG, "sdmd_create: dtype %d unknown (sparse handles: sdmd_create_sparse)", dtype);
  sdmd_s* h = new (std::nothrow) sdmd_s();
  if (!h) return fail(SDMD_ERR_OOM, "sdmd_create: host allocation failed");
  CK(cudaGetDevice(&h->device));
  CK(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
  h->n = n;
  h->m = m;
  h->depth = depth;
  h->cap = m + (depth > 1 ? depth : 0);
  h->dtype = dtype;
  h->elem = (dtype == SDMD_U8) ? 1 : (dtype == SDMD_C64 ? 8 : 4);
  h->gsz = (dtype == SDMD_C64) ? 16 : 8;
  h->slot_bytes = ((n * h->elem + kSlotAlign - 1) / kSlotAlign) * kSlotAlign;
  gram_row_schedule(h->slot_bytes, h->num_sms, &h->chunk, &h->nblk);
  const size_t ring_bytes = (size_t)h->cap * (size_t)h->slot_bytes;
  const size_t ws_bytes = (size_t)modes_ws_doubles(m) * sizeof(double);
  const size_t gbytes = (size_t)h->cap * h->cap * h->gsz;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&h->ring, ring_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&h->G, gbytes);
  if (e == cudaSuccess) e = cudaMalloc(&h->gtmp, gbytes);
  if (e == cudaSuccess) e = cudaMalloc(&h->partials, (size_t)m * h->nblk * h->gsz);
  h->nblk_alloc = h->nblk;
  if (e == cudaSuccess) e = cudaMalloc(&h->ticket, 4 * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMalloc(&h->ws, ws_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&h->status, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&h->r_dev, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&h->phi_sched, kPhiSchedWords * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(h->phi_sched, 0, kPhiSchedWords * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(h->ring, 0, ring_bytes);
  if (e == cudaSuccess) e = cudaMemset(h->G, 0, gbytes);
  if (e == cudaSuccess) e = cudaMemset(h->ticket, 0, 4 * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(h->ws, 0, ws_bytes);
  if (depth > 1) {
    h->ctx.resize(depth);
    for (PipeCtx& c : h->ctx) {
      if (e == cudaSuccess) e = cudaMalloc(&c.ws, ws_bytes);
      if (e == cudaSuccess) e = cudaMemset(c.ws, 0, ws_bytes);
      if (e == cudaSuccess) e = cudaMalloc(&c.r_dev, sizeof(int));
      if (e == cudaSuccess) e = cudaMalloc(&c.phi_sched, kPhiSchedWords * sizeof(unsigned));
      if (e == cudaSuccess) e = cudaMemset(c.phi_sched, 0, kPhiSchedWords * sizeof(unsigned));
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c.st, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.ev_g, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.ev_done, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.ev_modes, cudaEventDisableTiming);
    }
  }
  if (e == cudaSuccess) e = cudaMemset(h->status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(h->r_dev, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    const int code = (e == cudaErrorMemoryAllocation) ? SDMD_ERR_OOM : SDMD_ERR_CUDA;
    cudaGetLastError();
    free_all(h);
    delete h;
    return fail(code, "sdmd_create(n=%lld, m=%d): %s", (long long)n, m, cudaGetErrorString(e));
  }
  *out = h;
  return SDMD_OK;
}

int sdmd_create_sparse(int64_t n, int32_t m, int32_t nnz_max, sdmd_t* out) {
  if (!out) return fail(SDMD_ERR_ARG, "sdmd_create_sparse: out is NULL");
  *out = nullptr;
  if (n < 1 || n >= (int64_t(1) << 31)) return fail(SDMD_ERR_ARG, "sdmd_create_sparse: n=%lld out of range", (long long)n);
  if (m < 2 || m > SDMD_MAX_M) return fail(SDMD_ERR_ARG, "sdmd_create_sparse: m=%d not in [2, %d]", m, SDMD_MAX_M);
  if (nnz_max < 1) return fail(SDMD_ERR_ARG, "sdmd_create_sparse: nnz_max=%d", nnz_max);
  sdmd_s* h = new (std::nothrow) sdmd_s();
  if (!h) return fail(SDMD_ERR_OOM, "sdmd_create_sparse: host allocation failed");
  CK(cudaGetDevice(&h->device));
  CK(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
  h->n = n;
  h->m = m;
  h->cap = m;
  h->dtype = SDMD_C64_SPARSE;
  h->elem = 8;
  h->gsz = 16;
  h->nnz_max = nnz_max;
  h->nnz.assign(m, 0);
  h->nblk = m * sparse_chunks(nnz_max);
  const size_t ws_bytes = (size_t)modes_ws_doubles(m) * sizeof(double);
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&h->idx_ring, (size_t)m * nnz_max * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&h->val_ring, (size_t)m * nnz_max * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&h->tag, (size_t)n * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&h->tval, (size_t)n * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&h->G, (size_t)m * m * 16);
  if (e == cudaSuccess) e = cudaMalloc(&h->gtmp, (size_t)m * m * 16);
  if (e == cudaSuccess) e = cudaMalloc(&h->partials, (size_t)h->nblk * 16);
  if (e == cudaSuccess) e = cudaMalloc(&h->ticket, 4 * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMalloc(&h->ws, ws_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&h->status, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&h->r_dev, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(h->tag, 0xff, (size_t)n * sizeof(int));   // tag -1: no stamp
  if (e == cudaSuccess) e = cudaMemset(h->G, 0, (size_t)m * m * 16);
  if (e == cudaSuccess) e = cudaMemset(h->ticket, 0, 4 * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(h->status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    const int code = (e == cudaErrorMemoryAllocation) ? SDMD_ERR_OOM : SDMD_ERR_CUDA;
    cudaGetLastError();
    free_all(h);
    delete h;
    return fail(code, "sdmd_create_sparse(n=%lld, m=%d, nnz_max=%d): %s", (long long)n, m, nnz_max,
                cudaGetErrorString(e));
  }
  *out = h;
  return SDMD_OK;
}

int sdmd_push_sparse(sdmd_t h, int32_t nnz, const int32_t* idx, const void* vals, void* stream) {
  if (!h) return fail(SDMD_ERR_ARG, "sdmd_push_sparse: NULL handle");
  if (h->dtype != SDMD_C64_SPARSE) return fail(SDMD_ERR_UNSUPPORTED, "sdmd_push_sparse: dense handle");
  if (nnz < 0 || nnz > h->nnz_max) return fail(SDMD_ERR_ARG, "sdmd_push_sparse: nnz=%d not in [0, %d]", nnz, h->nnz_max);
  if (nnz > 0 && (!idx || !vals)) return fail(SDMD_ERR_ARG, "sdmd_push_sparse: NULL idx or vals");
  DeviceScope ds(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (nnz > 0 && ptr_kind(idx) != kDevice) {
    for (int32_t i = 0; i < nnz; ++i) {
      if (idx[i] < 0 || (int64_t)idx[i] >= h->n)
        return fail(SDMD_ERR_ARG, "sdmd_push_sparse: idx[%d]=%d outside [0, %lld)", i, idx[i], (long long)h->n);
      if (i > 0 && idx[i] <= idx[i - 1])
        return fail(SDMD_ERR_ARG, "sdmd_push_sparse: indices not strictly increasing at %d", i);
    }
  }
  const int32_t s = h->head;
  int* sidx = h->idx_ring + (int64_t)s * h->nnz_max;
  float2* sval = h->val_ring + (int64_t)s * h->nnz_max;
  if (nnz > 0) {
    TraceScope ts(h, SDMD_K_INGEST, st);
    CK(cudaMemcpyAsync(sidx, idx, (size_t)nnz * sizeof(int), cudaMemcpyDefault, st));
    CK(cudaMemcpyAsync(sval, vals, (size_t)nnz * sizeof(float2), cudaMemcpyDefault, st));
  }
  h->nnz[s] = nnz;
  h->stamp = (h->stamp == 0x7ffffffe) ? 1 : h->stamp + 1;
  SparseRowArgs a;
  a.idx_ring = h->idx_ring;
  a.val_ring = h->val_ring;
  a.nnz_max = h->nnz_max;
  a.tag = h->tag;
  a.tval = h->tval;
  a.n = h->n;
  a.stamp = h->stamp;
  a.c = (int32_t)(h->count + 1 < h->m ? h->count + 1 : h->m);
  a.s_first = (h->count + 1 <= h->m) ? 0 : (s + 1) % h->cap;
  a.s_new = s;
  a.m = h->cap;
  int nb = 0;
  for (int jj = 0; jj < a.c; ++jj) {
    a.chunk_start[jj] = nb;
    nb += sparse_chunks(h->nnz[(a.s_first + jj) % h->cap]);
  }
  for (int j = 0; j < h->m; ++j) a.nnz[j] = h->nnz[j];
  a.nblk = nb;
  a.partials = static_cast<double2*>(h->partials);
  a.ticket = h->ticket;
  a.G = h->G;
  {
    TraceScope ts(h, SDMD_K_GRAM_ROW, st);
    CK(launch_sparse_scatter(sidx, sval, nnz, h->n, h->stamp, h->tag, h->tval, h->status, st));
    CK(launch_sparse_row(a, st));
  }
  h->head = (s + 1) % h->cap;
  h->count += 1;
  return SDMD_OK;
}

int sdmd_destroy(sdmd_t h) {
  if (!h) return SDMD_OK;
  DeviceScope ds(h->device);
  cudaDeviceSynchronize();
  free_all(h);
  delete h;
  return SDMD_OK;
}

namespace {

bool is_pinned_host(const void* x) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, x) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeHost;
}

// The copy stream, two staging slots and their events of
// SDMD_OPT_HOST_EARLY_READ (made on first use).
int ensure_stage(sdmd_s* h) {
  if (h->stage) return SDMD_OK;
  if (cudaStreamCreateWithFlags(&h->cst, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_h2d, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_stage_free[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_stage_free[1], cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return fail(SDMD_ERR_CUDA, "host early read: stream or event creation failed");
  }
  if (cudaMalloc(&h->stage, 2 * (size_t)h->slot_bytes) != cudaSuccess) {
    cudaGetLastError();
    h->stage = nullptr;
    return fail(SDMD_ERR_OOM, "host early read: staging allocation failed");
  }
  return SDMD_OK;
}

// Ingest into slot `head` (after every in-flight reader of that slot).
// With SDMD_OPT_HOST_EARLY_READ, a snapshot in pinned host memory is copied
// at once on the handle's copy stream into one of two staging slots (after
// the push stream has moved that slot's previous snapshot into the ring), so
// the host-to-device transfer overlaps the kernels queued before it; the push
// stream then waits for it and copies device to device into the ring slot.
int ingest(sdmd_s* h, const void* x, cudaStream_t st) {
  if (h->host_early && is_pinned_host(x)) {
    const int rc = ensure_stage(h);
    if (rc != SDMD_OK) return rc;
    const int b = (int)(h->stage_i++ & 1);
    uint8_t* sb = h->stage + (int64_t)b * h->slot_bytes;
    const size_t bytes = (size_t)(h->n * h->elem);
    CK(cudaStreamWaitEvent(h->cst, h->ev_stage_free[b], 0));
    CK(cudaMemcpyAsync(sb, x, bytes, cudaMemcpyHostToDevice, h->cst));
    CK(cudaEventRecord(h->ev_h2d, h->cst));
    {
      const int rc = wait_ring_readers(h, st);
      if (rc != SDMD_OK) return rc;
    }
    TraceScope ts(h, SDMD_K_INGEST, st);
    CK(cudaStreamWaitEvent(st, h->ev_h2d, 0));
    CK(copy_snapshot(h->ring + (int64_t)h->head * h->slot_bytes, sb, bytes, h->num_sms, st));
    CK(cudaEventRecord(h->ev_stage_free[b], st));
    return SDMD_OK;
  }
  {
    const int rc = wait_ring_readers(h, st);
    if (rc != SDMD_OK) return rc;
  }
  TraceScope ts(h, SDMD_K_INGEST, st);
  CK(copy_snapshot(h->ring + (int64_t)h->head * h->slot_bytes, x, (size_t)(h->n * h->elem), h->num_sms, st));
  return SDMD_OK;
}

// Gram row of the snapshot just ingested into slot `s`, then advance the ring.
int gram_row_and_advance(sdmd_s* h, int32_t s, cudaStream_t st) {
  GramRowArgs a;
  a.ring = h->ring;
  a.slot_bytes = h->slot_bytes;
  a.chunk = h->chunk;
  a.nblk = h->nblk;
  a.c = (int32_t)(h->count + 1 < h->m ? h->count + 1 : h->m);
  a.s_first = (int32_t)((h->count + 1 - a.c) % h->cap);
  a.s_new = s;
  a.m = h->cap;
  a.partials = h->partials;
  a.ticket = h->ticket;
  a.G = h->G;
  a.status = h->status;
  {
    TraceScope ts(h, SDMD_K_GRAM_ROW, st);
    CK(launch_gram_row(h->dtype, h->f32_fp64 != 0, a, st));
  }
  h->head = (s + 1) % h->cap;
  h->count += 1;
  return SDMD_OK;
}

}  // namespace

int sdmd_push(sdmd_t h, const void* x, void* stream) {
  if (!h) return fail(SDMD_ERR_ARG, "sdmd_push: NULL handle");
  if (h->dtype == SDMD_C64_SPARSE) return fail(SDMD_ERR_UNSUPPORTED, "sdmd_push: sparse handle (use sdmd_push_sparse)");
  if (!x) return fail(SDMD_ERR_ARG, "sdmd_push: NULL snapshot");
  DeviceScope ds(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = flush_pending(h, st);
  if (rc == SDMD_OK) rc = ingest(h, x, st);
  if (rc == SDMD_OK) rc = gram_row_and_advance(h, h->head, st);
  return rc;
}

namespace {

// Lazily allocated scratch of the tensor-core Gram pass.
int ensure_gram_full_scratch(sdmd_s* h) {
  if (h->gf_partials) return SDMD_OK;
  cudaError_t e = cudaMalloc(&h->gf_partials, (size_t)kGramFullMaxCtas * 128 * 128 * sizeof(long long));
  if (e == cudaSuccess) e = cudaMalloc(&h->gf_sched, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(h->gf_sched, 0, sizeof(unsigned));
  if (e != cudaSuccess) return fail(SDMD_ERR_OOM, "tensor-core Gram scratch: %s", cudaGetErrorString(e));
  return SDMD_OK;
}

// The k newest of the c resident FP32 snapshots against the window (k = c:
// the whole Gram): up to 16 of them in one pass on the CUDA cores (FP32
// products; the pass is bound by the window's reads), more in BF16x3 on the
// tensor cores.
int gram_f32_tensor(sdmd_s* h, int c, int k, cudaStream_t st) {
  const int rc0 = ensure_gram_full_scratch(h);
  if (rc0 != SDMD_OK) return rc0;
  if (k <= kGramF32SimtMaxTargets && c <= SDMD_MAX_M) {
    GramF32SimtArgs sa;
    sa.ring = h->ring;
    sa.slot_bytes = h->slot_bytes;
    sa.n = h->n;
    sa.m = h->cap;
    sa.start = oldest_slot(h);
    sa.c = c;
    sa.k = k;
    sa.partials = reinterpret_cast<float2*>(h->gf_partials);
    sa.G = static_cast<double*>(h->G);
    TraceScope ts(h, SDMD_K_GRAM_ROW, st);
    CK(launch_gram_f32_simt(sa, h->num_sms, st));
    return SDMD_OK;
  }
  GramF32Args ga;
  ga.ring = h->ring;
  ga.slot_bytes = h->slot_bytes;
  ga.n = h->n;
  ga.m = h->cap;
  ga.start = oldest_slot(h);
  ga.t_tgt = ga.k = ga.t_old = ga.nold = 0;
  ga.split = (h->f32_bf16x3 == 2) ? 2 : 3;
  ga.partials = reinterpret_cast<float2*>(h->gf_partials);
  ga.G = static_cast<double*>(h->G);
  ga.status = h->status;
  TraceScope ts(h, SDMD_K_GRAM_ROW, st);
  CK(launch_gram_f32_tc(ga, c, k, h->num_sms, nullptr, st));
  return SDMD_OK;
}

}  // namespace

int sdmd_push_batch(sdmd_t h, int32_t k, const void* X, int64_t ld, void* stream) {
  if (!h) return fail(SDMD_ERR_ARG, "sdmd_push_batch: NULL handle");
  if (h->dtype == SDMD_C64_SPARSE) return fail(SDMD_ERR_UNSUPPORTED, "sdmd_push_batch: sparse handle");
  if (!X || k < 1 || k > h->m || ld < h->n)
    return fail(SDMD_ERR_ARG, "sdmd_push_batch: k=%d (1..%d), ld=%lld (>= n) or NULL data", k, h->m, (long long)ld);
  DeviceScope ds(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  {
    const int rc = flush_pending(h, st);
    if (rc != SDMD_OK) return rc;
  }
  const int c_after = (int)(h->count + k < h->m ? h->count + k : h->m);
  const size_t elem_bytes = (size_t)h->elem;
  const uint8_t* src = static_cast<const uint8_t*>(X);
  const bool u8_tc = h->dtype == SDMD_U8 && h->rebuild_tensor;
  const bool f32_tc = h->dtype == SDMD_F32 && h->f32_bf16x3 && k >= 2;
  if (!u8_tc && !f32_tc) {
    // k ordinary pushes (one Gram-row pass each)
    for (int j = 0; j < k; ++j) {
      const int rc = sdmd_push(h, src + (size_t)j * ld * elem_bytes, stream);
      if (rc != SDMD_OK) return rc;
    }
    return SDMD_OK;
  }
  const int rc0 = ensure_gram_full_scratch(h);
  if (rc0 != SDMD_OK) return rc0;
  // every ring-reader wait first: a failure there leaves the handle as it was
  for (int j = 0; j < k; ++j) {
    const int rc = wait_ring_readers(h, st, h->count + j);
    if (rc != SDMD_OK) return rc;
  }
  const int32_t head0 = h->head;
  const int64_t count0 = h->count;
  int copied = 0;
  cudaError_t e = cudaSuccess;
  for (int j = 0; j < k && e == cudaSuccess; ++j) {        // ingest only
    TraceScope ts(h, SDMD_K_INGEST, st);
    e = copy_snapshot(h->ring + (int64_t)((head0 + j) % h->cap) * h->slot_bytes, src + (size_t)j * ld * elem_bytes,
                      (size_t)(h->n * h->elem), h->num_sms, st);
    if (e == cudaSuccess) ++copied;
  }
  if (e == cudaSuccess) {
    // rows and columns of the k new snapshots in one pass over the window
    // (its arguments read the advanced ring)
    h->head = (int32_t)((head0 + k) % h->cap);
    h->count = count0 + k;
    const int kt = k < c_after ? k : c_after;
    if (f32_tc) {
      const int rc = gram_f32_tensor(h, c_after, kt, st);
      if (rc == SDMD_OK) return SDMD_OK;
      e = cudaErrorLaunchFailure;
    } else {
      GramFullArgs ga;
      ga.ring = h->ring;
      ga.slot_bytes = h->slot_bytes;
      ga.n = h->n;
      ga.m = h->cap;
      ga.start = oldest_slot(h);
      ga.c = c_after;
      ga.k = kt;
      ga.partials = h->gf_partials;
      ga.sched = h->gf_sched;
      ga.G = static_cast<long long*>(h->G);
      ga.status = h->status;
      TraceScope ts(h, SDMD_K_GRAM_ROW, st);
      e = launch_gram_full_tc(ga, nullptr, st);
      if (e == cudaSuccess) return SDMD_OK;
    }
    cudaGetLastError();
    h->head = head0;
    h->count = count0;
  } else {
    cudaGetLastError();
  }
  // Failure after `copied` snapshots went into the ring: those become
  // ordinary pushes (one Gram-row pass each, in order), so G matches the
  // ring again, and the call reports the error.
  for (int j = 0; j < copied; ++j) {
    const int rc = gram_row_and_advance(h, h->head, st);
    if (rc != SDMD_OK) return rc;
  }
  return fail(SDMD_ERR_CUDA, "sdmd_push_batch: %s; %d of %d snapshots pushed as single rows", cudaGetErrorString(e),
              copied, k);
}

extern "C++" int sdmd::push_many_plan(sdmd_t const* hs, const void* const* xs, int count, cudaStream_t st,
                                      BatchPlan* plan) {
  if (!hs || !xs || !plan || count < 1 || count > kMaxBatchJobs)
    return fail(SDMD_ERR_ARG, "sdmd_push_many: count=%d not in [1, %d] or NULL arrays", count, kMaxBatchJobs);
  for (int i = 0; i < count; ++i) {
    if (!hs[i] || !xs[i]) return fail(SDMD_ERR_ARG, "sdmd_push_many: NULL handle or snapshot %d", i);
    if (hs[i]->dtype == SDMD_C64_SPARSE) return fail(SDMD_ERR_UNSUPPORTED, "sdmd_push_many: sparse handle %d", i);
    if (hs[i]->device != hs[0]->device) return fail(SDMD_ERR_ARG, "sdmd_push_many: handles on different devices");
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return fail(SDMD_ERR_ARG, "sdmd_push_many: handle %d appears twice", i);
  }
  // deferred work and ring-reader waits of every handle before the plan:
  // a failure here changes no handle's ring
  for (int i = 0; i < count; ++i) {
    int rc = flush_pending(hs[i], st);
    if (rc == SDMD_OK) rc = wait_ring_readers(hs[i], st);
    if (rc != SDMD_OK) return rc;
  }
  BatchArgs& ba = plan->args;
  ba.njobs = count;
  ba.nitems = 0;
  ba.grab = hs[0]->ticket + 2;
  ba.status = hs[0]->status;
  plan->ncopies = count;
  for (int i = 0; i < count; ++i) {
    const sdmd_s* h = hs[i];
    const int32_t s_new = h->head;
    plan->dst[i] = h->ring + (int64_t)s_new * h->slot_bytes;
    plan->src[i] = xs[i];
    plan->bytes[i] = (size_t)(h->n * h->elem);
    RowJob& J = ba.job[i];
    J.ring = h->ring;
    J.slot_bytes = h->slot_bytes;
    J.chunk = h->chunk;
    J.partials = h->partials;
    J.ticket = h->ticket;
    J.G = h->G;
    J.nblk = h->nblk;
    J.c = (int32_t)(h->count + 1 < h->m ? h->count + 1 : h->m);
    J.s_first = (int32_t)((h->count + 1 - J.c) % h->cap);
    J.s_new = s_new;
    J.m = h->cap;
    J.mode = (h->dtype == SDMD_U8) ? 0 : (h->dtype == SDMD_F32 ? (h->f32_fp64 ? 3 : 1) : 2);
    J.item0 = ba.nitems;
    ba.nitems += h->nblk;
  }
  return SDMD_OK;
}

extern "C++" int sdmd::push_many_finish(sdmd_t const* hs, int count, int copied, bool launched, cudaStream_t st) {
  int rc = SDMD_OK;
  for (int i = 0; i < count && i < copied; ++i) {
    sdmd_s* h = hs[i];
    if (launched) {
      h->head = (h->head + 1) % h->cap;
      h->count += 1;
    } else {                 // its snapshot is in the ring: its own Gram row
      const int r = gram_row_and_advance(h, h->head, st);
      if (rc == SDMD_OK) rc = r;
    }
  }
  return rc;
}

int sdmd_push_many(const sdmd_t* hs, const void* const* xs, int32_t count, void* stream) {
  if (!hs || count < 1) return fail(SDMD_ERR_ARG, "sdmd_push_many: count=%d not in [1, %d] or NULL arrays", count,
                                    kMaxBatchJobs);
  if (!hs[0]) return fail(SDMD_ERR_ARG, "sdmd_push_many: NULL handle or snapshot 0");
  DeviceScope ds(hs[0]->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  BatchPlan plan;
  const int rc = push_many_plan(hs, xs, count, st, &plan);
  if (rc != SDMD_OK) return rc;
  int copied = 0;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < plan.ncopies && e == cudaSuccess; ++i) {
    TraceScope ts(hs[i], SDMD_K_INGEST, st);
    e = cudaMemcpyAsync(plan.dst[i], plan.src[i], plan.bytes[i], cudaMemcpyDefault, st);
    if (e == cudaSuccess) ++copied;
  }
  bool launched = false;
  if (e == cudaSuccess) {
    TraceScope ts(hs[0], SDMD_K_GRAM_ROW, st);
    e = launch_gram_rows_batched(plan.args, st);
    launched = e == cudaSuccess;
  }
  if (e != cudaSuccess) cudaGetLastError();
  const int rf = push_many_finish(hs, count, copied, launched, st);
  if (e != cudaSuccess)
    return fail(SDMD_ERR_CUDA, "sdmd_push_many: %s; %d of %d snapshots pushed", cudaGetErrorString(e),
                launched ? count : copied, count);
  return rf;
}

int sdmd_rebuild(sdmd_t h, void* stream) {
  if (!h) return fail(SDMD_ERR_ARG, "sdmd_rebuild: NULL handle");
  DeviceScope ds(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  {
    int rc = flush_pending(h, st);
    if (rc == SDMD_OK) rc = wait_modes_readers(h, st);
    if (rc != SDMD_OK) return rc;
  }
  const int c = resident(h);
  const int first = oldest_slot(h);
  if (h->dtype == SDMD_F32 && h->f32_bf16x3 && c >= 1) return gram_f32_tensor(h, c, c, st);
  if (h->dtype == SDMD_U8 && h->rebuild_tensor && c >= 1) {
    // one pass over the window on the tensor cores, exact int64
    const int rc0 = ensure_gram_full_scratch(h);
    if (rc0 != SDMD_OK) return rc0;
    GramFullArgs ga;
    ga.ring = h->ring;
    ga.slot_bytes = h->slot_bytes;
    ga.n = h->n;
    ga.m = h->cap;
    ga.start = first;
    ga.c = c;
    ga.k = c;
    ga.partials = h->gf_partials;
    ga.sched = h->gf_sched;
    ga.G = static_cast<long long*>(h->G);
    ga.status = h->status;
    TraceScope ts(h, SDMD_K_GRAM_ROW, st);
    CK(launch_gram_full_tc(ga, nullptr, st));
    return SDMD_OK;
  }
  // rows in time order: the final value of entry (i, j) comes from the row of
  // the later snapshot, exactly as when it was streamed
  for (int jj = 0; jj < c; ++jj) {
    const int s = (first + jj) % h->cap;
    if (h->dtype == SDMD_C64_SPARSE) {
      h->stamp = (h->stamp == 0x7ffffffe) ? 1 : h->stamp + 1;
      SparseRowArgs a;
      a.idx_ring = h->idx_ring;
      a.val_ring = h->val_ring;
      a.nnz_max = h->nnz_max;
      a.tag = h->tag;
      a.tval = h->tval;
      a.n = h->n;
      a.stamp = h->stamp;
      a.c = c;
      a.s_first = first;
      a.s_new = s;
      a.m = h->cap;
      int nb = 0;
      for (int k = 0; k < c; ++k) {
        a.chunk_start[k] = nb;
        nb += sparse_chunks(h->nnz[(first + k) % h->cap]);
      }
      for (int j = 0; j < h->m; ++j) a.nnz[j] = h->nnz[j];
      a.nblk = nb;
      a.partials = static_cast<double2*>(h->partials);
      a.ticket = h->ticket;
      a.G = h->G;
      TraceScope ts(h, SDMD_K_GRAM_ROW, st);
      CK(launch_sparse_scatter(h->idx_ring + (int64_t)s * h->nnz_max, h->val_ring + (int64_t)s * h->nnz_max,
                               h->nnz[s], h->n, h->stamp, h->tag, h->tval, h->status, st));
      CK(launch_sparse_row(a, st));
    } else {
      GramRowArgs a;
      a.ring = h->ring;
      a.slot_bytes = h->slot_bytes;
      a.chunk = h->chunk;
      a.nblk = h->nblk;
      a.c = c;
      a.s_first = first;
      a.s_new = s;
      a.m = h->cap;
      a.partials = h->partials;
      a.ticket = h->ticket;
      a.G = h->G;
      a.status = h->status;
      TraceScope ts(h, SDMD_K_GRAM_ROW, st);
      CK(launch_gram_row(h->dtype, h->f32_fp64 != 0, a, st));
    }
  }
  return SDMD_OK;
}

int sdmd_count(sdmd_t h, int64_t* count) {
  if (!h || !count) return fail(SDMD_ERR_ARG, "sdmd_count: NULL argument");
  *count = h->count;
  return SDMD_OK;
}

int sdmd_gram(sdmd_t h, void* G, void* stream) {
  if (!h || !G) return fail(SDMD_ERR_ARG, "sdmd_gram: NULL argument");
  DeviceScope ds(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int c = resident(h);
  if (c == 0) return SDMD_OK;
  const bool direct = ptr_kind(G) == kDevice;
  uint64_t* dst = direct ? static_cast<uint64_t*>(G) : static_cast<uint64_t*>(h->gtmp);
  gather_gram_kernel<<<(c * c + 255) / 256, 256, 0, st>>>(static_cast<const uint64_t*>(h->G), h->cap, c,
                                                           oldest_slot(h), (int)(h->gsz / 8), dst);
  CK(cudaGetLastError());
  if (!direct) return copy_out(G, h->gtmp, (size_t)c * c * h->gsz, st);
  return SDMD_OK;
}

int sdmd_modes_many(const sdmd_t* hs, int32_t count, const int32_t* r, void* const* lambda, int32_t* r_out,
                    void* stream) {
  if (!hs || !r || count < 1 || count > kMaxModesJobs)
    return fail(SDMD_ERR_ARG, "sdmd_modes_many: count=%d not in [1, %d] or NULL arrays", count, kMaxModesJobs);
  for (int i = 0; i < count; ++i) {
    const sdmd_s* h = hs[i];
    if (!h) return fail(SDMD_ERR_ARG, "sdmd_modes_many: NULL handle %d", i);
    if (h->dtype != SDMD_F32 && h->dtype != SDMD_U8)
      return fail(SDMD_ERR_UNSUPPORTED, "sdmd_modes_many: handle %d is not a real dense handle", i);
    if (h->device != hs[0]->device) return fail(SDMD_ERR_ARG, "sdmd_modes_many: handles on different devices");
    for (int j = 0; j < i; ++j)
      if (hs[j] == h) return fail(SDMD_ERR_ARG, "sdmd_modes_many: handle %d appears twice", i);
    const int c = resident(h);
    if (c < 3) return fail(SDMD_ERR_NOT_READY, "sdmd_modes_many: handle %d has %d snapshots, need >= 3", i, c);
    if (r[i] < 1 || r[i] > h->m - 1)
      return fail(SDMD_ERR_ARG, "sdmd_modes_many: r[%d]=%d not in [1, %d]", i, r[i], h->m - 1);
    if (lambda && lambda[i] && ptr_kind(lambda[i]) == kPageable)
      return fail(SDMD_ERR_ARG, "sdmd_modes_many: lambda[%d] must be device or pinned host memory", i);
  }
  if (r_out && ptr_kind(r_out) == kPageable)
    return fail(SDMD_ERR_ARG, "sdmd_modes_many: r_out must be device or pinned host memory");
  DeviceScope ds(hs[0]->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ModesBatch b;
  b.count = count;
  for (int i = 0; i < count; ++i) {
    sdmd_s* h = hs[i];
    const int rc = flush_pending(h, st);
    if (rc != SDMD_OK) return rc;
    ModesArgs& a = b.job[i];
    a.G = h->G;
    a.g_is_int = (h->dtype == SDMD_U8) ? 1 : 0;
    a.m = h->cap;
    a.ws_m = h->m;
    a.c = resident(h);
    a.start = oldest_slot(h);
    a.r_req = r[i];
    a.ws = h->ws;
    a.status = h->status;
    a.r_dev = h->r_dev;
  }
  {
    TraceScope ts(hs[0], SDMD_K_MODES, st);
    CK(launch_modes_batch(b, st));
  }
  for (int i = 0; i < count; ++i) {
    sdmd_s* h = hs[i];
    const ModesLayout L = modes_layout(h->m);
    if (lambda && lambda[i]) CK(cudaMemcpyAsync(lambda[i], h->ws + L.lamout, (size_t)r[i] * 16, cudaMemcpyDefault, st));
    if (r_out) CK(cudaMemcpyAsync(r_out + i, h->r_dev, sizeof(int32_t), cudaMemcpyDefault, st));
    h->last_r = r[i];
    h->last_p = resident(h) - 1;
    h->modes_count = h->count;
  }
  return SDMD_OK;
}

int sdmd_newest_row(sdmd_t h, void* row, void* stream) {
  if (!h || !row) return fail(SDMD_ERR_ARG, "sdmd_newest_row: NULL argument");
  DeviceScope ds(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  {
    const int rc = flush_pending(h, st);
    if (rc != SDMD_OK) return rc;
  }
  const int c = resident(h);
  if (c == 0) return fail(SDMD_ERR_NOT_READY, "sdmd_newest_row: no snapshot pushed yet");
  const int32_t s_new = (int32_t)((h->head + h->cap - 1) % h->cap);
  const bool direct = ptr_kind(row) == kDevice;
  uint64_t* dst = direct ? static_cast<uint64_t*>(row) : static_cast<uint64_t*>(h->gtmp);
  newest_row_kernel<<<(c + 127) / 128, 128, 0, st>>>(static_cast<const uint64_t*>(h->G), h->cap, c, oldest_slot(h),
                                                      s_new, (int)(h->gsz / 8), dst);
  CK(cudaGetLastError());
  if (!direct) return copy_out(row, h->gtmp, (size_t)c * h->gsz, st);
  return SDMD_OK;
}

int sdmd_set_newest_row(sdmd_t h, const void* row, void* stream) {
  if (!h || !row) return fail(SDMD_ERR_ARG, "sdmd_set_newest_row: NULL argument");
  DeviceScope ds(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  {
    const int rc = flush_pending(h, st);
    if (rc != SDMD_OK) return rc;
  }
  const int c = resident(h);
  if (c == 0) return fail(SDMD_ERR_NOT_READY, "sdmd_set_newest_row: no snapshot pushed yet");
  const int32_t s_new = (int32_t)((h->head + h->cap - 1) % h->cap);
  const uint64_t* src = static_cast<const uint64_t*>(row);
  if (ptr_kind(row) != kDevice) {      // staged through the gather scratch, in stream order
    CK(cudaMemcpyAsync(h->gtmp, row, (size_t)c * h->gsz, cudaMemcpyDefault, st));
    src = static_cast<const uint64_t*>(h->gtmp);
  }
  set_newest_row_kernel<<<(c + 127) / 128, 128, 0, st>>>(static_cast<uint64_t*>(h->G), h->cap, c, oldest_slot(h),
                                                          s_new, (int)(h->gsz / 8), src);
  CK(cudaGetLastError());
  if (ptr_kind(row) == kPageable) CK(cudaStreamSynchronize(st));   // the caller may reuse its buffer
  return SDMD_OK;
}

int sdmd_modes(sdmd_t h, int32_t r, void* phi, void* lambda, int32_t* r_out, void* stream) {
  if (!h) return fail(SDMD_ERR_ARG, "sdmd_modes: NULL handle");
  const bool cplx = (h->dtype == SDMD_C64 || h->dtype == SDMD_C64_SPARSE);
  if (h->dtype == SDMD_C64_SPARSE && phi)
    return fail(SDMD_ERR_UNSUPPORTED, "sdmd_modes: Fourier-sparse handles return no dense Phi (use "
                                      "sdmd_fourier_modes after this call)");
  const int c = resident(h);
  if (c < 3) return fail(SDMD_ERR_NOT_READY, "sdmd_modes: %d snapshots resident, need >= 3", c);
  if (r < 1 || r > h->m - 1) return fail(SDMD_ERR_ARG, "sdmd_modes: r=%d not in [1, %d]", r, h->m - 1);
  DeviceScope ds(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  {
    const int rc = flush_pending(h, st);
    if (rc != SDMD_OK) return rc;
  }
  if (phi && ptr_kind(phi) != kDevice)
    return fail(SDMD_ERR_ARG, "sdmd_modes: phi must be device memory (n x r complex64)");
  ModesArgs a;
  a.G = h->G;
  a.g_is_int = (h->dtype == SDMD_U8) ? 1 : 0;
  a.m = h->cap;
  a.ws_m = h->m;
  a.c = c;
  a.start = oldest_slot(h);
  a.r_req = r;
  a.ws = h->ws;
  a.status = h->status;
  a.r_dev = h->r_dev;
  {
    TraceScope ts(h, SDMD_K_MODES, st);
    if (cplx) {
      // eig of the Hermitian G_X by the real df64 solver on its 2p x 2p real
      // embedding when that fits on chip, else the FP64 Jacobi sweeps
      if (modes_embed_ok(c, r)) {
        ModesArgs e = a;
        e.embed_cx = 1;
        e.r_req = 2 * ((r < c - 1) ? r : c - 1);
        CK(launch_modes_small(e, st));
        a.cx_pre = 1;
      }
      CK(launch_modes_complex(a, st));
    } else {
      CK(launch_modes_small(a, st));
    }
  }
  const ModesLayout L = modes_layout(h->m);
  if (phi) {
    PhiArgs pa;
    pa.ring = h->ring;
    pa.slot_bytes = h->slot_bytes;
    pa.n = h->n;
    pa.dtype = h->dtype;
    pa.m = h->cap;
    pa.start = a.start;
    pa.p = c - 1;
    pa.r = r;
    pa.Mf = reinterpret_cast<const float*>(h->ws + L.Mf);
    pa.r_dev = h->r_dev;
    pa.phi = static_cast<float*>(phi);
    pa.status = h->status;
    pa.tensor = h->phi_tensor != 0;
    pa.fit_modes = h->phi_tensor == 1;
    pa.sched = h->phi_sched;
    TraceScope ts(h, SDMD_K_PHI, st);
    CK(launch_phi(pa, st));
  }
  h->last_r = r;
  h->last_p = c - 1;
  h->modes_count = h->count;
  if (lambda) {
    const int rc = copy_out(lambda, h->ws + L.lamout, (size_t)r * 16, st);
    if (rc != SDMD_OK) return rc;
  }
  if (r_out) {
    const int rc = copy_out(r_out, h->r_dev, sizeof(int32_t), st);
    if (rc != SDMD_OK) return rc;
  }
  return SDMD_OK;
}

int sdmd_step(sdmd_t h, const void* x, int32_t r, void* phi, void* lambda, int32_t* r_out, void* stream) {
  if (!h) return fail(SDMD_ERR_ARG, "sdmd_step: NULL handle");
  if (h->dtype != SDMD_F32 && h->dtype != SDMD_U8)
    return fail(SDMD_ERR_UNSUPPORTED, "sdmd_step: real dense handles only");
  if (r < 1 || r > h->m - 1) return fail(SDMD_ERR_ARG, "sdmd_step: r=%d not in [1, %d]", r, h->m - 1);
  if (h->depth < 2) {                // no pipeline: push + modes in stream order
    int rc = sdmd_push(h, x, stream);
    if (rc != SDMD_OK) return rc;
    return resident(h) >= 3 ? sdmd_modes(h, r, phi, lambda, r_out, stream) : SDMD_OK;
  }
  if (!x) return fail(SDMD_ERR_ARG, "sdmd_step: NULL snapshot");
  if (phi && ptr_kind(phi) != kDevice) return fail(SDMD_ERR_ARG, "sdmd_step: phi must be device memory");
  if ((lambda && ptr_kind(lambda) == kPageable) || (r_out && ptr_kind(r_out) == kPageable))
    return fail(SDMD_ERR_ARG, "sdmd_step: lambda / r_out must be device or pinned host memory");
  DeviceScope ds(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // Phi of frame f runs fused with the Gram row of frame f + dfuse (uint8
  // windows on the tensor cores, both windows full): one pass over the union
  // of the two windows instead of two passes over nearly the same slots.
  const int dfuse = h->depth - 1;
  const bool can_fuse = h->dtype == SDMD_U8 && h->phi_tensor && (h->m - 1) + dfuse < 256;
  const int64_t t = h->count;        // push index of this frame
  cudaEvent_t fr0 = nullptr, fr1 = nullptr;
  const bool ftrace = (t + 1 >= 3) && trace_pair(h, SDMD_K_FRAME, &fr0, &fr1);
  if (ftrace) CK(cudaEventRecord(fr0, st));
  while (!h->pending.empty() && h->ctx[h->pending.front()].frame < t - dfuse) {   // overdue: alone
    const int rc = flush_one(h, st);
    if (rc != SDMD_OK) return rc;
  }
  {
    const int rc = ingest(h, x, st);
    if (rc != SDMD_OK) return rc;
  }
  const int32_t s_new = h->head;
  const int c_t = (int32_t)(t + 1 < h->m ? t + 1 : h->m);
  bool fused = false;
  if (!h->pending.empty() && h->ctx[h->pending.front()].frame == t - dfuse) {
    PipeCtx& kf = h->ctx[h->pending.front()];
    if (can_fuse && kf.p == h->m - 1 && c_t == h->m) {
      if (!h->fgpart) {
        if (cudaMalloc(&h->fgpart, (size_t)kFusedMaxCtas * 256 * sizeof(long long)) != cudaSuccess) {
          cudaGetLastError();
          return fail(SDMD_ERR_OOM, "sdmd_step: fused Gram scratch allocation failed");
        }
      }
      PhiArgs pa = ctx_phi_args(h, kf);
      pa.fuse = 1;
      pa.ktot = kf.p + dfuse;        // X' of frame f, then the snapshots up to x_t
      pa.g0 = dfuse - 1;             // the window of x_t: rows g0 .. ktot - 1
      pa.gpart = h->fgpart;
      const int32_t slot0 = (kf.start + 1 + pa.g0) % h->cap;
      CK(cudaStreamWaitEvent(st, kf.ev_modes, 0));
      {
        TraceScope ts(h, SDMD_K_FUSED, st);
        CK(launch_phi_fused(pa, static_cast<long long*>(h->G), h->cap, s_new, slot0, st));
      }
      CK(cudaEventRecord(kf.ev_done, st));
      if (kf.fr1) CK(cudaEventRecord(kf.fr1, st));
      kf.fr1 = nullptr;
      kf.phi_pending = false;
      h->pending.pop_front();
      fused = true;
    } else {
      const int rc = flush_one(h, st);
      if (rc != SDMD_OK) return rc;
    }
  }
  if (fused) {
    h->head = (s_new + 1) % h->cap;
    h->count += 1;
  } else {
    const int rc = gram_row_and_advance(h, s_new, st);
    if (rc != SDMD_OK) return rc;
  }
  const int c = resident(h);
  if (c < 3) return SDMD_OK;         // window too short: push only
  const int ci = (int)(h->steps % h->depth);
  PipeCtx& k = h->ctx[ci];
  if (k.phi_pending) {               // (not reached with dfuse = depth - 1) its Phi first
    const int rc = flush_pending(h, st);
    if (rc != SDMD_OK) return rc;
  }
  if (k.busy) {                      // its workspace still belongs to an older frame
    CK(cudaStreamWaitEvent(st, k.ev_done, 0));
    k.busy = false;
  }
  // the eigensolver reads the window's G in place once this frame's row is in
  CK(cudaEventRecord(k.ev_g, st));
  CK(cudaStreamWaitEvent(k.st, k.ev_g, 0));
  ModesArgs a;
  a.G = h->G;
  a.g_is_int = (h->dtype == SDMD_U8) ? 1 : 0;
  a.m = h->cap;
  a.ws_m = h->m;
  a.c = c;
  a.start = oldest_slot(h);
  a.r_req = r;
  a.ws = k.ws;
  a.status = h->status;
  a.r_dev = k.r_dev;
  {
    TraceScope ts(h, SDMD_K_MODES, k.st);
    CK(launch_modes_small(a, k.st));
  }
  const ModesLayout L = modes_layout(h->m);
  if (lambda) CK(cudaMemcpyAsync(lambda, k.ws + L.lamout, (size_t)r * 16, cudaMemcpyDefault, k.st));
  if (r_out) CK(cudaMemcpyAsync(r_out, k.r_dev, sizeof(int32_t), cudaMemcpyDefault, k.st));
  CK(cudaEventRecord(k.ev_modes, k.st));
  k.phi = static_cast<float*>(phi);
  k.r = r;
  k.start = oldest_slot(h);
  k.p = c - 1;
  k.frame = h->count - 1;
  k.busy = true;
  if (phi && can_fuse) {             // Phi later, with a Gram row (or at the next sync)
    k.phi_pending = true;
    k.fr1 = ftrace ? fr1 : nullptr;
    h->pending.push_back(ci);
  } else {
    if (phi) {
      TraceScope ts(h, SDMD_K_PHI, k.st);
      CK(launch_phi(ctx_phi_args(h, k), k.st));
    }
    CK(cudaEventRecord(k.ev_done, k.st));
    if (ftrace) CK(cudaEventRecord(fr1, k.st));
  }
  h->steps += 1;
  return SDMD_OK;
}

int sdmd_autotune(sdmd_t h, int64_t* chunk_bytes, double* us, void* stream) {
  if (!h) return fail(SDMD_ERR_ARG, "sdmd_autotune: NULL handle");
  if (h->dtype == SDMD_C64_SPARSE) return fail(SDMD_ERR_UNSUPPORTED, "sdmd_autotune: dense handles only");
  if (h->count < 1) return fail(SDMD_ERR_NOT_READY, "sdmd_autotune: no snapshot pushed yet");
  DeviceScope ds(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  {
    // the timing passes rewrite the newest row and column of G (FP32 windows:
    // in each schedule's summation order), which every in-flight frame's
    // eigensolver reads in place
    int rc = flush_pending(h, st);
    if (rc == SDMD_OK) rc = wait_modes_readers(h, st);
    if (rc != SDMD_OK) return rc;
  }
  static const int kCands[] = {1, 2, 3, 4, 6};   // chunks per SM
  int64_t cch[5];
  int32_t cnb[5];
  int32_t need = h->nblk;
  for (int i = 0; i < 5; ++i) {
    gram_row_schedule_k(h->slot_bytes, h->num_sms, kCands[i], &cch[i], &cnb[i]);
    if (cnb[i] > need) need = cnb[i];
  }
  if (need > h->nblk_alloc) {
    CK(cudaStreamSynchronize(st));
    void* np = nullptr;
    if (cudaMalloc(&np, (size_t)h->m * need * h->gsz) != cudaSuccess) {
      cudaGetLastError();
      return fail(SDMD_ERR_OOM, "sdmd_autotune: partials allocation failed");
    }
    cudaFree(h->partials);
    h->partials = np;
    h->nblk_alloc = need;
  }
  // the newest snapshot's Gram row over the current window, without advancing
  GramRowArgs a;
  a.ring = h->ring;
  a.slot_bytes = h->slot_bytes;
  a.c = resident(h);
  a.s_first = oldest_slot(h);
  a.s_new = (int32_t)((h->head + h->cap - 1) % h->cap);
  a.m = h->cap;
  a.partials = h->partials;
  a.ticket = h->ticket;
  a.G = h->G;
  a.status = h->status;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  double best = 1e30;
  int bi = 1;
  int rc = SDMD_OK;
  for (int i = 0; i < 5 && rc == SDMD_OK; ++i) {
    bool dup = false;
    for (int j = 0; j < i; ++j) dup = dup || (cch[j] == cch[i]);
    if (dup) continue;
    a.chunk = cch[i];
    a.nblk = cnb[i];
    cudaError_t e = launch_gram_row(h->dtype, h->f32_fp64 != 0, a, st);   // warm-up
    double tot = 0.0;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventRecord(e0, st);
      if (e == cudaSuccess) e = launch_gram_row(h->dtype, h->f32_fp64 != 0, a, st);
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      tot += ms;
    }
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "sdmd_autotune: timing pass");
      break;
    }
    if (tot < best) {
      best = tot;
      bi = i;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != SDMD_OK) return rc;
  h->chunk = cch[bi];
  h->nblk = cnb[bi];
  a.chunk = h->chunk;                 // the newest row once more with the kept schedule
  a.nblk = h->nblk;
  CK(launch_gram_row(h->dtype, h->f32_fp64 != 0, a, st));
  if (chunk_bytes) *chunk_bytes = h->chunk;
  if (us) *us = 1e3 * best / 3.0;
  return SDMD_OK;
}

int sdmd_sync(sdmd_t h, void* stream) {
  if (!h) return fail(SDMD_ERR_ARG, "sdmd_sync: NULL handle");
  DeviceScope ds(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  {
    const int rc = flush_pending(h, st);
    if (rc != SDMD_OK) return rc;
  }
  for (PipeCtx& k : h->ctx) {
    if (k.busy) {
      CK(cudaStreamWaitEvent(st, k.ev_done, 0));
      k.busy = false;
    }
  }
  return SDMD_OK;
}

int sdmd_svd(sdmd_t h, int32_t r, double* sigma, double* V, void* stream) {
  if (!h) return fail(SDMD_ERR_ARG, "sdmd_svd: NULL handle");
  if (h->last_r == 0) return fail(SDMD_ERR_NOT_READY, "sdmd_svd: no sdmd_modes call yet");
  if (r != h->last_r) return fail(SDMD_ERR_ARG, "sdmd_svd: r=%d differs from the last sdmd_modes r=%d", r, h->last_r);
  DeviceScope ds(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const ModesLayout L = modes_layout(h->m);
  if (sigma) {
    const int rc = copy_out(sigma, h->ws + L.sig, (size_t)r * sizeof(double), st);
    if (rc != SDMD_OK) return rc;
  }
  if (V) {
    const bool cplx = (h->dtype == SDMD_C64 || h->dtype == SDMD_C64_SPARSE);
    const int64_t p2 = (int64_t)(h->m - 1 > 1 ? h->m - 1 : 1) * (h->m - 1 > 1 ? h->m - 1 : 1);
    // complex windows: V is complex (interleaved), the sixth array of the cx region
    const double* src = cplx ? h->ws + L.cx + 10 * p2 : h->ws + L.V;
    const int rc = copy_out(V, src, (size_t)r * h->last_p * sizeof(double) * (cplx ? 2 : 1), st);
    if (rc != SDMD_OK) return rc;
  }
  return SDMD_OK;
}

int sdmd_set_option(sdmd_t h, int32_t option, int64_t value) {
  if (!h) return fail(SDMD_ERR_ARG, "sdmd_set_option: NULL handle");
  switch (option) {
    case SDMD_OPT_PHI_TENSOR:
      if (value < 0 || value > 2) return fail(SDMD_ERR_ARG, "sdmd_set_option: SDMD_OPT_PHI_TENSOR value %lld not in 0..2", (long long)value);
      h->phi_tensor = (int32_t)value;
      return SDMD_OK;
    case SDMD_OPT_REBUILD_TENSOR:
      h->rebuild_tensor = value ? 1 : 0;
      return SDMD_OK;
    case SDMD_OPT_F32_BF16X3:
      if (value < 0 || value > 2) return fail(SDMD_ERR_ARG, "sdmd_set_option: SDMD_OPT_F32_BF16X3 value %lld not in 0..2", (long long)value);
      h->f32_bf16x3 = (int32_t)value;
      return SDMD_OK;
    case SDMD_OPT_F32_FP64:
      h->f32_fp64 = value ? 1 : 0;
      return SDMD_OK;
    case SDMD_OPT_HOST_EARLY_READ:
      if (h->dtype == SDMD_C64_SPARSE) return fail(SDMD_ERR_UNSUPPORTED, "sdmd_set_option: sparse handle");
      h->host_early = value ? 1 : 0;
      return SDMD_OK;
    default:
      return fail(SDMD_ERR_ARG, "sdmd_set_option: unknown option %d", option);
  }
}

int sdmd_trace(sdmd_t h, int32_t enable) {
  if (!h) return fail(SDMD_ERR_ARG, "sdmd_trace: NULL handle");
  h->trace = enable != 0;
  for (int k = 0; k < SDMD_K_COUNT; ++k) h->tr_used[k] = 0;
  return SDMD_OK;
}

int sdmd_trace_read(sdmd_t h, int32_t kernel, int64_t* launches, double* total_ms) {
  if (!h || !launches || !total_ms) return fail(SDMD_ERR_ARG, "sdmd_trace_read: NULL argument");
  if (kernel < 0 || kernel >= SDMD_K_COUNT) return fail(SDMD_ERR_ARG, "sdmd_trace_read: kernel %d", kernel);
  DeviceScope ds(h->device);
  double tot = 0.0;
  const size_t used = h->tr_used[kernel];
  for (size_t i = 0; i < used; ++i) {
    float ms = 0.f;
    CK(cudaEventSynchronize(h->tr_ev[kernel][2 * i + 1]));
    CK(cudaEventElapsedTime(&ms, h->tr_ev[kernel][2 * i], h->tr_ev[kernel][2 * i + 1]));
    tot += ms;
  }
  *launches = (int64_t)used;
  *total_ms = tot;
  h->tr_used[kernel] = 0;
  return SDMD_OK;
}

int sdmd_trace_times(sdmd_t h, int32_t kernel, double* ms, int32_t cap, int32_t* count) {
  if (!h || !ms || !count || cap < 0) return fail(SDMD_ERR_ARG, "sdmd_trace_times: bad argument");
  if (kernel < 0 || kernel >= SDMD_K_COUNT) return fail(SDMD_ERR_ARG, "sdmd_trace_times: kernel %d", kernel);
  DeviceScope ds(h->device);
  const size_t used = h->tr_used[kernel];
  int32_t k = 0;
  for (size_t i = 0; i < used; ++i) {
    float t = 0.f;
    CK(cudaEventSynchronize(h->tr_ev[kernel][2 * i + 1]));
    CK(cudaEventElapsedTime(&t, h->tr_ev[kernel][2 * i], h->tr_ev[kernel][2 * i + 1]));
    if (k < cap) ms[k++] = t;
  }
  *count = k;
  h->tr_used[kernel] = 0;
  return SDMD_OK;
}

int sdmd_amplitudes(sdmd_t h, void* b, int32_t* bg_index, void* stream) {
  if (!h) return fail(SDMD_ERR_ARG, "sdmd_amplitudes: NULL handle");
  if (h->modes_count != h->count || h->last_r < 1)
    return fail(SDMD_ERR_NOT_READY, "sdmd_amplitudes: no sdmd_modes call since the last push");
  DeviceScope ds(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const ModesLayout L = modes_layout(h->m);
  if (b) {
    const int rc = copy_out(b, h->ws + L.bamp, (size_t)h->last_r * 16, st);
    if (rc != SDMD_OK) return rc;
  }
  if (bg_index) {
    double v = -1.0;
    const int64_t pl = h->m - 1 > 1 ? h->m - 1 : 1;
    CK(cudaMemcpyAsync(&v, h->ws + L.bamp + 2 * pl, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *bg_index = (int32_t)v;
  }
  return SDMD_OK;
}

int sdmd_fourier_modes(sdmd_t h, int32_t r, int32_t* idx, void* phi, int64_t cap, int64_t* count, void* stream) {
  if (!h) return fail(SDMD_ERR_ARG, "sdmd_fourier_modes: NULL handle");
  if (h->dtype != SDMD_C64_SPARSE) return fail(SDMD_ERR_UNSUPPORTED, "sdmd_fourier_modes: Fourier-sparse handles only");
  if (h->modes_count != h->count || h->last_r < 1)
    return fail(SDMD_ERR_NOT_READY, "sdmd_fourier_modes: no sdmd_modes call since the last push");
  if (r != h->last_r) return fail(SDMD_ERR_ARG, "sdmd_fourier_modes: r=%d differs from the last sdmd_modes r=%d", r, h->last_r);
  if (!count || cap < 0) return fail(SDMD_ERR_ARG, "sdmd_fourier_modes: NULL count or negative cap");
  if (cap > 0 && (!idx || !phi || ptr_kind(idx) != kDevice || ptr_kind(phi) != kDevice))
    return fail(SDMD_ERR_ARG, "sdmd_fourier_modes: idx and phi must be device memory when cap > 0");
  DeviceScope ds(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t nw = (h->n + 31) / 32;
  if (!h->fbits) {
    cudaError_t e = cudaMalloc(&h->fbits, (size_t)nw * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&h->fprefix, (size_t)nw * sizeof(unsigned long long) + 8);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(SDMD_ERR_OOM, "sdmd_fourier_modes: bitmap allocation failed");
    }
  }
  const ModesLayout L = modes_layout(h->m);
  FourierPhiArgs fa;
  fa.idx_ring = h->idx_ring;
  fa.val_ring = h->val_ring;
  fa.nnz_max = h->nnz_max;
  for (int j = 0; j < SDMD_MAX_M; ++j) fa.nnz[j] = (j < h->m) ? h->nnz[j] : 0;
  fa.m = h->cap;
  fa.start = oldest_slot(h);
  fa.p = h->last_p;
  fa.r = r;
  fa.R = h->last_r;
  fa.Mf = reinterpret_cast<const float*>(h->ws + L.Mf);
  fa.n = h->n;
  fa.bitmap = h->fbits;
  fa.prefix = h->fprefix;
  fa.count = h->fprefix + nw;
  fa.idx_out = idx;
  fa.phi_out = static_cast<float2*>(phi);
  fa.cap = cap;
  {
    TraceScope ts(h, SDMD_K_PHI, st);
    CK(launch_fourier_phi(fa, cap > 0, st));
  }
  unsigned long long total = 0;
  CK(cudaMemcpyAsync(&total, fa.count, sizeof(total), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  *count = (int64_t)total;
  if (cap > 0 && (int64_t)total > cap)
    return fail(SDMD_ERR_ARG, "sdmd_fourier_modes: %lld coefficients in the support, cap %lld", (long long)total,
                (long long)cap);
  return SDMD_OK;
}

int sdmd_reconstruct(sdmd_t h, int64_t t, int32_t what, float* out, void* stream) {
  if (what == SDMD_RECON_BACKGROUND_SLOW || what == SDMD_RECON_FOREGROUND_SLOW)
    return fail(SDMD_ERR_ARG, "sdmd_reconstruct: the slow-mode variants take a tolerance (sdmd_reconstruct_ex)");
  return sdmd_reconstruct_ex(h, t, what, 0.0, out, stream);
}

int sdmd_pod_modes(sdmd_t h, int32_t r, float* U, void* stream) {
  if (!h) return fail(SDMD_ERR_ARG, "sdmd_pod_modes: NULL handle");
  if (h->dtype != SDMD_U8 && h->dtype != SDMD_F32)
    return fail(SDMD_ERR_UNSUPPORTED, "sdmd_pod_modes: real dense handles only");
  if (h->modes_count != h->count || h->last_r < 1)
    return fail(SDMD_ERR_NOT_READY, "sdmd_pod_modes: no sdmd_modes call since the last push");
  if (r != h->last_r) return fail(SDMD_ERR_ARG, "sdmd_pod_modes: r=%d differs from the last sdmd_modes r=%d", r, h->last_r);
  if (!U || ptr_kind(U) != kDevice || (reinterpret_cast<uintptr_t>(U) & 3u) != 0)
    return fail(SDMD_ERR_ARG, "sdmd_pod_modes: U must be device memory (n x r floats)");
  DeviceScope ds(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const ModesLayout L = modes_layout(h->m);
  PhiArgs pa;
  pa.ring = h->ring;
  pa.slot_bytes = h->slot_bytes;
  pa.n = h->n;
  pa.dtype = h->dtype;
  pa.m = h->cap;
  pa.start = oldest_slot(h);
  pa.p = h->last_p;
  pa.r = r;
  pa.Mf = nullptr;
  pa.r_dev = h->r_dev;
  pa.phi = U;
  pa.status = h->status;
  pa.tensor = 0;
  pa.sched = h->phi_sched;
  TraceScope ts(h, SDMD_K_PHI, st);
  CK(launch_pod_modes(pa, h->ws + L.V, h->ws + L.sig, reinterpret_cast<float*>(h->ws + L.Mu), st));
  return SDMD_OK;
}

int sdmd_reconstruct_ex(sdmd_t h, int64_t t, int32_t what, double tol, float* out, void* stream) {
  if (!h) return fail(SDMD_ERR_ARG, "sdmd_reconstruct: NULL handle");
  if (h->dtype != SDMD_U8 && h->dtype != SDMD_F32)
    return fail(SDMD_ERR_UNSUPPORTED, "sdmd_reconstruct: real dense handles only");
  if (h->modes_count != h->count || h->last_r < 1)
    return fail(SDMD_ERR_NOT_READY, "sdmd_reconstruct: no sdmd_modes call since the last push");
  if (what < SDMD_RECON_MODES || what > SDMD_RECON_FOREGROUND_SLOW)
    return fail(SDMD_ERR_ARG, "sdmd_reconstruct: what=%d", what);
  const bool fg = (what == SDMD_RECON_FOREGROUND || what == SDMD_RECON_FOREGROUND_SLOW);
  if (!(tol >= 0.0)) return fail(SDMD_ERR_ARG, "sdmd_reconstruct: tol must be >= 0");
  const int c = h->last_p + 1;
  if (t < 0 || (fg && t > c - 1))
    return fail(SDMD_ERR_ARG, "sdmd_reconstruct: t=%lld out of range", (long long)t);
  if (!out || ptr_kind(out) != kDevice || (reinterpret_cast<uintptr_t>(out) & 15u) != 0)
    return fail(SDMD_ERR_ARG, "sdmd_reconstruct: out must be 16-byte aligned device memory (n floats)");
  DeviceScope ds(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const ModesLayout L = modes_layout(h->m);
  const int64_t pl = h->m - 1 > 1 ? h->m - 1 : 1;
  ReconArgs ra;
  ra.ring = h->ring;
  ra.slot_bytes = h->slot_bytes;
  ra.n = h->n;
  ra.dtype = h->dtype;
  ra.m = h->cap;
  ra.start = oldest_slot(h);
  ra.p = h->last_p;
  ra.R = h->last_r;
  ra.Mf = reinterpret_cast<const float*>(h->ws + L.Mf);
  ra.lamout = h->ws + L.lamout;
  ra.bamp = h->ws + L.bamp;
  ra.bgi = h->ws + L.bamp + 2 * pl;
  ra.r_dev = h->r_dev;
  ra.t = t;
  ra.what = what;
  ra.urec = reinterpret_cast<float*>(h->ws + L.urec);
  ra.out = out;
  ra.xt_slot = fg ? (int32_t)((ra.start + t) % h->cap) : -1;
  ra.slow_tol = tol;
  CK(launch_reconstruct(ra, st));
  return SDMD_OK;
}

int sdmd_modes_phase_cycles(sdmd_t h, int64_t* cycles, int32_t count, void* stream) {
  if (!h || !cycles || count < 1 || count > 16) return fail(SDMD_ERR_ARG, "sdmd_modes_phase_cycles: bad argument");
  DeviceScope ds(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const ModesLayout L = modes_layout(h->m);
  CK(cudaMemcpyAsync(cycles, h->ws + L.clk, (size_t)count * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return SDMD_OK;
}

int sdmd_status(sdmd_t h, void* stream) {
  if (!h) return fail(SDMD_ERR_ARG, "sdmd_status: NULL handle");
  DeviceScope ds(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  {
    const int rc = flush_pending(h, st);
    if (rc != SDMD_OK) return rc;
  }
  for (PipeCtx& k : h->ctx)
    if (k.busy) CK(cudaStreamWaitEvent(st, k.ev_done, 0));
  int v = 0;
  CK(cudaMemcpyAsync(&v, h->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemsetAsync(h->status, 0, sizeof(int), st));
  CK(cudaStreamSynchronize(st));
  if (v & kDevTimeout) return fail(SDMD_ERR_TIMEOUT, "device wait timed out");
  if (v & kDevRank) return fail(SDMD_ERR_RANK, "eigensolver iteration cap reached");
  if (v & kDevRange) return fail(SDMD_ERR_ARG, "sparse coefficient index outside [0, n) (entry skipped)");
  return SDMD_OK;
}

}  // extern "C"
