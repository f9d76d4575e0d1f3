// Gram row without any device allocation (sdmd_gram_row_static).
//
// Same computation as the Gram-row kernel behind sdmd_push -- g_j = <x_j, y>
// for c snapshots x_j and one snapshot y -- for callers that cannot allocate
// device memory. Its only scratch (per-CTA partial sums and a completion
// ticket) lives in a file-scope __device__ array of fixed size, so the entry
// point never calls cudaMalloc, cudaFree or any allocating routine.
//
// Unlike the ring-buffer kernel it reads caller buffers with no zero padding,
// so it handles a ragged tail of fewer than 16 bytes with scalar loads.
// Summation order (FP32 path) differs from sdmd_push's kernel: results agree
// to rounding, not bit for bit; uint8 results are exact either way.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>

#include <mutex>
#include <type_traits>

#include "sdmd.h"
#include "sdmd_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxRows = SDMD_GRAM_ROW_STATIC_MAX_C;       // snapshots per call
constexpr int kMaxBlocks = 512;                            // CTAs per call
constexpr int64_t kChunkAlign = 4096;                      // bytes per CTA, multiple of
constexpr int64_t kPartialBytes = (int64_t)kMaxRows * kMaxBlocks * 8;

// [kMaxRows][kMaxBlocks] 8-byte partials, then the 4-byte completion ticket.
// Shared by every call in the process on this device; the host code below
// only ever passes its device address (from cudaGetSymbolAddress).
__device__ __align__(256) unsigned char g_gram_row_scratch[kPartialBytes + 256];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Formats the message that sdmd_last_error() returns on this thread.
int set_err(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  return sdmd::set_last_error(code, buf);
}

__device__ __forceinline__ long long warp_sum(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One CTA per byte range [beg, end) of the snapshots; warp w takes snapshots
// w, w+8, ... Lanes stride 16-byte vectors; the last CTA's ragged tail
// (nbytes % 16 bytes) is added by lane 0 with scalar loads.
template <bool kU8>
__global__ void __launch_bounds__(kThreads)
gram_row_static_kernel(const uint8_t* X, int64_t ld_bytes, int c, const uint8_t* y, int64_t nbytes,
                       int64_t chunk, int nblk, void* g, unsigned char* scratch) {
  using Acc = typename std::conditional<kU8, long long, double>::type;
  Acc* P = reinterpret_cast<Acc*>(scratch);
  unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch + kPartialBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t beg = (int64_t)blockIdx.x * chunk;
  const int64_t end = min(beg + chunk, nbytes);
  const int64_t vend = beg + ((end - beg) / 16) * 16;
  for (int j = warp; j < c; j += kWarps) {
    const uint8_t* xj = X + (int64_t)j * ld_bytes;
    Acc s = 0;
    for (int64_t o = beg + 16 * lane; o < vend; o += 16 * 32 * 4) {
      // up to 4 independent 16-byte vectors per lane per step
      if constexpr (kU8) {
        unsigned int t = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t q = o + u * 512;
          if (q < vend) {
            const uint4 a = __ldcs(reinterpret_cast<const uint4*>(xj + q));
            const uint4 b = __ldg(reinterpret_cast<const uint4*>(y + q));
            t = __dp4a(a.x, b.x, t);
            t = __dp4a(a.y, b.y, t);
            t = __dp4a(a.z, b.z, t);
            t = __dp4a(a.w, b.w, t);
          }
        }
        s += (long long)t;   // <= 64 products of 255^2 per step: no u32 overflow
      } else {
        float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t q = o + u * 512;
          if (q < vend) {
            const float4 a = __ldcs(reinterpret_cast<const float4*>(xj + q));
            const float4 b = __ldg(reinterpret_cast<const float4*>(y + q));
            f0 = fmaf(a.x, b.x, f0);
            f1 = fmaf(a.y, b.y, f1);
            f2 = fmaf(a.z, b.z, f2);
            f3 = fmaf(a.w, b.w, f3);
          }
        }
        s += (double)((f0 + f1) + (f2 + f3));
      }
    }
    s = warp_sum(s);
    if (lane == 0) {
      for (int64_t q = vend; q < end; q += (kU8 ? 1 : 4)) {
        if constexpr (kU8)
          s += (long long)xj[q] * (long long)y[q];
        else
          s += (double)(*reinterpret_cast<const float*>(xj + q) * *reinterpret_cast<const float*>(y + q));
      }
      P[(int64_t)j * nblk + blockIdx.x] = s;
    }
  }
  // last CTA to finish sums the partials in a fixed order
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == (unsigned int)nblk - 1u);
  __syncthreads();
  if (!last) return;
  __threadfence();
  Acc* out = static_cast<Acc*>(g);
  for (int j = warp; j < c; j += kWarps) {
    Acc s = 0;
    for (int b = lane; b < nblk; b += 32) s += __ldcg(P + (int64_t)j * nblk + b);
    s = warp_sum(s);
    if (lane == 0) out[j] = s;
  }
  if (threadIdx.x == 0) *ticket = 0u;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device address of the scratch array on the current device, looked up once
// per device (the first call on each device does the lookup).
int scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_err(SDMD_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_err(SDMD_ERR_UNSUPPORTED, "device ordinal %d >= %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_gram_row_scratch);
    if (e != cudaSuccess || !p)
      return set_err(SDMD_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return SDMD_OK;
}

}  // namespace

extern "C" SDMD_API int sdmd_gram_row_static(int32_t dtype, const void* X, int64_t ld, int32_t c,
                                             const void* y, int64_t n, void* g, void* stream) {
  if (dtype != SDMD_F32 && dtype != SDMD_U8) return set_err(SDMD_ERR_ARG, "dtype %d unknown", dtype);
  if (c < 1 || c > kMaxRows) return set_err(SDMD_ERR_ARG, "c=%d not in [1, %d]", c, kMaxRows);
  if (n < 1 || n > (int64_t(1) << 34)) return set_err(SDMD_ERR_ARG, "n=%lld out of range", (long long)n);
  if (ld < n) return set_err(SDMD_ERR_ARG, "ld=%lld < n=%lld", (long long)ld, (long long)n);
  const int64_t elem = (dtype == SDMD_U8) ? 1 : 4;
  const int64_t ld_bytes = ld * elem, nbytes = n * elem;
  if (!X || !y || !g) return set_err(SDMD_ERR_ARG, "NULL buffer");
  if ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(y)) % 16 != 0 || ld_bytes % 16 != 0)
    return set_err(SDMD_ERR_ARG, "X and y must be 16-byte aligned and ld * sizeof(elem) a multiple of 16");
  if (!is_device_ptr(X) || !is_device_ptr(y) || !is_device_ptr(g))
    return set_err(SDMD_ERR_ARG, "X, y and g must be device memory");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0, sdev = 0;
  cudaGetDevice(&dev);
  // the scratch address is this device's; a stream of another device would
  // launch the kernel there with a foreign address
  cudaError_t e = cudaStreamGetDevice(st, &sdev);
  if (e != cudaSuccess) return set_err(SDMD_ERR_ARG, "cudaStreamGetDevice: %s", cudaGetErrorString(e));
  if (sdev != dev)
    return set_err(SDMD_ERR_ARG, "stream belongs to device %d, the current device is %d", sdev, dev);
  unsigned char* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != SDMD_OK) return rc;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // split n into CTA chunks of whole 4 KiB units; at most kMaxBlocks CTAs
  const int64_t units = (nbytes + kChunkAlign - 1) / kChunkAlign;
  int64_t want = 2LL * (sms > 0 ? sms : 1);
  if (want > kMaxBlocks) want = kMaxBlocks;
  if (want > units) want = units;
  const int64_t per = (units + want - 1) / want;
  const int64_t chunk = per * kChunkAlign;
  const int nblk = (int)((units + per - 1) / per);
  if (nblk > kMaxBlocks) return set_err(SDMD_ERR_ARG, "split needs %d CTAs > %d", nblk, kMaxBlocks);
  // the ticket must start at zero; the partials are always written before read
  e = cudaMemsetAsync(scratch + kPartialBytes, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return set_err(SDMD_ERR_CUDA, "cudaMemsetAsync(ticket): %s", cudaGetErrorString(e));
  const uint8_t* Xb = static_cast<const uint8_t*>(X);
  const uint8_t* yb = static_cast<const uint8_t*>(y);
  if (dtype == SDMD_U8)
    gram_row_static_kernel<true><<<nblk, kThreads, 0, st>>>(Xb, ld_bytes, c, yb, nbytes, chunk, nblk, g, scratch);
  else
    gram_row_static_kernel<false><<<nblk, kThreads, 0, st>>>(Xb, ld_bytes, c, yb, nbytes, chunk, nblk, g, scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_err(SDMD_ERR_CUDA, "gram_row_static launch: %s", cudaGetErrorString(e));
  return SDMD_OK;
}
