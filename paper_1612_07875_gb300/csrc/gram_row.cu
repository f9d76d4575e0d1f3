// Streaming Gram row: the one new row/column of G = X^H X per pushed snapshot
// (Sec. 3.1, Eq. 12b; Algorithm 1, the X^T X[:, -1] product). Every resident
// snapshot x_j is dotted with the new snapshot x_new; O(n m) work that reads
// each window byte exactly once, so the kernel is HBM-bound.
//
// Decomposition: the n dimension (in bytes, padded to whole 4 KiB units) is
// split into `nblk` contiguous chunks, one per CTA, about two CTAs per SM.
// A CTA stages its chunk of x_new in shared memory 16 KiB at a time; each of
// its 8 warps streams whole slots (warp w takes slots w, w+8, ...) with
// 16-byte loads, 8 in flight per lane, and reduces each slot's sub-chunk with
// warp shuffles into a per-CTA accumulator. The per-CTA partials go to a
// small [slot][CTA] array; the last CTA to finish (atomic ticket, no waiting)
// sums them in a fixed order and writes row and column `s_new` of G.
//
//  - uint8: __dp4a (4 u8 x u8 products summed into u32). A lane sums at most
//    16 KiB / 32 = 512 products (< 255^2 * 512 < 2^32) before the value goes
//    to int64, so the result is exact and independent of order.
//  - float32: four FP32 FMA chains of 8 products per step per lane, then the
//    step's sum is added in FP64; the cross-lane / cross-CTA sums are FP64 in
//    a fixed order, so results are deterministic for a given schedule.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sdmd_internal.cuh"

namespace sdmd {

namespace {

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

// Stage `len` bytes (multiple of 16) of x_new into shared memory.
__device__ __forceinline__ void stage_xnew(uint8_t* xs, const uint8_t* src, int len) {
  for (int o = threadIdx.x * 16; o < len; o += blockDim.x * 16)
    *reinterpret_cast<uint4*>(xs + o) = __ldcg(reinterpret_cast<const uint4*>(src + o));
}

// Last CTA: fixed-order sums of the per-CTA partials, symmetric insert into G.
template <typename Acc>
__device__ void finish_row(const GramRowArgs& a) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int t = atomicAdd(a.ticket, 1u);
    last = (t == (unsigned int)a.nblk - 1u);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Acc* P = static_cast<const Acc*>(a.partials);
  Acc* G = static_cast<Acc*>(a.G);
  for (int j = warp; j < a.c; j += kGrWarps) {
    Acc s = 0;
    for (int b = lane; b < a.nblk; b += 32) s += __ldcg(P + (int64_t)j * a.nblk + b);
    s = warp_sum(s);
    if (lane == 0) {
      G[(int64_t)a.s_new * a.m + j] = s;
      G[(int64_t)j * a.m + a.s_new] = s;
    }
  }
  if (threadIdx.x == 0) *a.ticket = 0u;  // ready for the next launch
}

__global__ void __launch_bounds__(kGrThreads)
gram_row_u8_kernel(GramRowArgs a) {
  __shared__ __align__(16) uint8_t xs[kGrSub];
  __shared__ long long acc[SDMD_MAX_M];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t beg = (int64_t)blockIdx.x * a.chunk;
  const int64_t end = min(beg + a.chunk, a.slot_bytes);
  for (int j = threadIdx.x; j < a.c; j += blockDim.x) acc[j] = 0;
  const uint8_t* xnew = a.ring + (int64_t)a.s_new * a.slot_bytes;
  for (int64_t sub = beg; sub < end; sub += kGrSub) {
    const int len = (int)min((int64_t)kGrSub, end - sub);   // multiple of kGrStep
    __syncthreads();
    stage_xnew(xs, xnew + sub, len);
    __syncthreads();
    for (int j = warp; j < a.c; j += kGrWarps) {
      const uint8_t* xj = a.ring + (int64_t)j * a.slot_bytes + sub;
      unsigned int s = 0;
      for (int o = lane * 16; o < len; o += kGrStep) {
        uint4 v[kGrUnroll];
#pragma unroll
        for (int u = 0; u < kGrUnroll; ++u)
          v[u] = __ldcs(reinterpret_cast<const uint4*>(xj + o + u * 512));
#pragma unroll
        for (int u = 0; u < kGrUnroll; ++u) {
          const uint4 w = *reinterpret_cast<const uint4*>(xs + o + u * 512);
          s = __dp4a(v[u].x, w.x, s);
          s = __dp4a(v[u].y, w.y, s);
          s = __dp4a(v[u].z, w.z, s);
          s = __dp4a(v[u].w, w.w, s);
        }
      }
      const long long t = warp_sum((long long)s);
      if (lane == 0) acc[j] += t;
    }
  }
  __syncthreads();
  long long* P = static_cast<long long*>(a.partials);
  for (int j = threadIdx.x; j < a.c; j += blockDim.x) P[(int64_t)j * a.nblk + blockIdx.x] = acc[j];
  finish_row<long long>(a);
}

__global__ void __launch_bounds__(kGrThreads)
gram_row_f32_kernel(GramRowArgs a) {
  __shared__ __align__(16) uint8_t xs[kGrSub];
  __shared__ double acc[SDMD_MAX_M];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t beg = (int64_t)blockIdx.x * a.chunk;
  const int64_t end = min(beg + a.chunk, a.slot_bytes);
  for (int j = threadIdx.x; j < a.c; j += blockDim.x) acc[j] = 0.0;
  const uint8_t* xnew = a.ring + (int64_t)a.s_new * a.slot_bytes;
  for (int64_t sub = beg; sub < end; sub += kGrSub) {
    const int len = (int)min((int64_t)kGrSub, end - sub);
    __syncthreads();
    stage_xnew(xs, xnew + sub, len);
    __syncthreads();
    for (int j = warp; j < a.c; j += kGrWarps) {
      const uint8_t* xj = a.ring + (int64_t)j * a.slot_bytes + sub;
      double s = 0.0;
      for (int o = lane * 16; o < len; o += kGrStep) {
        float4 v[kGrUnroll];
#pragma unroll
        for (int u = 0; u < kGrUnroll; ++u)
          v[u] = __ldcs(reinterpret_cast<const float4*>(xj + o + u * 512));
        float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;
#pragma unroll
        for (int u = 0; u < kGrUnroll; ++u) {
          const float4 w = *reinterpret_cast<const float4*>(xs + o + u * 512);
          f0 = fmaf(v[u].x, w.x, f0);
          f1 = fmaf(v[u].y, w.y, f1);
          f2 = fmaf(v[u].z, w.z, f2);
          f3 = fmaf(v[u].w, w.w, f3);
        }
        s += (double)((f0 + f1) + (f2 + f3));
      }
      s = warp_sum(s);
      if (lane == 0) acc[j] += s;
    }
  }
  __syncthreads();
  double* P = static_cast<double*>(a.partials);
  for (int j = threadIdx.x; j < a.c; j += blockDim.x) P[(int64_t)j * a.nblk + blockIdx.x] = acc[j];
  finish_row<double>(a);
}

}  // namespace

void gram_row_schedule(int64_t slot_bytes, int num_sms, int64_t* chunk, int32_t* nblk) {
  const int64_t units = (slot_bytes + kGrStep - 1) / kGrStep;
  int64_t want = 2LL * (num_sms > 0 ? num_sms : 1);
  if (want > units) want = units;
  const int64_t per = (units + want - 1) / want;     // units per CTA
  *chunk = per * kGrStep;
  *nblk = (int32_t)((units + per - 1) / per);
}

cudaError_t launch_gram_row(int dtype, const GramRowArgs& a, cudaStream_t st) {
  if (dtype == SDMD_U8)
    gram_row_u8_kernel<<<a.nblk, kGrThreads, 0, st>>>(a);
  else
    gram_row_f32_kernel<<<a.nblk, kGrThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sdmd
