// Exact DMD modes Phi = X' (V Sigma^-1 W) (Sec. 2.2, Eq. 9; Algorithm 2's
// phi = X[:, 1:] * vsiw). X' is read in place from the ring buffer (logical
// columns 1..c-1 of the window); M = V Sigma^-1 W is the small p x r complex
// matrix produced by the FP64 kernel, rounded to FP32 here.
//
// A CTA owns a tile of kPos positions and streams the p slots of X' through
// shared memory in chunks of kSlots slots with cp.async double buffering
// (each chunk row is kPos contiguous elements of one slot: 16-byte copies,
// fully coalesced). Each thread owns kPos / 256 positions and KT modes and
// accumulates 2*KT FP32 sums per position against M broadcast from shared
// memory; gridDim.y tiles the modes. Columns beyond the kept rank have M = 0
// and come out as zeros.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sdmd_internal.cuh"

namespace sdmd {

namespace {

constexpr int kPhiThreads = 256;
constexpr int kSlots = 32;          // slots per staged chunk

template <typename T>
struct PhiTraits;
template <>
struct PhiTraits<uint8_t> {
  static constexpr int kPos = 512;  // positions per tile (2 per thread)
};
template <>
struct PhiTraits<float> {
  static constexpr int kPos = 256;  // positions per tile (1 per thread)
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_le1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// Stage slots [a0, a0 + ns) of the position tile starting at i0 (elements).
template <typename T>
__device__ __forceinline__ void stage_chunk(const PhiArgs& a, uint8_t* buf, int a0, int ns, int64_t i0) {
  constexpr int kPos = PhiTraits<T>::kPos;
  constexpr int kRowBytes = kPos * (int)sizeof(T);
  constexpr int kVec = kRowBytes / 16;
  for (int idx = threadIdx.x; idx < ns * kVec; idx += kPhiThreads) {
    const int s = idx / kVec, v = idx - s * kVec;
    const int slot = (a.start + 1 + a0 + s) % a.m;
    const uint8_t* src = a.ring + (int64_t)slot * a.slot_bytes + i0 * (int64_t)sizeof(T) + 16 * v;
    cp_async16(buf + s * kRowBytes + 16 * v, src);
  }
}

template <typename T, int KT>
__global__ void __launch_bounds__(kPhiThreads, 2) phi_tile_kernel(PhiArgs a) {
  constexpr int kPos = PhiTraits<T>::kPos;
  constexpr int kPer = kPos / kPhiThreads;               // positions per thread
  constexpr int kRowBytes = kPos * (int)sizeof(T);
  extern __shared__ __align__(16) uint8_t smem[];
  uint8_t* buf0 = smem;
  uint8_t* buf1 = smem + kSlots * kRowBytes;
  float* Ms = reinterpret_cast<float*>(smem + 2 * kSlots * kRowBytes);   // p x 2*KT
  const int k0 = blockIdx.y * KT;
  const int kt = min(KT, a.r - k0);
  for (int idx = threadIdx.x; idx < a.p * 2 * KT; idx += kPhiThreads) {
    const int row = idx / (2 * KT), q = idx - row * (2 * KT);
    Ms[idx] = (q < 2 * kt) ? a.Mf[(int64_t)row * 2 * a.r + 2 * k0 + q] : 0.f;
  }
  const int64_t ntiles = (a.n + kPos - 1) / kPos;
  const int nchunks = (a.p + kSlots - 1) / kSlots;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t i0 = tile * kPos;
    float acc[kPer][2 * KT];
#pragma unroll
    for (int u = 0; u < kPer; ++u)
#pragma unroll
      for (int q = 0; q < 2 * KT; ++q) acc[u][q] = 0.f;
    __syncthreads();   // previous tile's buffers are free
    stage_chunk<T>(a, buf0, 0, min(kSlots, a.p), i0);
    cp_async_commit();
    for (int c = 0; c < nchunks; ++c) {
      uint8_t* cur = (c & 1) ? buf1 : buf0;
      uint8_t* nxt = (c & 1) ? buf0 : buf1;
      const int a0 = c * kSlots;
      const int ns = min(kSlots, a.p - a0);
      if (c + 1 < nchunks) {
        stage_chunk<T>(a, nxt, a0 + kSlots, min(kSlots, a.p - a0 - kSlots), i0);
        cp_async_commit();
        cp_async_wait_le1();
      } else {
        cp_async_wait_all();
      }
      __syncthreads();
      for (int s = 0; s < ns; ++s) {
        float x[kPer];
        if constexpr (sizeof(T) == 1) {
          const unsigned short v = *reinterpret_cast<const unsigned short*>(cur + s * kRowBytes + 2 * threadIdx.x);
          x[0] = (float)(v & 0xffu);
          x[1] = (float)(v >> 8);
        } else {
          x[0] = *reinterpret_cast<const float*>(cur + s * kRowBytes + 4 * threadIdx.x);
        }
        const float4* mrow = reinterpret_cast<const float4*>(Ms + (a0 + s) * 2 * KT);
#pragma unroll
        for (int q4 = 0; q4 < KT / 2; ++q4) {
          const float4 mv = mrow[q4];
#pragma unroll
          for (int u = 0; u < kPer; ++u) {
            acc[u][4 * q4 + 0] = fmaf(x[u], mv.x, acc[u][4 * q4 + 0]);
            acc[u][4 * q4 + 1] = fmaf(x[u], mv.y, acc[u][4 * q4 + 1]);
            acc[u][4 * q4 + 2] = fmaf(x[u], mv.z, acc[u][4 * q4 + 2]);
            acc[u][4 * q4 + 3] = fmaf(x[u], mv.w, acc[u][4 * q4 + 3]);
          }
        }
      }
      __syncthreads();   // `cur` may be overwritten by the next stage
    }
    // write: mode k, positions i0 + kPer*tid + u (complex64)
    const int64_t ibase = i0 + (int64_t)kPer * threadIdx.x;
#pragma unroll
    for (int q = 0; q < KT; ++q) {
      if (q < kt) {
        float2* col = reinterpret_cast<float2*>(a.phi) + (int64_t)(k0 + q) * a.n;
#pragma unroll
        for (int u = 0; u < kPer; ++u)
          if (ibase + u < a.n) col[ibase + u] = make_float2(acc[u][2 * q], acc[u][2 * q + 1]);
      }
    }
  }
}

template <typename T, int KT>
cudaError_t launch_t(const PhiArgs& a, cudaStream_t st, int sms) {
  constexpr int kPos = PhiTraits<T>::kPos;
  const size_t smem = 2 * kSlots * kPos * sizeof(T) + (size_t)a.p * 2 * KT * sizeof(float);
  static size_t attr = 0;
  if (smem > attr) {
    cudaError_t e = cudaFuncSetAttribute(phi_tile_kernel<T, KT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    attr = smem;
  }
  const int64_t ntiles = (a.n + kPos - 1) / kPos;
  const int ky = (a.r + KT - 1) / KT;
  int64_t bx = (int64_t)2 * sms;                // persistent: two CTAs per SM over all mode tiles
  bx = (bx + ky - 1) / ky;
  if (bx < 1) bx = 1;
  if (bx > ntiles) bx = ntiles;
  dim3 grid((unsigned)bx, (unsigned)ky);
  phi_tile_kernel<T, KT><<<grid, kPhiThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_for_type(const PhiArgs& a, cudaStream_t st, int sms) {
  // modes per pass: the smallest even tile >= r, at most 16
  const int kt = a.r >= 16 ? 16 : ((a.r + 1) / 2) * 2;
  switch (kt) {
    case 2: return launch_t<T, 2>(a, st, sms);
    case 4: return launch_t<T, 4>(a, st, sms);
    case 6: return launch_t<T, 6>(a, st, sms);
    case 8: return launch_t<T, 8>(a, st, sms);
    case 10: return launch_t<T, 10>(a, st, sms);
    case 12: return launch_t<T, 12>(a, st, sms);
    case 14: return launch_t<T, 14>(a, st, sms);
    default: return launch_t<T, 16>(a, st, sms);
  }
}

}  // namespace

cudaError_t launch_phi(const PhiArgs& a, cudaStream_t st) {
  if (a.tensor && a.dtype == SDMD_U8) {
    const cudaError_t e = launch_phi_tc(a, st);
    if (e != cudaErrorNotSupported) return e;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (a.dtype == SDMD_U8) return launch_for_type<uint8_t>(a, st, sms > 0 ? sms : 1);
  return launch_for_type<float>(a, st, sms > 0 ? sms : 1);
}

}  // namespace sdmd
