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
//
// The same kernel with a real p x r matrix and real output, reading X
// (columns 0..c-2) instead of X', gives the POD modes U = X V Sigma^-1
// (Sec. 2.1, Eq. 4) for sdmd_pod_modes. Complex64 windows (dense complex
// handles) take the complex product X' M (four FMAs per position and mode).
#include <cuda_runtime.h>
#include <stdint.h>

#include "sdmd_internal.cuh"

namespace sdmd {

namespace {

constexpr int kPhiThreads = 256;

template <typename T>
struct PhiTraits;
template <>
struct PhiTraits<uint8_t> {
  static constexpr int kPos = 512;  // positions per tile (2 per thread)
  static constexpr int kSlots = 32; // slots per staged chunk
};
template <>
struct PhiTraits<float> {
  static constexpr int kPos = 256;  // positions per tile (1 per thread)
  static constexpr int kSlots = 32;
};
template <>
struct PhiTraits<float2> {          // complex64 (re, im)
  static constexpr int kPos = 256;
  static constexpr int kSlots = 16; // 2 x 16 x 2 KB staged: two CTAs per SM
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
    const int slot = (a.start + a.xoff + a0 + s) % a.m;
    const uint8_t* src = a.ring + (int64_t)slot * a.slot_bytes + i0 * (int64_t)sizeof(T) + 16 * v;
    cp_async16(buf + s * kRowBytes + 16 * v, src);
  }
}

template <typename T, int KT, bool kReal>
__global__ void __launch_bounds__(kPhiThreads, 2) phi_tile_kernel(PhiArgs a) {
  constexpr int kPos = PhiTraits<T>::kPos;
  constexpr int kPer = kPos / kPhiThreads;               // positions per thread
  constexpr int kRowBytes = kPos * (int)sizeof(T);
  constexpr int kW = kReal ? KT : 2 * KT;                // sums per position
  constexpr int kSlots = PhiTraits<T>::kSlots;
  extern __shared__ __align__(16) uint8_t smem[];
  uint8_t* buf0 = smem;
  uint8_t* buf1 = smem + kSlots * kRowBytes;
  float* Ms = reinterpret_cast<float*>(smem + 2 * kSlots * kRowBytes);   // p x kW
  const int k0 = blockIdx.y * KT;
  const int kt = min(KT, a.r - k0);
  for (int idx = threadIdx.x; idx < a.p * kW; idx += kPhiThreads) {
    const int row = idx / kW, q = idx - row * kW;
    if constexpr (kReal)
      Ms[idx] = (q < kt) ? a.Mf[(int64_t)row * a.r + k0 + q] : 0.f;
    else
      Ms[idx] = (q < 2 * kt) ? a.Mf[(int64_t)row * 2 * a.r + 2 * k0 + q] : 0.f;
  }
  const int64_t ntiles = (a.n + kPos - 1) / kPos;
  const int nchunks = (a.p + kSlots - 1) / kSlots;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t i0 = tile * kPos;
    float acc[kPer][kW];
#pragma unroll
    for (int u = 0; u < kPer; ++u)
#pragma unroll
      for (int q = 0; q < kW; ++q) acc[u][q] = 0.f;
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
        if constexpr (sizeof(T) == 8) {   // complex64: phi += x m, 4 FMAs per mode
          const float2 xc = *reinterpret_cast<const float2*>(cur + s * kRowBytes + 8 * threadIdx.x);
          const float4* mrow = reinterpret_cast<const float4*>(Ms + (a0 + s) * kW);
#pragma unroll
          for (int q2 = 0; q2 < KT / 2; ++q2) {
            const float4 mv = mrow[q2];            // modes 2 q2 and 2 q2 + 1: (re, im, re, im)
            acc[0][4 * q2 + 0] = fmaf(-xc.y, mv.y, fmaf(xc.x, mv.x, acc[0][4 * q2 + 0]));
            acc[0][4 * q2 + 1] = fmaf(xc.y, mv.x, fmaf(xc.x, mv.y, acc[0][4 * q2 + 1]));
            acc[0][4 * q2 + 2] = fmaf(-xc.y, mv.w, fmaf(xc.x, mv.z, acc[0][4 * q2 + 2]));
            acc[0][4 * q2 + 3] = fmaf(xc.y, mv.z, fmaf(xc.x, mv.w, acc[0][4 * q2 + 3]));
          }
          continue;
        }
        float x[kPer];
        if constexpr (sizeof(T) == 1) {
          const unsigned short v = *reinterpret_cast<const unsigned short*>(cur + s * kRowBytes + 2 * threadIdx.x);
          x[0] = (float)(v & 0xffu);
          x[1] = (float)(v >> 8);
        } else {
          x[0] = *reinterpret_cast<const float*>(cur + s * kRowBytes + 4 * threadIdx.x);
        }
        if constexpr (kReal) {
          const float2* mrow = reinterpret_cast<const float2*>(Ms + (a0 + s) * kW);
#pragma unroll
          for (int q2 = 0; q2 < KT / 2; ++q2) {
            const float2 mv = mrow[q2];
#pragma unroll
            for (int u = 0; u < kPer; ++u) {
              acc[u][2 * q2 + 0] = fmaf(x[u], mv.x, acc[u][2 * q2 + 0]);
              acc[u][2 * q2 + 1] = fmaf(x[u], mv.y, acc[u][2 * q2 + 1]);
            }
          }
        } else {
          const float4* mrow = reinterpret_cast<const float4*>(Ms + (a0 + s) * kW);
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
      }
      __syncthreads();   // `cur` may be overwritten by the next stage
    }
    // write: mode k, positions i0 + kPer*tid + u (complex64, or FP32 when real)
    const int64_t ibase = i0 + (int64_t)kPer * threadIdx.x;
#pragma unroll
    for (int q = 0; q < KT; ++q) {
      if (q < kt) {
        if constexpr (kReal) {
          float* col = a.phi + (int64_t)(k0 + q) * a.n;
#pragma unroll
          for (int u = 0; u < kPer; ++u)
            if (ibase + u < a.n) col[ibase + u] = acc[u][q];
        } else {
          float2* col = reinterpret_cast<float2*>(a.phi) + (int64_t)(k0 + q) * a.n;
#pragma unroll
          for (int u = 0; u < kPer; ++u)
            if (ibase + u < a.n) col[ibase + u] = make_float2(acc[u][2 * q], acc[u][2 * q + 1]);
        }
      }
    }
  }
}

template <typename T, int KT, bool kReal>
cudaError_t launch_t(const PhiArgs& a, cudaStream_t st, int sms) {
  constexpr int kPos = PhiTraits<T>::kPos;
  constexpr int kSlots = PhiTraits<T>::kSlots;
  const size_t smem = 2 * kSlots * kPos * sizeof(T) + (size_t)a.p * (kReal ? KT : 2 * KT) * sizeof(float);
  {
    const cudaError_t e = smem_optin(reinterpret_cast<const void*>(phi_tile_kernel<T, KT, kReal>), smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t ntiles = (a.n + kPos - 1) / kPos;
  const int ky = (a.r + KT - 1) / KT;
  int64_t bx = (int64_t)2 * sms;                // persistent: two CTAs per SM over all mode tiles
  bx = (bx + ky - 1) / ky;
  if (bx < 1) bx = 1;
  if (bx > ntiles) bx = ntiles;
  dim3 grid((unsigned)bx, (unsigned)ky);
  phi_tile_kernel<T, KT, kReal><<<grid, kPhiThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T, bool kReal>
cudaError_t launch_for_type(const PhiArgs& a, cudaStream_t st, int sms) {
  // modes per pass: the smallest even tile >= r, at most 16
  const int kt = a.r >= 16 ? 16 : ((a.r + 1) / 2) * 2;
  switch (kt) {
    case 2: return launch_t<T, 2, kReal>(a, st, sms);
    case 4: return launch_t<T, 4, kReal>(a, st, sms);
    case 6: return launch_t<T, 6, kReal>(a, st, sms);
    case 8: return launch_t<T, 8, kReal>(a, st, sms);
    case 10: return launch_t<T, 10, kReal>(a, st, sms);
    case 12: return launch_t<T, 12, kReal>(a, st, sms);
    case 14: return launch_t<T, 14, kReal>(a, st, sms);
    default: return launch_t<T, 16, kReal>(a, st, sms);
  }
}

// Mu[j][k] = V[k][j] / sigma_k for the kept modes, zero beyond (V vector k
// at V + k * p, FP64, from the eigensolver)
__global__ void pod_weights_kernel(const double* V, const double* sig, const int* r_dev, int p, int r, float* Mu) {
  const int re = *r_dev;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < p * r; idx += gridDim.x * blockDim.x) {
    const int j = idx / r, k = idx - j * r;
    const double s = sig[k];
    Mu[idx] = (k < re && s > 0.0) ? (float)(V[(int64_t)k * p + j] / s) : 0.f;
  }
}

}  // namespace

cudaError_t launch_phi(const PhiArgs& a, cudaStream_t st) {
  if (a.tensor && a.dtype == SDMD_U8 && !a.real_out && a.xoff == 1) {
    const cudaError_t e = launch_phi_tc(a, st);
    if (e != cudaErrorNotSupported) return e;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (a.real_out) {
    if (a.dtype == SDMD_U8) return launch_for_type<uint8_t, true>(a, st, sms > 0 ? sms : 1);
    return launch_for_type<float, true>(a, st, sms > 0 ? sms : 1);
  }
  if (a.dtype == SDMD_U8) return launch_for_type<uint8_t, false>(a, st, sms > 0 ? sms : 1);
  if (a.dtype == SDMD_C64) return launch_for_type<float2, false>(a, st, sms > 0 ? sms : 1);
  return launch_for_type<float, false>(a, st, sms > 0 ? sms : 1);
}

cudaError_t launch_pod_modes(const PhiArgs& a, const double* V, const double* sig, float* Mu, cudaStream_t st) {
  const int total = a.p * a.r;
  pod_weights_kernel<<<(total + 255) / 256, 256, 0, st>>>(V, sig, a.r_dev, a.p, a.r, Mu);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  PhiArgs b = a;
  b.Mf = Mu;
  b.xoff = 0;
  b.real_out = 1;
  b.tensor = 0;
  return launch_phi(b, st);
}

}  // namespace sdmd
