// Exact DMD modes Phi = X' (V Sigma^-1 W) (Sec. 2.2, Eq. 9; Algorithm 2's
// phi = X[:, 1:] * vsiw). X' is read in place from the ring buffer (logical
// columns 1..c-1 of the window); M = V Sigma^-1 W is the small p x r complex
// matrix produced by the FP64 kernel, rounded to FP32 here.
//
// Each thread owns 4 consecutive positions and a tile of up to kModeTile
// modes: it walks the p slots of X' (4 loads in flight), accumulating
// 2 * kModeTile FP32 partial sums per position against M broadcast from
// shared memory, and writes complex64 outputs (column-major n x r).
// Columns beyond the kept rank have M = 0 and come out as zeros.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sdmd_internal.cuh"

namespace sdmd {

namespace {

constexpr int kPhiThreads = 256;
constexpr int kModeTile = 8;

template <typename T>
__device__ __forceinline__ void load4(const uint8_t* base, int64_t i0, float (&x)[4]);

template <>
__device__ __forceinline__ void load4<uint8_t>(const uint8_t* base, int64_t i0, float (&x)[4]) {
  const unsigned int v = __ldcs(reinterpret_cast<const unsigned int*>(base + i0));
  x[0] = (float)(v & 0xffu);
  x[1] = (float)((v >> 8) & 0xffu);
  x[2] = (float)((v >> 16) & 0xffu);
  x[3] = (float)(v >> 24);
}

template <>
__device__ __forceinline__ void load4<float>(const uint8_t* base, int64_t i0, float (&x)[4]) {
  const float4 v = __ldcs(reinterpret_cast<const float4*>(base + 4 * i0));
  x[0] = v.x;
  x[1] = v.y;
  x[2] = v.z;
  x[3] = v.w;
}

template <typename T>
__global__ void __launch_bounds__(kPhiThreads) phi_simt_kernel(PhiArgs a) {
  extern __shared__ float Ms[];                 // p x (2 * kModeTile)
  const int k0 = blockIdx.y * kModeTile;
  const int kt = min(kModeTile, a.r - k0);
  for (int idx = threadIdx.x; idx < a.p * 2 * kModeTile; idx += blockDim.x) {
    const int row = idx / (2 * kModeTile), q = idx - row * (2 * kModeTile);
    Ms[idx] = (q < 2 * kt) ? a.Mf[(int64_t)row * 2 * a.r + 2 * k0 + q] : 0.f;
  }
  __syncthreads();
  const int64_t nq = (a.n + 3) / 4;
  for (int64_t qd = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; qd < nq;
       qd += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = 4 * qd;
    float acc[4][2 * kModeTile];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int q = 0; q < 2 * kModeTile; ++q) acc[u][q] = 0.f;
    int a0 = 0;
    for (; a0 + 4 <= a.p; a0 += 4) {
      float x[4][4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int slot = (a.start + 1 + a0 + s) % a.m;
        load4<T>(a.ring + (int64_t)slot * a.slot_bytes, i0, x[s]);
      }
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const float* mrow = Ms + (a0 + s) * 2 * kModeTile;
#pragma unroll
        for (int q = 0; q < 2 * kModeTile; ++q) {
          const float mv = mrow[q];
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[u][q] = fmaf(x[s][u], mv, acc[u][q]);
        }
      }
    }
    for (; a0 < a.p; ++a0) {
      float x[4];
      const int slot = (a.start + 1 + a0) % a.m;
      load4<T>(a.ring + (int64_t)slot * a.slot_bytes, i0, x);
      const float* mrow = Ms + a0 * 2 * kModeTile;
#pragma unroll
      for (int q = 0; q < 2 * kModeTile; ++q) {
        const float mv = mrow[q];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u][q] = fmaf(x[u], mv, acc[u][q]);
      }
    }
    float2* out = reinterpret_cast<float2*>(a.phi);
#pragma unroll
    for (int q = 0; q < kModeTile; ++q) {
      if (q < kt) {
        float2* col = out + (int64_t)(k0 + q) * a.n;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (i0 + u < a.n) col[i0 + u] = make_float2(acc[u][2 * q], acc[u][2 * q + 1]);
      }
    }
  }
}

}  // namespace

cudaError_t launch_phi(const PhiArgs& a, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t nq = (a.n + 3) / 4;
  int64_t bx = (nq + kPhiThreads - 1) / kPhiThreads;
  const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 8;
  if (bx > cap) bx = cap;
  dim3 grid((unsigned)bx, (unsigned)((a.r + kModeTile - 1) / kModeTile));
  const size_t smem = (size_t)a.p * 2 * kModeTile * sizeof(float);
  if (a.dtype == SDMD_U8)
    phi_simt_kernel<uint8_t><<<grid, kPhiThreads, smem, st>>>(a);
  else
    phi_simt_kernel<float><<<grid, kPhiThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sdmd
