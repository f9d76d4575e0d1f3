// Reconstruction from the exact DMD of the window (Sec. 2.2 and Sec. 3.3,
// Eq. 11; Algorithm 3): x_hat(t) = sum_k b_k phi_k lambda_k^t over a set of
// modes, t = 0 for x_1 (the oldest snapshot of X).
//
// Phi = X' M with M = V Sigma^-1 W (Eq. 9) and the window snapshots are real,
// so x_hat(t) = X' Re(M c) with c_k = b_k lambda_k^t: one p-vector of real
// weights u = Re(M c) and one pass over X' (a GEMV), without forming Phi.
//  - weights kernel (one CTA): c_k in FP64 for the selected modes (all kept
//    modes, or the background mode argmin |log lambda|), u in FP64, stored as
//    two floats hi + lo so that the pass below carries ~48 bits of u;
//  - pass kernel: each thread owns 16 consecutive uint8 positions (or 4
//    float32), loops over the p slots of X' (a CTA reads 4 KiB contiguous per
//    slot per step; 8 slots' loads in flight per thread), accumulates
//    x * hi + x * lo in FP32 and writes x_hat, or x_t - x_hat (foreground:
//    the snapshot minus its background).
#include <cuda_runtime.h>
#include <stdint.h>

#include "sdmd_internal.cuh"

namespace sdmd {

namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) recon_weights_kernel(ReconArgs a) {
  __shared__ double cre[SDMD_MAX_M], cim[SDMD_MAX_M];
  const int re = *a.r_dev;
  const int bg = (int)*a.bgi;
  for (int k = threadIdx.x; k < a.R; k += kThreads) {
    double cr = 0.0, ci = 0.0;
    const double lr = a.lamout[2 * k], li = a.lamout[2 * k + 1];
    bool use = k < re;
    if (a.what == SDMD_RECON_BACKGROUND || a.what == SDMD_RECON_FOREGROUND) {
      use = use && k == bg;
    } else if (a.what == SDMD_RECON_BACKGROUND_SLOW || a.what == SDMD_RECON_FOREGROUND_SLOW) {
      const double m2 = lr * lr + li * li;    // |log lambda| with the principal log
      const double lg = (m2 > 0.0) ? 0.5 * log(m2) : -INFINITY;
      use = use && m2 > 0.0 && sqrt(lg * lg + atan2(li, lr) * atan2(li, lr)) <= a.slow_tol;
    }
    if (use) {
      double pr = 1.0, pi = 0.0;            // lambda^t (lambda^0 = 1)
      if (a.t != 0) {
        const double m2 = lr * lr + li * li;
        if (m2 > 0.0) {
          const double mag = exp((double)a.t * 0.5 * log(m2)), ang = (double)a.t * atan2(li, lr);
          pr = mag * cos(ang);
          pi = mag * sin(ang);
        } else {
          pr = 0.0;
        }
      }
      const double br = a.bamp[2 * k], bi = a.bamp[2 * k + 1];
      cr = br * pr - bi * pi;
      ci = br * pi + bi * pr;
    }
    cre[k] = cr;
    cim[k] = ci;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < a.p; q += kThreads) {
    double u = 0.0;
    const float* mrow = a.Mf + (int64_t)q * 2 * a.R;
    for (int k = 0; k < a.R; ++k) u += (double)mrow[2 * k] * cre[k] - (double)mrow[2 * k + 1] * cim[k];
    const float hi = (float)u;
    a.urec[2 * q] = hi;
    a.urec[2 * q + 1] = (float)(u - (double)hi);
  }
}

__device__ __forceinline__ void to_floats(const uint4& w, float (&x)[16]) {
  const unsigned v[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int b = 0; b < 4; ++b)   // 0x4B0000bb = 2^23 + byte, exact
      x[4 * i + b] = __uint_as_float(__byte_perm(v[i], 0x4B000000u, 0x7650u | (unsigned)b)) - 8388608.f;
}
__device__ __forceinline__ void to_floats(const float4& w, float (&x)[4]) {
  x[0] = w.x;
  x[1] = w.y;
  x[2] = w.z;
  x[3] = w.w;
}

template <typename T>
struct ReconVec;
template <>
struct ReconVec<uint8_t> {
  using V = uint4;
  static constexpr int kN = 16;
};
template <>
struct ReconVec<float> {
  using V = float4;
  static constexpr int kN = 4;
};

template <typename T>
__global__ void __launch_bounds__(kThreads, 3) recon_pass_kernel(ReconArgs a) {
  using V = typename ReconVec<T>::V;
  constexpr int kN = ReconVec<T>::kN;
  __shared__ float uh[SDMD_MAX_M], ul[SDMD_MAX_M];
  __shared__ int64_t off[SDMD_MAX_M];
  for (int q = threadIdx.x; q < a.p; q += kThreads) {
    uh[q] = a.urec[2 * q];
    ul[q] = a.urec[2 * q + 1];
    off[q] = (int64_t)((a.start + 1 + q) % a.m) * a.slot_bytes;
  }
  __syncthreads();
  const int64_t nvec = (a.n + kN - 1) / kN;
  for (int64_t v = (int64_t)blockIdx.x * kThreads + threadIdx.x; v < nvec; v += (int64_t)gridDim.x * kThreads) {
    const int64_t byte = v * kN * (int64_t)sizeof(T);   // in bounds: slots are padded to 4 KiB
    float y[kN];
#pragma unroll
    for (int i = 0; i < kN; ++i) y[i] = 0.f;
#pragma unroll 8
    for (int q = 0; q < a.p; ++q) {
      const V w = __ldcs(reinterpret_cast<const V*>(a.ring + off[q] + byte));
      float x[kN];
      to_floats(w, x);
      const float h = uh[q], l = ul[q];
#pragma unroll
      for (int i = 0; i < kN; ++i) y[i] = fmaf(x[i], l, fmaf(x[i], h, y[i]));
    }
    if (a.xt_slot >= 0) {        // foreground: x_t - background
      const V w = *reinterpret_cast<const V*>(a.ring + (int64_t)a.xt_slot * a.slot_bytes + byte);
      float x[kN];
      to_floats(w, x);
#pragma unroll
      for (int i = 0; i < kN; ++i) y[i] = x[i] - y[i];
    }
    const int64_t i0 = v * kN;
    if (i0 + kN <= a.n) {
#pragma unroll
      for (int i = 0; i < kN; i += 4)
        *reinterpret_cast<float4*>(a.out + i0 + i) = make_float4(y[i], y[i + 1], y[i + 2], y[i + 3]);
    } else {
#pragma unroll
      for (int i = 0; i < kN; ++i)
        if (i0 + i < a.n) a.out[i0 + i] = y[i];
    }
  }
}

}  // namespace

cudaError_t launch_reconstruct(const ReconArgs& a, cudaStream_t st) {
  recon_weights_kernel<<<1, kThreads, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms < 1) sms = 1;
  const int vec = (a.dtype == SDMD_U8) ? 16 : 4;
  const int64_t nvec = (a.n + vec - 1) / vec;
  int64_t blocks = (nvec + kThreads - 1) / kThreads;
  if (blocks > (int64_t)sms * 12) blocks = (int64_t)sms * 12;
  if (blocks < 1) blocks = 1;
  if (a.dtype == SDMD_U8)
    recon_pass_kernel<uint8_t><<<(unsigned)blocks, kThreads, 0, st>>>(a);
  else
    recon_pass_kernel<float><<<(unsigned)blocks, kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sdmd
