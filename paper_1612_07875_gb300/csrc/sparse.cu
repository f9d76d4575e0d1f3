// Gram row of Fourier-sparse snapshots (Sec. 3.5): SVD and DMD are invariant
// under unitary transforms such as an orthonormal FFT, so the Gram entries of
// the physical fields equal the inner products of their transform
// coefficients (Parseval), and snapshots that are sparse in that basis give
// sparse inner products g_j = sum_{k in S_j and S_new} conj(a_j[k]) b[k].
//
// Per push, two kernels:
//  1. scatter: every coefficient (k, b_k) of the new snapshot goes into a
//     dense lookup table of length n: val[k] = b_k, tag[k] = stamp, where the
//     stamp is unique to this push, so the table is never cleared and a
//     position belongs to the new snapshot exactly when its tag matches.
//  2. row: CTAs cover (slot, 2048-entry chunk) pairs of the resident slots'
//     coefficient lists; each entry of slot j looks its index up in the table
//     (sparse x dense gather, L2-resident for n up to a few million) and
//     accumulates conj(a) b; products in FP32, per-thread sums in FP32 over
//     at most 8 terms, CTA and cross-CTA sums in FP64 in a fixed order; the
//     last CTA (atomic ticket, no waiting) writes row/column s_new of the
//     Hermitian G.
// Indices outside [0, n) are skipped and raise kDevRange in the status word.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sdmd_internal.cuh"

namespace sdmd {

namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 2048;

__global__ void sparse_scatter_kernel(const int* idx, const float2* val, int nnz, int64_t n, int stamp,
                                      int* tag, float2* tval, int* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nnz) return;
  const int k = idx[i];
  if (k < 0 || (int64_t)k >= n) {
    atomicOr(status, kDevRange);
    return;
  }
  tval[k] = val[i];
  tag[k] = stamp;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kThreads) sparse_row_kernel(SparseRowArgs a) {
  __shared__ double red[2][kThreads / 32];
  __shared__ bool last;
  // CTA -> (window slot jj, chunk q) by the prefix table of chunk counts
  int jj = 0;
  while (jj + 1 < a.c && a.chunk_start[jj + 1] <= (int)blockIdx.x) ++jj;
  const int q = blockIdx.x - a.chunk_start[jj];
  const int slot = (a.s_first + jj) % a.m;
  const int nnz = a.nnz[slot];
  const int* idx = a.idx_ring + (int64_t)slot * a.nnz_max;
  const float2* val = a.val_ring + (int64_t)slot * a.nnz_max;
  const int e0 = q * kChunk, e1 = min(nnz, e0 + kChunk);
  float sr = 0.f, si = 0.f;
  for (int e = e0 + threadIdx.x; e < e1; e += kThreads) {
    const int k = __ldg(idx + e);
    if (k < 0 || (int64_t)k >= a.n) continue;
    if (__ldcg(a.tag + k) != a.stamp) continue;
    const float2 x = __ldg(val + e);
    const float2 y = __ldcg(a.tval + k);
    sr = fmaf(x.x, y.x, fmaf(x.y, y.y, sr));     // conj(x) * y
    si = fmaf(x.x, y.y, fmaf(-x.y, y.x, si));
  }
  double dr = warp_sum((double)sr), di = warp_sum((double)si);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[0][warp] = dr;
    red[1][warp] = di;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0, ti = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) {
      tr += red[0][w];
      ti += red[1][w];
    }
    a.partials[blockIdx.x] = make_double2(tr, ti);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(a.ticket, 1u) == (unsigned int)a.nblk - 1u);
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int j2 = warp; j2 < a.c; j2 += kThreads / 32) {
    const int b0 = a.chunk_start[j2], b1 = (j2 + 1 < a.c) ? a.chunk_start[j2 + 1] : a.nblk;
    double tr = 0.0, ti = 0.0;
    for (int b = b0 + lane; b < b1; b += 32) {
      const double2 v = __ldcg(a.partials + b);
      tr += v.x;
      ti += v.y;
    }
    tr = warp_sum(tr);
    ti = warp_sum(ti);
    if (lane == 0) {
      const int s2 = (a.s_first + j2) % a.m;
      if (s2 == a.s_new) ti = 0.0;  // <x, x> is real; drop the rounding residue
      double2* G = static_cast<double2*>(a.G);
      G[(int64_t)s2 * a.m + a.s_new] = make_double2(tr, ti);
      G[(int64_t)a.s_new * a.m + s2] = make_double2(tr, -ti);
    }
  }
  if (threadIdx.x == 0) *a.ticket = 0u;
}


// --------------------------------------------- modes in coefficient space --
// Phi-hat = X'-hat M (Eq. 9 with the snapshots in Fourier coefficient space,
// Sec. 3.5): column j of X'-hat is sparse, so Phi-hat is nonzero only on the
// union of the X' supports. The union is marked in a bitmap, counted with an
// exclusive popcount prefix and compacted (sorted coefficient indices); each
// union coefficient then gathers its value from every X' slot by binary
// search in the slot's sorted index list and accumulates the r mode values.

__global__ void fphi_mark_kernel(FourierPhiArgs a) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = (int)(t / a.nnz_max), e = (int)(t - (int64_t)j * a.nnz_max);
  if (j >= a.p) return;
  const int slot = (a.start + 1 + j) % a.m;
  if (e >= a.nnz[slot]) return;
  const int k = a.idx_ring[(int64_t)slot * a.nnz_max + e];
  if (k < 0 || (int64_t)k >= a.n) return;             // rejected at push (status word)
  atomicOr(a.bitmap + (k >> 5), 1u << (k & 31));
}

constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads) fphi_scan_kernel(FourierPhiArgs a) {
  __shared__ unsigned long long part[kScanThreads];
  const int64_t nw = (a.n + 31) / 32;
  const int64_t per = (nw + kScanThreads - 1) / kScanThreads;
  const int64_t w0 = (int64_t)threadIdx.x * per, w1 = (w0 + per < nw) ? w0 + per : nw;
  unsigned long long s = 0;
  for (int64_t w = w0; w < w1; ++w) s += (unsigned)__popc(a.bitmap[w]);
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < kScanThreads; o <<= 1) {      // inclusive scan of the thread sums
    const unsigned long long v = (threadIdx.x >= (unsigned)o) ? part[threadIdx.x - o] : 0ull;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned long long run = (threadIdx.x > 0) ? part[threadIdx.x - 1] : 0ull;
  for (int64_t w = w0; w < w1; ++w) {
    a.prefix[w] = run;
    run += (unsigned)__popc(a.bitmap[w]);
  }
  if (threadIdx.x == kScanThreads - 1) *a.count = part[kScanThreads - 1];
}

__global__ void fphi_compact_kernel(FourierPhiArgs a) {
  const int64_t nw = (a.n + 31) / 32;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x) {
    unsigned bits = a.bitmap[w];
    unsigned long long pos = a.prefix[w];
    while (bits) {
      const int b = __ffs(bits) - 1;
      if (pos < (unsigned long long)a.cap) a.idx_out[pos] = (int)(w * 32 + b);
      ++pos;
      bits &= bits - 1u;
    }
  }
}

constexpr int kFModes = 16;   // modes per thread (grid.y tiles the modes)

__global__ void __launch_bounds__(256) fphi_rows_kernel(FourierPhiArgs a) {
  __shared__ float2 Ms[SDMD_MAX_M * kFModes];
  const int k0 = blockIdx.y * kFModes;
  const int kt = (a.r - k0 < kFModes) ? a.r - k0 : kFModes;
  for (int idx = threadIdx.x; idx < a.p * kFModes; idx += blockDim.x) {
    const int j = idx / kFModes, q = idx - j * kFModes;
    Ms[idx] = (q < kt) ? make_float2(a.Mf[(int64_t)j * 2 * a.R + 2 * (k0 + q)], a.Mf[(int64_t)j * 2 * a.R + 2 * (k0 + q) + 1])
                       : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const unsigned long long total = *a.count;
  const int64_t lim = (total < (unsigned long long)a.cap) ? (int64_t)total : a.cap;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < lim; u += (int64_t)gridDim.x * blockDim.x) {
    const int k = a.idx_out[u];
    float2 acc[kFModes];
#pragma unroll
    for (int q = 0; q < kFModes; ++q) acc[q] = make_float2(0.f, 0.f);
    for (int j = 0; j < a.p; ++j) {
      const int slot = (a.start + 1 + j) % a.m;
      const int* list = a.idx_ring + (int64_t)slot * a.nnz_max;
      int lo = 0, hi = a.nnz[slot];                    // first entry >= k
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(list + mid) < k) lo = mid + 1;
        else hi = mid;
      }
      if (lo < a.nnz[slot] && __ldg(list + lo) == k) {
        const float2 v = __ldg(a.val_ring + (int64_t)slot * a.nnz_max + lo);
        const float2* mr = Ms + j * kFModes;
#pragma unroll
        for (int q = 0; q < kFModes; ++q) {
          acc[q].x = fmaf(v.x, mr[q].x, fmaf(-v.y, mr[q].y, acc[q].x));
          acc[q].y = fmaf(v.x, mr[q].y, fmaf(v.y, mr[q].x, acc[q].y));
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kFModes; ++q)
      if (q < kt) a.phi_out[(int64_t)(k0 + q) * a.cap + u] = acc[q];
  }
}

}  // namespace

int sparse_chunks(int nnz) { return nnz > 0 ? (nnz + kChunk - 1) / kChunk : 1; }

cudaError_t launch_sparse_scatter(const int* idx, const float2* val, int nnz, int64_t n, int stamp, int* tag,
                                  float2* tval, int* status, cudaStream_t st) {
  if (nnz <= 0) return cudaSuccess;
  sparse_scatter_kernel<<<(nnz + kThreads - 1) / kThreads, kThreads, 0, st>>>(idx, val, nnz, n, stamp, tag, tval,
                                                                               status);
  return cudaGetLastError();
}

cudaError_t launch_sparse_row(const SparseRowArgs& a, cudaStream_t st) {
  sparse_row_kernel<<<a.nblk, kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fourier_phi(const FourierPhiArgs& a, bool rows, cudaStream_t st) {
  if (a.p < 1 || a.p > SDMD_MAX_M - 1) return cudaErrorNotSupported;
  const int64_t nw = (a.n + 31) / 32;
  cudaError_t e = cudaMemsetAsync(a.bitmap, 0, (size_t)nw * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  const int64_t marks = (int64_t)a.p * a.nnz_max;
  fphi_mark_kernel<<<(unsigned)((marks + 255) / 256), 256, 0, st>>>(a);
  fphi_scan_kernel<<<1, kScanThreads, 0, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess || !rows) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms < 1) sms = 1;
  int64_t cb = (nw + 255) / 256;
  if (cb > (int64_t)sms * 8) cb = (int64_t)sms * 8;
  fphi_compact_kernel<<<(unsigned)(cb > 0 ? cb : 1), 256, 0, st>>>(a);
  int64_t rb = (a.cap + 255) / 256;
  if (rb > (int64_t)sms * 8) rb = (int64_t)sms * 8;
  dim3 grid((unsigned)(rb > 0 ? rb : 1), (unsigned)((a.r + kFModes - 1) / kFModes));
  fphi_rows_kernel<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sdmd
