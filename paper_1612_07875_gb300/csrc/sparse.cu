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

}  // namespace sdmd
