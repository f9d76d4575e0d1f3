// The multi-column catch-up of FP32 windows for a few new snapshots (Sec. 3.1,
// Eq. 12a-b for k new columns at once; the paper's future-work multi-column
// update): G[i][t] = <x_i, x_t> for the k <= 16 newest snapshots t against all
// c <= 256 window snapshots i, in one pass over the window.
//
// Why CUDA cores. Per window element the pass does k multiply-adds (8 for the
// usual catch-up of 8 frames) against 4 bytes read: 2 FMA per byte, about 14
// TFMA/s at the copy bandwidth, a fraction of the FP32 rate. The work is
// bound by the window's reads, not by arithmetic, so it stays a plain
// tall-skinny product on the FP32 pipes; the tensor-core BF16x3 pass
// (gram_f32_tc.cu) is kept for larger k and for the full rebuild.
//
// Precision: FP32 products, accumulated in FP32 over runs of 64 positions per
// (row, target), each run added to a compensated (hi, lo) pair with an
// error-free two-sum; the per-CTA pairs are added in FP64 in CTA order. The
// error is that of the BF16x3 pass or below: |G_ij - <x_i, x_j>| <= 1e-6
// sum_p |x_ip x_jp|. Chunks go to CTAs statically (chunk b, b + grid, ...),
// so the result is the same on every run.
//
// Layout. A CTA of 256 threads takes 64-position chunks b, b + grid, ... (at
// any moment the CTAs read neighbouring pieces of every row, which HBM sees
// as one stream per row); a chunk of every window row (256 bytes, in time
// order) is copied with cp.async into one of three stages (rows padded to 272
// bytes: a warp's 16-byte reads of 32 consecutive rows fall in distinct
// banks). The k targets are the last k rows of the same stage and are read
// with broadcast loads. A warp's copy instruction moves 512 contiguous bytes
// (two rows).
//
// Rows per thread. Windows of at most 128 rows: thread r owns row r over the
// whole chunk (per 4 positions one 16-byte read of its row, k broadcast reads
// of the targets, 4k FMAs). Longer windows: thread t owns rows t mod 128 and
// t mod 128 + 128 over half of the chunk (positions 32 (t / 128) ...), so each
// broadcast target read feeds two rows. A broadcast read costs a whole
// shared-memory cycle for 16 bytes, and at k = 8 and one row per thread those
// reads were two thirds of the shared-memory cycles of a chunk; two rows per
// thread cut the chunk's shared-memory cycles by a third. A run then spans two
// chunks (still 64 positions), and the two halves' pairs are added at the end.
// Measured at n = 2^22, c = 256 (fraction of the copy peak): 0.83 at k = 4,
// 0.70 at k = 8 (0.61 with one row per thread), 0.45 at k = 16 (0.40); at
// c = 128 two rows per thread over half chunks measured slower than one row
// (0.43 against 0.49 at k = 8), hence the split by window length. Also
// measured and dropped: two threads per row (each half of the targets) and
// contiguous chunk runs per CTA with L2 bulk prefetch (0.44 instead of 0.59).
// The tail chunk (n not a multiple of 64) is summed with both factors masked,
// since the ring's row padding past n holds no data.
#include <cuda_runtime.h>
#include <stdint.h>

#include "df64.cuh"
#include "sdmd_internal.cuh"
#include "tc_util.cuh"

namespace sdmd {

namespace {

using namespace tc;

constexpr int kSRows = 256;                            // window rows (at most)
constexpr int kSThreads = kSRows;                      // one window row per thread
constexpr int kSPos = 64;                              // positions per chunk (= FP32 run)
constexpr int kSStages = 3;
constexpr int kSRowFloats = kSPos + 4;                 // 272-byte rows in a stage
constexpr int kSStageFloats = kSRows * kSRowFloats;
constexpr int kSSmem = (kSStages * kSStageFloats + kSRowFloats) * 4;   // stages + a zero row: 209,168 B
constexpr int kSRowsPerPass = 2 * kSThreads / 32;      // rows copied per pass of all warps
constexpr int kSPasses = kSRows / kSRowsPerPass;       // 16

// kT: targets padded (4, 8 or 16). kR: window rows per thread. kR = 1: thread
// r owns row r over all 64 positions of a chunk. kR = 2: thread t owns rows
// t mod 128 and t mod 128 + 128 over half of the chunk's positions (t / 128),
// so each broadcast read of a target feeds two rows; the halves' pairs are
// added at the end.
template <int kT, int kR>
__global__ void __launch_bounds__(kSThreads, 1) gram_f32_simt_kernel(GramF32SimtArgs a) {
  static_assert(kR == 1 || kR == 2, "one or two rows per thread");
  constexpr int kRowStep = kSRows / kR;   // distance between a thread's rows
  constexpr int kPosT = kSPos / kR;       // positions per thread and chunk
  constexpr int kRunChunks = kR;          // chunks per FP32 run: runs of 64 positions per thread
  extern __shared__ __align__(16) float sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c = a.c, k = a.k, t0 = c - k;
  const int lr = tid % kRowStep, half = tid / kRowStep;
  // this CTA's chunks: b, b + grid, ...
  const int64_t nch = (a.n + kSPos - 1) / kSPos;
  const int64_t mine = (nch > (int64_t)blockIdx.x) ? (nch - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  // the rows this thread copies: 2 warp + (lane >> 4) + 16 q, 16-byte piece lane & 15
  const uint8_t* rowp[kSPasses];
#pragma unroll
  for (int q = 0; q < kSPasses; ++q) {
    const int r = 2 * warp + (lane >> 4) + kSRowsPerPass * q;
    rowp[q] = (r < c) ? a.ring + (int64_t)((a.start + r) % a.m) * a.slot_bytes + 16 * (lane & 15) : nullptr;
  }
  const unsigned sm0 = smem_u32(sm);
  auto issue = [&](int64_t it) {
    if (it < mine) {
      const int64_t boff = (blockIdx.x + it * (int64_t)gridDim.x) * (kSPos * 4);
      const unsigned st = sm0 + (unsigned)((it % kSStages) * kSStageFloats * 4);
#pragma unroll
      for (int q = 0; q < kSPasses; ++q) {
        const int r = 2 * warp + (lane >> 4) + kSRowsPerPass * q;
        if (r < c) cp_async16(st + (unsigned)((r * kSRowFloats + 4 * (lane & 15)) * 4), rowp[q] + boff);
      }
    }
    cp_async_commit();   // one group per chunk, empty past the end
  };

  // targets past k, and rows past c, read a zero row (no guards in the inner loop)
  float* zrow = sm + kSStages * kSStageFloats;
  for (int q = tid; q < kSRowFloats; q += kSThreads) zrow[q] = 0.f;   // visible after the loop's first barrier
  // warp-uniform: does any lane of this warp own a row (the first / the second)?
  const int wrow0 = lr - lane;
  const bool any0 = wrow0 < c, any1 = (kR == 2) && (wrow0 + kRowStep < c);
  float hi[kR][kT], lo[kR][kT], acc[kR][kT];   // acc: the current FP32 run
#pragma unroll
  for (int i = 0; i < kR; ++i)
#pragma unroll
    for (int j = 0; j < kT; ++j) hi[i][j] = lo[i][j] = acc[i][j] = 0.f;
  for (int s = 0; s < kSStages - 1; ++s) issue(s);
  for (int64_t it = 0; it < mine; ++it) {
    cp_async_wait<kSStages - 2>();   // this thread's copies of chunk `it` have landed
    __syncthreads();                 // ... everyone's; and chunk it-1 is summed (its stage is free)
    issue(it + kSStages - 1);
    const float* st = sm + (it % kSStages) * kSStageFloats;
    const int64_t p0 = (blockIdx.x + it * (int64_t)gridDim.x) * kSPos + half * kPosT;
    if (any0) {
      const float* tj[kT];
#pragma unroll
      for (int j = 0; j < kT; ++j) tj[j] = ((j < k) ? st + (t0 + j) * kSRowFloats : zrow) + half * kPosT;
      const float* wr[kR];
#pragma unroll
      for (int i = 0; i < kR; ++i) {
        const int r = lr + i * kRowStep;
        wr[i] = ((r < c) ? st + r * kSRowFloats : zrow) + half * kPosT;
      }
      if (p0 + kPosT <= a.n) {
        if (kR == 1 || !any1) {   // one row for every lane of this warp
#pragma unroll
          for (int q = 0; q < kPosT; q += 4) {
            const float4 w = *reinterpret_cast<const float4*>(wr[0] + q);
#pragma unroll
            for (int j = 0; j < kT; ++j) {
              const float4 t = *reinterpret_cast<const float4*>(tj[j] + q);
              acc[0][j] = fmaf(w.x, t.x, acc[0][j]);
              acc[0][j] = fmaf(w.y, t.y, acc[0][j]);
              acc[0][j] = fmaf(w.z, t.z, acc[0][j]);
              acc[0][j] = fmaf(w.w, t.w, acc[0][j]);
            }
          }
        } else {
#pragma unroll
          for (int q = 0; q < kPosT; q += 4) {
            const float4 w0 = *reinterpret_cast<const float4*>(wr[0] + q);
            const float4 w1 = *reinterpret_cast<const float4*>(wr[kR - 1] + q);
#pragma unroll
            for (int j = 0; j < kT; ++j) {
              const float4 t = *reinterpret_cast<const float4*>(tj[j] + q);
              acc[0][j] = fmaf(w0.x, t.x, acc[0][j]);
              acc[kR - 1][j] = fmaf(w1.x, t.x, acc[kR - 1][j]);
              acc[0][j] = fmaf(w0.y, t.y, acc[0][j]);
              acc[kR - 1][j] = fmaf(w1.y, t.y, acc[kR - 1][j]);
              acc[0][j] = fmaf(w0.z, t.z, acc[0][j]);
              acc[kR - 1][j] = fmaf(w1.z, t.z, acc[kR - 1][j]);
              acc[0][j] = fmaf(w0.w, t.w, acc[0][j]);
              acc[kR - 1][j] = fmaf(w1.w, t.w, acc[kR - 1][j]);
            }
          }
        }
      } else {   // tail chunk: positions past n hold no data (mask both factors)
        const int nv = (int)(a.n - p0);   // may be <= 0 for the second half
        for (int q = 0; q < nv; ++q) {
#pragma unroll
          for (int i = 0; i < kR; ++i) {
            const float w = wr[i][q];
#pragma unroll
            for (int j = 0; j < kT; ++j) acc[i][j] = fmaf(w, tj[j][q], acc[i][j]);
          }
        }
      }
      if ((it + 1) % kRunChunks == 0 || it + 1 == mine) {   // a run of 64 positions ends
#pragma unroll
        for (int i = 0; i < kR; ++i)
#pragma unroll
          for (int j = 0; j < kT; ++j) {   // error-free two-sum into the compensated pair
            const dd sm2 = two_sum(hi[i][j], acc[i][j]);
            hi[i][j] = sm2.hi;
            lo[i][j] += sm2.lo;
            acc[i][j] = 0.f;
          }
      }
    }
  }
  cp_async_wait<0>();
  if (kR == 2) {   // add the second half's pairs to the first half's (stage 0 is free after the barrier)
    __syncthreads();
    float2* xs = reinterpret_cast<float2*>(sm) + (int64_t)lr * (kR * kT);
    if (half == 1) {
#pragma unroll
      for (int i = 0; i < kR; ++i)
#pragma unroll
        for (int j = 0; j < kT; ++j) xs[i * kT + j] = make_float2(hi[i][j], lo[i][j]);
    }
    __syncthreads();
    if (half == 1) return;
#pragma unroll
    for (int i = 0; i < kR; ++i)
#pragma unroll
      for (int j = 0; j < kT; ++j) {
        const float2 o = xs[i * kT + j];
        const dd sm2 = two_sum(hi[i][j], o.x);
        hi[i][j] = sm2.hi;
        lo[i][j] += o.y + sm2.lo;
      }
  }
#pragma unroll
  for (int i = 0; i < kR; ++i) {
    const int r = lr + i * kRowStep;
    if (r < c) {
#pragma unroll
      for (int j = 0; j < kT; ++j)
        if (j < k) a.partials[((int64_t)blockIdx.x * kSRows + r) * kGramF32SimtMaxTargets + j] = {hi[i][j], lo[i][j]};
    }
  }
}

// G's entries from the per-CTA pairs, FP64 in CTA order: block i = window row
// i, thread j = target j; a pair of targets is written once (from the row of
// the later one), both G[i][t] and G[t][i] in physical slots.
__global__ void gram_f32_simt_finish_kernel(GramF32SimtArgs a, int ctas) {
  const int i = blockIdx.x, t0 = a.c - a.k;
  const int pi = (a.start + i) % a.m;
  for (int j = threadIdx.x; j < a.k; j += blockDim.x) {
    if (i >= t0 && t0 + j > i) continue;
    double g = 0.0;
    for (int b = 0; b < ctas; ++b) {
      const float2 v = a.partials[((int64_t)b * kSRows + i) * kGramF32SimtMaxTargets + j];
      g += (double)v.x + (double)v.y;
    }
    const int pj = (a.start + t0 + j) % a.m;
    a.G[(int64_t)pi * a.m + pj] = g;
    a.G[(int64_t)pj * a.m + pi] = g;
  }
}

}  // namespace

cudaError_t launch_gram_f32_simt(const GramF32SimtArgs& a, int num_sms, cudaStream_t st) {
  if (a.c < 1 || a.c > kSRows || a.k < 1 || a.k > kGramF32SimtMaxTargets || a.k > a.c || a.n < 1)
    return cudaErrorNotSupported;
  {
    const void* ks[] = {reinterpret_cast<const void*>(gram_f32_simt_kernel<4, 1>),
                        reinterpret_cast<const void*>(gram_f32_simt_kernel<8, 1>),
                        reinterpret_cast<const void*>(gram_f32_simt_kernel<16, 1>),
                        reinterpret_cast<const void*>(gram_f32_simt_kernel<4, 2>),
                        reinterpret_cast<const void*>(gram_f32_simt_kernel<8, 2>),
                        reinterpret_cast<const void*>(gram_f32_simt_kernel<16, 2>)};
    for (const void* f : ks) {
      const cudaError_t e = smem_optin(f, kSSmem);
      if (e != cudaSuccess) return e;
    }
  }
  const int64_t nch = (a.n + kSPos - 1) / kSPos;
  int64_t ctas = (num_sms < kGramF32MaxCtas) ? num_sms : kGramF32MaxCtas;
  if (ctas > nch) ctas = nch;
  if (ctas < 1) ctas = 1;
  const dim3 grid((unsigned)ctas);
  // two rows per thread once the window has more rows than half the threads
  if (a.c > kSRows / 2) {
    if (a.k <= 4)
      gram_f32_simt_kernel<4, 2><<<grid, kSThreads, kSSmem, st>>>(a);
    else if (a.k <= 8)
      gram_f32_simt_kernel<8, 2><<<grid, kSThreads, kSSmem, st>>>(a);
    else
      gram_f32_simt_kernel<16, 2><<<grid, kSThreads, kSSmem, st>>>(a);
  } else {
    if (a.k <= 4)
      gram_f32_simt_kernel<4, 1><<<grid, kSThreads, kSSmem, st>>>(a);
    else if (a.k <= 8)
      gram_f32_simt_kernel<8, 1><<<grid, kSThreads, kSSmem, st>>>(a);
    else
      gram_f32_simt_kernel<16, 1><<<grid, kSThreads, kSSmem, st>>>(a);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  gram_f32_simt_finish_kernel<<<a.c, 32, 0, st>>>(a, (int)ctas);
  return cudaGetLastError();
}

}  // namespace sdmd
