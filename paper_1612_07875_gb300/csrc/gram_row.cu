// Streaming Gram row: the one new row/column of G = X^H X per pushed snapshot
// (Sec. 3.1, Eq. 12b; Algorithm 1, the X^T X[:, -1] product). Every resident
// snapshot x_j is dotted with the new snapshot x_new; O(n m) work that reads
// each window byte exactly once, so the kernel is HBM-bound.
//
// Decomposition: the n dimension (bytes, padded to whole 4 KiB units) is cut
// into `nblk` contiguous chunks, about two per SM. One persistent CTA per SM
// takes chunks from a counter (atomicAdd), so a launch is not held back by
// SMs that another stream's kernel occupies, and walks each chunk in
// sub-chunks of up to 32 KiB: thread 0 brings the sub-chunk of x_new into
// shared memory with one bulk copy (TMA, cp.async.bulk), then each of the 8
// warps streams its slots (warp w takes slots w, w+8, ...) in 4 KiB pieces
// through its own 4-stage shared-memory ring: lane 0 issues cp.async.bulk
// copies that complete on one mbarrier per stage, the lanes wait on the
// barrier, consume the piece (16 bytes per lane per step) and hand the stage
// back. That keeps 128 KiB of loads in flight per SM without register
// pressure. Each slot's sub-chunk sum is reduced with warp shuffles into a
// per-chunk accumulator; the per-chunk partials go to a [slot][chunk] array
// and the last CTA to finish (atomic ticket, no waiting) sums them in a
// fixed order and writes row and column `s_new` of G, so the result does not
// depend on which CTA took which chunk.
//
//  - uint8: __dp4a (4 u8 x u8 products into u32). A lane sums at most
//    32 KiB / 32 = 1024 products (< 2^32 / 255^2) before the value goes to
//    int64, so the result is exact and independent of order.
//  - float32: four FP32 FMA chains of 8 products per piece per lane, then the
//    piece's sum is added in FP64; cross-lane and cross-CTA sums are FP64 in a
//    fixed order, so results are deterministic for a given schedule.
//  - complex64: the same with conj(x_j) x_new split into real and imaginary
//    FP32 chains; G is Hermitian (complex128).
//
// Every mbarrier wait is bounded (about one second of SM clock); on expiry
// the kernel raises kDevTimeout in the handle's status word, stops issuing
// copies, waits (bounded) for the copies it has in flight, and finishes.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sdmd_internal.cuh"

namespace sdmd {

namespace {

constexpr int kStages = 4;
constexpr int kPiece = 4096;                       // bytes per bulk copy
constexpr int kXSub = 24576;                       // largest chunk (x_new bytes staged per chunk)
constexpr long long kWaitCycles = 2000000000LL;    // ~1 s at 2 GHz

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

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on phase `parity` of barrier `bar`; false on expiry.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

struct Smem {
  uint8_t stage[kGrWarps][kStages][kPiece];   // per-warp piece rings
  uint8_t xs[2][kXSub];                       // x_new pieces of the current and the next chunk
  unsigned long long bar[kGrWarps][kStages];  // one mbarrier per stage
  unsigned long long xbar[2];                 // x_new barriers
  int cq[2];                                  // chunk index of chunk ordinal k at [k & 1]
  int fail;                                   // a wait expired in some warp
  long long acc_i[SDMD_MAX_M];
  double acc_d[SDMD_MAX_M];
  double acc_im[SDMD_MAX_M];                  // imaginary parts (complex snapshots)
  int last;
};

// Element modes of the kernel.
// kModeF64: FP32 snapshots with FP64 products and sums (the reference Gram;
// a product of two FP32 values is exact in FP64).
enum { kModeU8 = 0, kModeF32 = 1, kModeC64 = 2, kModeF64 = 3 };

template <typename Acc>
__device__ void finish_row(const GramRowArgs& a, Smem& sm) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int t = atomicAdd(a.ticket, 1u);
    sm.last = (t == gridDim.x - 1u);
  }
  __syncthreads();
  if (!sm.last) return;
  __threadfence();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Acc* P = static_cast<const Acc*>(a.partials);
  Acc* G = static_cast<Acc*>(a.G);
  for (int jj = warp; jj < a.c; jj += kGrWarps) {
    Acc s = 0;
    for (int b = lane; b < a.nblk; b += 32) s += __ldcg(P + (int64_t)jj * a.nblk + b);
    s = warp_sum(s);
    if (lane == 0) {
      const int j = (a.s_first + jj) % a.m;
      G[(int64_t)a.s_new * a.m + j] = s;
      G[(int64_t)j * a.m + a.s_new] = s;
    }
  }
  if (threadIdx.x == 0) {                // ready for the next launch
    a.ticket[0] = 0u;
    a.ticket[1] = 0u;
  }
}

// Complex version: G[j][s_new] = <x_j, x_new> = g_j and G[s_new][j] = conj(g_j).
__device__ void finish_row_c64(const GramRowArgs& a, Smem& sm) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int t = atomicAdd(a.ticket, 1u);
    sm.last = (t == gridDim.x - 1u);
  }
  __syncthreads();
  if (!sm.last) return;
  __threadfence();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double2* P = static_cast<const double2*>(a.partials);
  double2* G = static_cast<double2*>(a.G);
  for (int jj = warp; jj < a.c; jj += kGrWarps) {
    double sr = 0.0, si = 0.0;
    for (int b = lane; b < a.nblk; b += 32) {
      const double2 v = __ldcg(P + (int64_t)jj * a.nblk + b);
      sr += v.x;
      si += v.y;
    }
    sr = warp_sum(sr);
    si = warp_sum(si);
    if (lane == 0) {
      const int j = (a.s_first + jj) % a.m;
      if (j == a.s_new) si = 0.0;   // <x, x> is real; drop the rounding residue
      G[(int64_t)j * a.m + a.s_new] = make_double2(sr, si);
      G[(int64_t)a.s_new * a.m + j] = make_double2(sr, -si);
    }
  }
  if (threadIdx.x == 0) {
    a.ticket[0] = 0u;
    a.ticket[1] = 0u;
  }
}

template <int kMode>
__global__ void __launch_bounds__(kGrThreads, 1) gram_row_bulk_kernel(GramRowArgs a) {
  constexpr bool kU8 = (kMode == kModeU8);
  extern __shared__ __align__(128) uint8_t smem_raw[];
  Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = threadIdx.x; j < a.c; j += blockDim.x) {
    sm.acc_i[j] = 0;
    sm.acc_d[j] = 0.0;
    sm.acc_im[j] = 0.0;
  }
  if (threadIdx.x == 0) {
    for (int w = 0; w < kGrWarps; ++w)
      for (int s = 0; s < kStages; ++s) mbar_init(smem_u32(&sm.bar[w][s]), 1);
    mbar_init(smem_u32(&sm.xbar[0]), 1);
    mbar_init(smem_u32(&sm.xbar[1]), 1);
    sm.fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  const uint8_t* xnew = a.ring + (int64_t)a.s_new * a.slot_bytes;
  const int nmine = (a.c > warp) ? (a.c - warp + kGrWarps - 1) / kGrWarps : 0;  // slots of this warp
  // chunk ordinal k of this CTA -> chunk index sm.cq[k & 1] (>= nblk: none)
  auto chunk_len = [&](int ch) -> int { return (int)min(a.chunk, a.slot_bytes - (int64_t)ch * a.chunk); };
  auto issue_x = [&](int k, int ch) {          // x_new's piece of chunk ordinal k
    const unsigned xb = smem_u32(&sm.xbar[k & 1]);
    const int len = chunk_len(ch);
    mbar_expect_tx(xb, (unsigned)len);
    bulk_g2s(smem_u32(sm.xs[k & 1]), xnew + (int64_t)ch * a.chunk, (unsigned)len, xb);
  };
  if (threadIdx.x == 0) {
    const int c0 = (int)atomicAdd(a.ticket + 1, 1u);
    sm.cq[0] = c0;
    if (c0 < a.nblk) issue_x(0, c0);
  }
  // per-warp item stream: item (k, i) = piece i % np of slot i / np of chunk
  // ordinal k; lane 0 keeps the ring kStages items ahead, into chunk k + 1
  // once it is known
  unsigned consumed = 0, issued = 0;   // items of this warp (all chunks)
  int kc = 0, ic = 0;                  // issue cursor: chunk ordinal, item
  bool failed = false;                 // a bounded wait expired: stop issuing, drain, finish
  auto top_up = [&](int k) {           // chunk ordinals k and k + 1 are known
    if (lane != 0 || failed) return;
    while (issued - consumed < (unsigned)kStages && kc <= k + 1) {
      const int ch = sm.cq[kc & 1];
      if (ch >= a.nblk) break;
      const int np = chunk_len(ch) / kPiece;
      if (ic >= nmine * np) {
        ++kc;
        ic = 0;
        continue;
      }
      const unsigned s = issued % kStages;
      const int j = (a.s_first + warp + kGrWarps * (ic / np)) % a.m;
      const unsigned b = smem_u32(&sm.bar[warp][s]);
      mbar_expect_tx(b, kPiece);
      bulk_g2s(smem_u32(sm.stage[warp][s]),
               a.ring + (int64_t)j * a.slot_bytes + (int64_t)ch * a.chunk + (int64_t)kPiece * (ic % np), kPiece, b);
      ++ic;
      ++issued;
    }
  };
  for (int k = 0;; ++k) {
    __syncthreads();                   // chunk k - 1 fully consumed: xs[(k + 1) & 1] is free
    if (threadIdx.x == 0) {
      const int ch = sm.cq[k & 1];
      int nx = a.nblk;
      if (ch < a.nblk && !sm.fail) nx = (int)atomicAdd(a.ticket + 1, 1u);
      sm.cq[(k + 1) & 1] = nx;
      if (nx < a.nblk) issue_x(k + 1, nx);
    }
    __syncthreads();
    const int ch = sm.cq[k & 1];
    if (ch >= a.nblk) break;
    const int np = chunk_len(ch) / kPiece;
    const int nitems = nmine * np;
    top_up(k);
    if (!failed && !mbar_wait(smem_u32(&sm.xbar[k & 1]), (unsigned)((k >> 1) & 1))) failed = true;
    failed = __any_sync(0xffffffffu, failed);
    unsigned int su = 0;
    double sd = 0.0, si = 0.0;
    const uint8_t* xs = sm.xs[k & 1];
    for (int it = 0; it < nitems && !failed; ++it) {
      const unsigned s = consumed % kStages, par = (consumed / kStages) & 1;
      const int q = it % np;
      bool bad = !mbar_wait(smem_u32(&sm.bar[warp][s]), par);
      if (__any_sync(0xffffffffu, bad)) {
        failed = true;
        break;
      }
      const uint8_t* piece = sm.stage[warp][s];
      const uint8_t* xq = xs + kPiece * q;
      if constexpr (kU8) {
#pragma unroll
        for (int u = 0; u < kPiece / 512; ++u) {
          const uint4 v = *reinterpret_cast<const uint4*>(piece + 16 * lane + 512 * u);
          const uint4 w = *reinterpret_cast<const uint4*>(xq + 16 * lane + 512 * u);
          su = __dp4a(v.x, w.x, su);
          su = __dp4a(v.y, w.y, su);
          su = __dp4a(v.z, w.z, su);
          su = __dp4a(v.w, w.w, su);
        }
      } else if constexpr (kMode == kModeF32) {
        float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;
#pragma unroll
        for (int u = 0; u < kPiece / 512; ++u) {
          const float4 v = *reinterpret_cast<const float4*>(piece + 16 * lane + 512 * u);
          const float4 w = *reinterpret_cast<const float4*>(xq + 16 * lane + 512 * u);
          f0 = fmaf(v.x, w.x, f0);
          f1 = fmaf(v.y, w.y, f1);
          f2 = fmaf(v.z, w.z, f2);
          f3 = fmaf(v.w, w.w, f3);
        }
        sd += (double)((f0 + f1) + (f2 + f3));
      } else if constexpr (kMode == kModeF64) {
        double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
#pragma unroll
        for (int u = 0; u < kPiece / 512; ++u) {
          const float4 v = *reinterpret_cast<const float4*>(piece + 16 * lane + 512 * u);
          const float4 w = *reinterpret_cast<const float4*>(xq + 16 * lane + 512 * u);
          d0 = fma((double)v.x, (double)w.x, d0);
          d1 = fma((double)v.y, (double)w.y, d1);
          d2 = fma((double)v.z, (double)w.z, d2);
          d3 = fma((double)v.w, (double)w.w, d3);
        }
        sd += (d0 + d1) + (d2 + d3);
      } else {
        // two complex64 values per 16 bytes: conj(v) * w
        float r0 = 0.f, r1 = 0.f, i0 = 0.f, i1 = 0.f;
#pragma unroll
        for (int u = 0; u < kPiece / 512; ++u) {
          const float4 v = *reinterpret_cast<const float4*>(piece + 16 * lane + 512 * u);
          const float4 w = *reinterpret_cast<const float4*>(xq + 16 * lane + 512 * u);
          r0 = fmaf(v.x, w.x, fmaf(v.y, w.y, r0));
          r1 = fmaf(v.z, w.z, fmaf(v.w, w.w, r1));
          i0 = fmaf(v.x, w.y, fmaf(-v.y, w.x, i0));
          i1 = fmaf(v.z, w.w, fmaf(-v.w, w.z, i1));
        }
        sd += (double)(r0 + r1);
        si += (double)(i0 + i1);
      }
      __syncwarp();                    // all lanes are done reading stage s
      ++consumed;
      top_up(k);
      if (q == np - 1) {               // this slot is finished for the chunk
        const int jj = warp + kGrWarps * (it / np);
        if constexpr (kU8) {
          const long long t = warp_sum((long long)su);
          if (lane == 0) sm.acc_i[jj] += t;
          su = 0;
        } else {
          const double t = warp_sum(sd);
          if (lane == 0) sm.acc_d[jj] += t;
          sd = 0.0;
          if constexpr (kMode == kModeC64) {
            const double ti = warp_sum(si);
            if (lane == 0) sm.acc_im[jj] += ti;
            si = 0.0;
          }
        }
      }
    }
    if (failed) {
      if (lane == 0) {
        atomicOr(a.status, kDevTimeout);
        sm.fail = 1;
      }
    }
    __syncthreads();
    // this chunk's partials (each thread writes and clears its own slots)
    for (int j = threadIdx.x; j < a.c; j += blockDim.x) {
      if constexpr (kU8) {
        static_cast<long long*>(a.partials)[(int64_t)j * a.nblk + ch] = sm.acc_i[j];
      } else if constexpr (kMode == kModeF32 || kMode == kModeF64) {
        static_cast<double*>(a.partials)[(int64_t)j * a.nblk + ch] = sm.acc_d[j];
      } else {
        static_cast<double2*>(a.partials)[(int64_t)j * a.nblk + ch] = make_double2(sm.acc_d[j], sm.acc_im[j]);
      }
      sm.acc_i[j] = 0;
      sm.acc_d[j] = 0.0;
      sm.acc_im[j] = 0.0;
    }
    if (sm.fail) {
      // copies issued but not consumed must land before the shared memory
      // is released (bounded waits); then stop
      if (lane == 0)
        for (unsigned gk = consumed; gk < issued; ++gk) mbar_wait(smem_u32(&sm.bar[warp][gk % kStages]), (gk / kStages) & 1);
      if (threadIdx.x == 0 && sm.cq[(k + 1) & 1] < a.nblk) mbar_wait(smem_u32(&sm.xbar[(k + 1) & 1]), (unsigned)(((k + 1) >> 1) & 1));
      break;
    }
  }
  if constexpr (kU8) {
    finish_row<long long>(a, sm);
  } else if constexpr (kMode == kModeF32 || kMode == kModeF64) {
    finish_row<double>(a, sm);
  } else {
    finish_row_c64(a, sm);
  }
}

// ---------------------------------------------------------------------------
// Batched rows: one new snapshot of each of up to kMaxBatchJobs handles (mixed
// n, window and element type) in one launch. Work items are (job, chunk)
// pairs over the concatenated chunk lists, taken from a counter by
// persistent CTAs. Each item is computed exactly as the single-handle kernel
// computes that chunk (same warp-to-slot assignment, piece order and per-lane
// sums), its partials go to the job's [slot][chunk] array, and the CTA that
// completes a job's last chunk reduces the job's row in the same fixed order,
// so every row is bit-identical to the handle's own sdmd_push.

struct BatchSmem {
  uint8_t stage[kGrWarps][kStages][kPiece];
  uint8_t xs[kXSub];
  unsigned long long bar[kGrWarps][kStages];
  unsigned long long xbar;
  int item, job, ch, fail, last;
  long long acc_i[SDMD_MAX_M];
  double acc_d[SDMD_MAX_M];
  double acc_im[SDMD_MAX_M];
};

template <int kMode>
__device__ __forceinline__ void piece_sums(const uint8_t* piece, const uint8_t* xq, int lane, unsigned& su, double& sd,
                                           double& si) {
  if constexpr (kMode == kModeU8) {
#pragma unroll
    for (int u = 0; u < kPiece / 512; ++u) {
      const uint4 v = *reinterpret_cast<const uint4*>(piece + 16 * lane + 512 * u);
      const uint4 w = *reinterpret_cast<const uint4*>(xq + 16 * lane + 512 * u);
      su = __dp4a(v.x, w.x, su);
      su = __dp4a(v.y, w.y, su);
      su = __dp4a(v.z, w.z, su);
      su = __dp4a(v.w, w.w, su);
    }
  } else if constexpr (kMode == kModeF32) {
    float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;
#pragma unroll
    for (int u = 0; u < kPiece / 512; ++u) {
      const float4 v = *reinterpret_cast<const float4*>(piece + 16 * lane + 512 * u);
      const float4 w = *reinterpret_cast<const float4*>(xq + 16 * lane + 512 * u);
      f0 = fmaf(v.x, w.x, f0);
      f1 = fmaf(v.y, w.y, f1);
      f2 = fmaf(v.z, w.z, f2);
      f3 = fmaf(v.w, w.w, f3);
    }
    sd += (double)((f0 + f1) + (f2 + f3));
  } else if constexpr (kMode == kModeF64) {
    double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
#pragma unroll
    for (int u = 0; u < kPiece / 512; ++u) {
      const float4 v = *reinterpret_cast<const float4*>(piece + 16 * lane + 512 * u);
      const float4 w = *reinterpret_cast<const float4*>(xq + 16 * lane + 512 * u);
      d0 = fma((double)v.x, (double)w.x, d0);
      d1 = fma((double)v.y, (double)w.y, d1);
      d2 = fma((double)v.z, (double)w.z, d2);
      d3 = fma((double)v.w, (double)w.w, d3);
    }
    sd += (d0 + d1) + (d2 + d3);
  } else {
    float r0 = 0.f, r1 = 0.f, i0 = 0.f, i1 = 0.f;
#pragma unroll
    for (int u = 0; u < kPiece / 512; ++u) {
      const float4 v = *reinterpret_cast<const float4*>(piece + 16 * lane + 512 * u);
      const float4 w = *reinterpret_cast<const float4*>(xq + 16 * lane + 512 * u);
      r0 = fmaf(v.x, w.x, fmaf(v.y, w.y, r0));
      r1 = fmaf(v.z, w.z, fmaf(v.w, w.w, r1));
      i0 = fmaf(v.x, w.y, fmaf(-v.y, w.x, i0));
      i1 = fmaf(v.z, w.w, fmaf(-v.w, w.z, i1));
    }
    sd += (double)(r0 + r1);
    si += (double)(i0 + i1);
  }
}

// One item: chunk `ch` of job `J`; returns false if a wait expired.
template <int kMode>
__device__ bool batch_item(const RowJob& J, int ch, BatchSmem& sm, unsigned& g, int item_no) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t beg = (int64_t)ch * J.chunk;
  const int len = (int)min(J.chunk, J.slot_bytes - beg);
  const int np = len / kPiece;
  const int nmine = (J.c > warp) ? (J.c - warp + kGrWarps - 1) / kGrWarps : 0;
  const int nitems = nmine * np;
  const uint8_t* xnew = J.ring + (int64_t)J.s_new * J.slot_bytes;
  if (threadIdx.x == 0) {
    const unsigned xb = smem_u32(&sm.xbar);
    mbar_expect_tx(xb, (unsigned)len);
    bulk_g2s(smem_u32(sm.xs), xnew + beg, (unsigned)len, xb);
  }
  auto issue = [&](int it) {
    const unsigned s = (g + it) % kStages;
    const int j = (J.s_first + warp + kGrWarps * (it / np)) % J.m;
    const unsigned b = smem_u32(&sm.bar[warp][s]);
    mbar_expect_tx(b, kPiece);
    bulk_g2s(smem_u32(sm.stage[warp][s]), J.ring + (int64_t)j * J.slot_bytes + beg + (int64_t)kPiece * (it % np), kPiece,
             b);
  };
  if (lane == 0)
    for (int it = 0; it < kStages && it < nitems; ++it) issue(it);
  bool failed = !mbar_wait(smem_u32(&sm.xbar), (unsigned)(item_no & 1));
  failed = __any_sync(0xffffffffu, failed);
  int consumed = 0;
  unsigned su = 0;
  double sd = 0.0, si = 0.0;
  for (int it = 0; it < nitems && !failed; ++it) {
    const unsigned gi = g + it, s = gi % kStages, par = (gi / kStages) & 1;
    const int q = it % np;
    const bool bad = !mbar_wait(smem_u32(&sm.bar[warp][s]), par);
    if (__any_sync(0xffffffffu, bad)) {
      failed = true;
      break;
    }
    piece_sums<kMode>(sm.stage[warp][s], sm.xs + kPiece * q, lane, su, sd, si);
    __syncwarp();
    ++consumed;
    if (lane == 0 && it + kStages < nitems) issue(it + kStages);
    if (q == np - 1) {
      const int jj = warp + kGrWarps * (it / np);
      if constexpr (kMode == kModeU8) {
        const long long t = warp_sum((long long)su);
        if (lane == 0) sm.acc_i[jj] += t;
        su = 0;
      } else {
        const double t = warp_sum(sd);
        if (lane == 0) sm.acc_d[jj] += t;
        sd = 0.0;
        if constexpr (kMode == kModeC64) {
          const double ti = warp_sum(si);
          if (lane == 0) sm.acc_im[jj] += ti;
          si = 0.0;
        }
      }
    }
  }
  if (failed && lane == 0) {           // copies in flight land before the memory is reused
    const int issued = nitems < consumed + kStages ? nitems : consumed + kStages;
    for (int it = consumed; it < issued; ++it) mbar_wait(smem_u32(&sm.bar[warp][(g + it) % kStages]), ((g + it) / kStages) & 1);
    mbar_wait(smem_u32(&sm.xbar), (unsigned)(item_no & 1));
  }
  g += nitems;
  return !failed;
}

template <typename Acc>
__device__ void batch_finish(const RowJob& J) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Acc* P = static_cast<const Acc*>(J.partials);
  Acc* G = static_cast<Acc*>(J.G);
  for (int jj = warp; jj < J.c; jj += kGrWarps) {
    Acc s = 0;
    for (int b = lane; b < J.nblk; b += 32) s += __ldcg(P + (int64_t)jj * J.nblk + b);
    s = warp_sum(s);
    if (lane == 0) {
      const int j = (J.s_first + jj) % J.m;
      G[(int64_t)J.s_new * J.m + j] = s;
      G[(int64_t)j * J.m + J.s_new] = s;
    }
  }
}

__device__ void batch_finish_c64(const RowJob& J) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double2* P = static_cast<const double2*>(J.partials);
  double2* G = static_cast<double2*>(J.G);
  for (int jj = warp; jj < J.c; jj += kGrWarps) {
    double sr = 0.0, si = 0.0;
    for (int b = lane; b < J.nblk; b += 32) {
      const double2 v = __ldcg(P + (int64_t)jj * J.nblk + b);
      sr += v.x;
      si += v.y;
    }
    sr = warp_sum(sr);
    si = warp_sum(si);
    if (lane == 0) {
      const int j = (J.s_first + jj) % J.m;
      if (j == J.s_new) si = 0.0;
      G[(int64_t)j * J.m + J.s_new] = make_double2(sr, si);
      G[(int64_t)J.s_new * J.m + j] = make_double2(sr, -si);
    }
  }
}

__global__ void __launch_bounds__(kGrThreads, 1) gram_rows_batched_kernel(const __grid_constant__ BatchArgs a) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  BatchSmem& sm = *reinterpret_cast<BatchSmem*>(smem_raw);
  for (int j = threadIdx.x; j < SDMD_MAX_M; j += blockDim.x) {
    sm.acc_i[j] = 0;
    sm.acc_d[j] = 0.0;
    sm.acc_im[j] = 0.0;
  }
  if (threadIdx.x == 0) {
    for (int w = 0; w < kGrWarps; ++w)
      for (int s = 0; s < kStages; ++s) mbar_init(smem_u32(&sm.bar[w][s]), 1);
    mbar_init(smem_u32(&sm.xbar), 1);
    sm.fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  unsigned g = 0;                      // this warp's pieces so far (ring position)
  for (int item_no = 0;; ++item_no) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const int it = sm.fail ? a.nitems : (int)atomicAdd(a.grab, 1u);
      int jb = 0;
      if (it < a.nitems)
        while (jb + 1 < a.njobs && a.job[jb + 1].item0 <= it) ++jb;
      sm.item = it;
      sm.job = jb;
      sm.ch = it - a.job[jb].item0;
    }
    __syncthreads();
    if (sm.item >= a.nitems) break;
    const RowJob& J = a.job[sm.job];
    const int ch = sm.ch;
    bool ok;
    if (J.mode == kModeU8) ok = batch_item<kModeU8>(J, ch, sm, g, item_no);
    else if (J.mode == kModeF32) ok = batch_item<kModeF32>(J, ch, sm, g, item_no);
    else if (J.mode == kModeF64) ok = batch_item<kModeF64>(J, ch, sm, g, item_no);
    else ok = batch_item<kModeC64>(J, ch, sm, g, item_no);
    if (!ok && (threadIdx.x & 31) == 0) {
      atomicOr(a.status, kDevTimeout);
      sm.fail = 1;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < J.c; j += blockDim.x) {
      if (J.mode == kModeU8) static_cast<long long*>(J.partials)[(int64_t)j * J.nblk + ch] = sm.acc_i[j];
      else if (J.mode == kModeF32 || J.mode == kModeF64)
        static_cast<double*>(J.partials)[(int64_t)j * J.nblk + ch] = sm.acc_d[j];
      else static_cast<double2*>(J.partials)[(int64_t)j * J.nblk + ch] = make_double2(sm.acc_d[j], sm.acc_im[j]);
      sm.acc_i[j] = 0;
      sm.acc_d[j] = 0.0;
      sm.acc_im[j] = 0.0;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) sm.last = (atomicAdd(J.ticket, 1u) == (unsigned)J.nblk - 1u);
    __syncthreads();
    if (sm.last) {                     // this job's chunks are all in: reduce its row
      __threadfence();
      if (J.mode == kModeU8) batch_finish<long long>(J);
      else if (J.mode == kModeF32 || J.mode == kModeF64) batch_finish<double>(J);
      else batch_finish_c64(J);
      if (threadIdx.x == 0) J.ticket[0] = 0u;
    }
  }
  // the last CTA out zeroes the batch counters for the next launch
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(a.grab + 1, 1u) == gridDim.x - 1u) {
      a.grab[0] = 0u;
      a.grab[1] = 0u;
    }
  }
}

}  // namespace

// Two chunks per SM: persistent CTAs take chunks as they free
// up, so a launch is not held back by SMs that another stream's kernel (a
// frame's eigensolver) occupies; the partials stay indexed by chunk, so the
// fixed-order reduction and the result do not change.
constexpr int kChunksPerSm = 2;

void gram_row_schedule(int64_t slot_bytes, int num_sms, int64_t* chunk, int32_t* nblk) {
  gram_row_schedule_k(slot_bytes, num_sms, kChunksPerSm, chunk, nblk);
}

void gram_row_schedule_k(int64_t slot_bytes, int num_sms, int chunks_per_sm, int64_t* chunk, int32_t* nblk) {
  const int64_t units = (slot_bytes + kPiece - 1) / kPiece;
  int64_t want = (int64_t)(chunks_per_sm > 0 ? chunks_per_sm : 1) * (num_sms > 0 ? num_sms : 1);
  if (want > units) want = units;
  int64_t per = (units + want - 1) / want;           // 4 KiB units per chunk
  if (per > kXSub / kPiece) per = kXSub / kPiece;   // at most 24 KiB (x_new double buffer)
  *chunk = per * kPiece;
  *nblk = (int32_t)((units + per - 1) / per);
}

cudaError_t launch_gram_row(int dtype, bool f64_ref, const GramRowArgs& a, cudaStream_t st) {
  const size_t smem = sizeof(Smem);
  {
    cudaError_t e = smem_optin(reinterpret_cast<const void*>(gram_row_bulk_kernel<kModeU8>), smem);
    if (e == cudaSuccess) e = smem_optin(reinterpret_cast<const void*>(gram_row_bulk_kernel<kModeF32>), smem);
    if (e == cudaSuccess) e = smem_optin(reinterpret_cast<const void*>(gram_row_bulk_kernel<kModeC64>), smem);
    if (e == cudaSuccess) e = smem_optin(reinterpret_cast<const void*>(gram_row_bulk_kernel<kModeF64>), smem);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ctas = a.nblk < sms ? a.nblk : (sms > 0 ? sms : 1);   // persistent
  if (dtype == SDMD_U8)
    gram_row_bulk_kernel<kModeU8><<<ctas, kGrThreads, smem, st>>>(a);
  else if (dtype == SDMD_C64)
    gram_row_bulk_kernel<kModeC64><<<ctas, kGrThreads, smem, st>>>(a);
  else if (f64_ref)
    gram_row_bulk_kernel<kModeF64><<<ctas, kGrThreads, smem, st>>>(a);
  else
    gram_row_bulk_kernel<kModeF32><<<ctas, kGrThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t batched_kernel_config(const BatchArgs& a, cudaKernelNodeParams* p) {
  const size_t smem = sizeof(BatchSmem);
  {
    const cudaError_t e = smem_optin(reinterpret_cast<const void*>(gram_rows_batched_kernel), smem);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ctas = a.nitems < sms ? a.nitems : (sms > 0 ? sms : 1);
  p->func = reinterpret_cast<void*>(gram_rows_batched_kernel);
  p->gridDim = dim3((unsigned)(ctas > 0 ? ctas : 1));
  p->blockDim = dim3(kGrThreads);
  p->sharedMemBytes = (unsigned)smem;
  p->kernelParams = nullptr;
  p->extra = nullptr;
  return cudaSuccess;
}

cudaError_t launch_gram_rows_batched(const BatchArgs& a, cudaStream_t st) {
  const size_t smem = sizeof(BatchSmem);
  {
    const cudaError_t e = smem_optin(reinterpret_cast<const void*>(gram_rows_batched_kernel), smem);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ctas = a.nitems < sms ? a.nitems : (sms > 0 ? sms : 1);
  gram_rows_batched_kernel<<<ctas, kGrThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sdmd
