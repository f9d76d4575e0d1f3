// Full-window Gram G = X^T X of uint8 snapshots on the 5th-generation tensor
// cores: the rebuild of Algorithm 1's first step (Sec. 2.1, Eq. 3) with one
// read of the window instead of one pass per row.
//
// Exactness. Pixels are centred, x' = x - 128 in [-128, 127], which fp16
// holds exactly; a product is at most 2^14 in magnitude and a sum of 1024 of
// them at most 2^24, so an FP32 tensor-memory accumulator that collects 1024
// positions holds an exact integer. Every 1024 positions the accumulator is
// drained into int64 sums, so G' = X'^T X' is exact for any n. A constant
// row of ones (1 at positions < n) rides along as one more snapshot, so the
// same MMAs give the column sums s_i = sum_k x'_ik and the count n, and
//   G_ij = G'_ij + 128 (s_i + s_j) + 128^2 n        (exact int64).
//
// GEMM. One launch: the rows of one K-major fp16 tile T (128 rows x 256
// positions, zero rows past the used ones) are a group of k <= 64 target
// snapshots, the ones row, then a block of older snapshots. D[128 x N] +=
// T T_B^T, where T_B is the first N = k + 1 (rounded up to 16) rows of the
// same tile, so A and B share one shared-memory descriptor and D holds every
// <x_i, x_j> with x_j a target. The host call covers the k newest snapshots
// of a window of c (k = c: a full rebuild) with groups of at most 64 targets,
// newest first, each paired with every older snapshot in blocks of
// 127 - (group size) rows (a group with nothing older: one launch of its
// own); a window of at most 127 snapshots is one launch whatever k. Pairs
// inside a group are recomputed by each of its launches, with the same
// (exact) result. Core matrix (rg, kg) = rows 8 rg .. 8 rg + 7
// x positions 8 kg .. 8 kg + 7 at (kg * 16 + rg) * 128 bytes: LBO 2048 B
// between K neighbours, SBO 128 B between row groups.
//
// Work: persistent CTAs take chunks of 4096 positions (16 K-steps of 256)
// from a global counter; the integer sums do not depend on which CTA took
// which chunk. Per CTA:
//   warps 9..11  load + convert: warp-private regions of 8 rows x 256 bytes,
//                cp.async copies (quarter warp = 128 contiguous bytes) into
//                a 2-deep staging ring (row pitch 272 B), conversion with a
//                byte permute (fp16 1024 + b) and one f16x2 subtraction of
//                1152, written into a 2-deep ring of fp16 tiles; bulk L2
//                prefetches keep the next 1-2 KiB of every row on its way;
//   warp 8       lane 0 issues 16 MMAs per K-step into one of two TMEM
//                accumulators (128 x N FP32) and commits every 4 K-steps;
//   warps 0..7   drain: each reads its 32 TMEM lanes x N/2 columns and adds
//                the exact integers into int64 registers; at the end the
//                CTA's partial G' goes to a [CTA][128][128] array.
// A second kernel sums the partials over CTAs and writes G (physical slots).
// Every wait is bounded; on expiry the status word gets kDevTimeout, all
// roles stop, copies and MMAs are waited for (bounded) and TMEM is freed.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sdmd_internal.cuh"
#include "tc_util.cuh"

namespace sdmd {

namespace {

using namespace tc;

constexpr int kDrainWarps = 8;       // warps 0..7
constexpr int kMmaWarp = 8;
constexpr int kConvWarp0 = 9;
constexpr int kConvWarps = 3;
constexpr int kThreads = 32 * (kConvWarp0 + kConvWarps);   // 384
constexpr int kRowsM = 128;          // MMA M
constexpr int kKst = 256;            // positions per K-step
constexpr int kStepsPerChunk = 16;   // scheduling unit: 4096 positions
constexpr int kStepsPerDrain = 4;    // 1024 positions per accumulator period
constexpr int kStages = 2;           // staging ring (u8)
constexpr int kTiles = 2;            // fp16 tile ring
constexpr int kPitch = 272;          // staging row pitch, bytes
constexpr int kTileBytes = kRowsM * kKst * 2;              // 65536
constexpr int kStageBytes = kRowsM * kPitch;               // 34816
constexpr int kTmemCols = 256;       // two accumulators of <= 128 columns

struct FullShared {
  unsigned long long tile_full[kTiles];   // tile converted (converter warps)
  unsigned long long tile_free[kTiles];   // MMAs reading the tile done (commit)
  unsigned long long acc_full[2];         // accumulator period done (commit + issuer's release)
  unsigned long long acc_empty[2];        // accumulator drained (drain warps)
  unsigned long long chunk_bar[2];        // chunk start published (by chunk parity)
  int chunk[2];
  int dflag[2];                           // 1: the period holds data, 0: stop
  int kend;                               // number of K-steps of this CTA (once known)
  int stop;
  unsigned tmem_base;
  int64_t tab[kRowsM];                    // ring byte offset of window row i
};

constexpr int kSmemBytes = kTiles * kTileBytes + kStages * kStageBytes + (int)sizeof(FullShared);


// 16 pixels -> 2 x 8 centred fp16 (x - 128): fp16 0x64bb = 1024 + b, minus 1152
__device__ __forceinline__ unsigned f16x2_centred(unsigned w, unsigned sel) {
  const unsigned t = __byte_perm(w, 0x64u, sel);
  unsigned d;
  asm("sub.rn.f16x2 %0, %1, %2;\n" : "=r"(d) : "r"(t), "r"(0x64806480u));
  return d;
}

__device__ __forceinline__ void raise_timeout(int* status, volatile int* stop) {
  atomicOr(status, kDevTimeout);
  *stop = 1;
}

struct Ring {
  int idx = 0;
  unsigned phase = 0;
  __device__ __forceinline__ void next(int size) {
    if (++idx == size) {
      idx = 0;
      phase ^= 1u;
    }
  }
};

__global__ void __launch_bounds__(kThreads, 1) gram_full_tc_kernel(GramFullArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* tiles = smem;
  uint8_t* stg = smem + kTiles * kTileBytes;
  FullShared& sh = *reinterpret_cast<FullShared*>(smem + kTiles * kTileBytes + kStages * kStageBytes);
  volatile int* stop = &sh.stop;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kt = a.k;                    // targets: tile rows 0 .. kt - 1; row kt is the ones row
  const int c = kt + a.nold;             // last tile row in use (the older block ends there)
  const int npad = ((kt + 1 + 15) / 16) * 16;
  const int64_t nchunks = (a.n + (int64_t)kKst * kStepsPerChunk - 1) / ((int64_t)kKst * kStepsPerChunk);

  if (tid == 0) {
    for (int b = 0; b < kTiles; ++b) {
      mbar_init(smem_u32(&sh.tile_full[b]), kConvWarps);
      mbar_init(smem_u32(&sh.tile_free[b]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&sh.acc_full[b]), 2);
      mbar_init(smem_u32(&sh.acc_empty[b]), kDrainWarps);
      mbar_init(smem_u32(&sh.chunk_bar[b]), 1);
    }
    sh.kend = 0x7fffffff;
    sh.stop = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == kMmaWarp) tmem_alloc(smem_u32(&sh.tmem_base), kTmemCols);
  for (int r = tid; r <= c; r += kThreads) {
    if (r == kt) continue;
    const int t = (r < kt) ? a.t_tgt + r : a.t_old + (r - kt - 1);   // window time index of tile row r
    sh.tab[r] = (int64_t)((a.start + t) % a.m) * a.slot_bytes;
  }
  // rows beyond the ones row stay zero in both tiles
  for (int idx = tid; idx < kTiles * kRowsM * (kKst / 8); idx += kThreads) {
    const int t = idx / (kRowsM * (kKst / 8)), rem = idx - t * (kRowsM * (kKst / 8));
    const int row = rem % kRowsM, kg = rem / kRowsM;
    if (row > c) *reinterpret_cast<uint4*>(tiles + t * kTileBytes + (kg * 16 + (row >> 3)) * 128 + (row & 7) * 16) =
                     make_uint4(0u, 0u, 0u, 0u);
  }
  fence_proxy_async();
  fence_before();
  __syncthreads();
  fence_after();
  const unsigned tbase = sh.tmem_base;

  if (warp >= kConvWarp0) {
    // ---------------- load + convert ----------------
    const int cw = warp - kConvWarp0;
    const int ngroups = (c + 1 + 7) / 8;                       // row groups incl. the ones row
    const unsigned stg0 = smem_u32(stg);
    // K-step sequence: chunk k covers K-steps 16 k .. 16 k + 15 of this CTA
    int ld_count = 0, nvalid = 0x7fffffff, cbase = 0;
    bool ended = false;
    // fix the position of K-step number ld_count (or -1 past the end)
    auto fix_next = [&]() -> int64_t {
      int64_t p0 = -1;
      if (!ended) {
        const int ck = ld_count / kStepsPerChunk, o = ld_count % kStepsPerChunk;
        if (o == 0) {
          const unsigned bar = smem_u32(&sh.chunk_bar[ck & 1]);
          if (cw == 0 && lane == 0) {
            sh.chunk[ck & 1] = (int)atomicAdd(a.sched, 1u);
            mbar_arrive(bar);
          }
          int ok = 1;
          if (lane == 0) ok = mbar_wait(bar, (unsigned)((ck >> 1) & 1));
          ok = __shfl_sync(0xffffffffu, ok, 0);
          __syncwarp();
          if (ok) {
            cbase = sh.chunk[ck & 1];
          } else {
            if (lane == 0) raise_timeout(a.status, stop);
            cbase = (int)nchunks;
          }
          if (cbase < nchunks) {               // this chunk's first 8 K-steps (2 KiB per row) into L2
            const int64_t x0 = (int64_t)cbase * kStepsPerChunk * kKst;
            for (int q = cw * 32 + lane; q <= c; q += kConvWarps * 32)
              if (q != kt) bulk_prefetch_l2(a.ring + sh.tab[q] + x0, 8 * kKst);
          }
        } else if (o == 8 && cbase < nchunks) {  // the second half
          const int64_t x0 = ((int64_t)cbase * kStepsPerChunk + 8) * kKst;
          for (int q = cw * 32 + lane; q <= c; q += kConvWarps * 32)
            if (q != kt) bulk_prefetch_l2(a.ring + sh.tab[q] + x0, 8 * kKst);
        }
        if (cbase < nchunks) {
          p0 = ((int64_t)cbase * kStepsPerChunk + o) * kKst;
        } else {
          ended = true;
          nvalid = ld_count;
        }
      }
      ++ld_count;
      return p0;
    };
    int ld_stage = 0;
    int64_t pos0 = -1, pos1 = -1;            // first position of the K-step in stage 0 / 1
    auto load_next = [&]() {
      const int64_t p0 = fix_next();
      if (ld_stage == 0) pos0 = p0;
      else pos1 = p0;
      if (p0 >= 0) {
        const unsigned dst = stg0 + (unsigned)(ld_stage * kStageBytes);
        for (int g = cw; g < ngroups; g += kConvWarps) {
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int row = 8 * g + 2 * t + (lane >> 4), ch = lane & 15;
            if (row <= c && row != kt)
              cp_async16(dst + (unsigned)(row * kPitch + 16 * ch), a.ring + sh.tab[row] + p0 + 16 * ch);
          }
        }
      }
      ld_stage ^= 1;
    };
    load_next();
    cp_async_commit();
    int stage = 0;
    Ring tb;
    for (int s = 0; !*stop; ++s) {
      const bool valid = !(ended && s >= nvalid);
      load_next();
      cp_async_commit();
      cp_async_wait<1>();                    // this lane's copies of K-step s have landed
      __syncwarp();                          // ... and those of the other lanes
      const int64_t p0 = (stage == 0) ? pos0 : pos1;
      const uint8_t* sb = stg + stage * kStageBytes;
      stage ^= 1;
      int ok = 1;
      if (lane == 0 && s >= kTiles) ok = mbar_wait(smem_u32(&sh.tile_free[tb.idx]), tb.phase ^ 1u);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) raise_timeout(a.status, stop);
        break;
      }
      if (!valid) {                          // hand the end on to the MMA issuer and stop
        if (cw == 0 && lane == 0) sh.kend = s;
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&sh.tile_full[tb.idx]));
        break;
      }
      uint8_t* tile = tiles + tb.idx * kTileBytes;
      for (int g = cw; g < ngroups; g += kConvWarps) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int row = 8 * g + (lane & 7), ch = (lane >> 3) + 4 * t;   // 16 positions 16 ch ..
          if (row > c) continue;
          const int64_t pos = p0 + 16 * ch;
          uint4 lo, hi;
          if (row != kt) {
            const uint4 w = *reinterpret_cast<const uint4*>(sb + row * kPitch + 16 * ch);
            lo.x = f16x2_centred(w.x, 0x4140u);
            lo.y = f16x2_centred(w.x, 0x4342u);
            lo.z = f16x2_centred(w.y, 0x4140u);
            lo.w = f16x2_centred(w.y, 0x4342u);
            hi.x = f16x2_centred(w.z, 0x4140u);
            hi.y = f16x2_centred(w.z, 0x4342u);
            hi.z = f16x2_centred(w.w, 0x4140u);
            hi.w = f16x2_centred(w.w, 0x4342u);
          } else {                           // the ones row
            lo = make_uint4(0x3C003C00u, 0x3C003C00u, 0x3C003C00u, 0x3C003C00u);
            hi = lo;
          }
          if (pos + 16 > a.n) {              // positions past n contribute nothing
            unsigned wv[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int64_t pa = pos + 2 * q;
              if (pa >= a.n) wv[q] = 0u;
              else if (pa + 1 >= a.n) wv[q] &= 0x0000FFFFu;   // element 0 is the low half
            }
            lo = make_uint4(wv[0], wv[1], wv[2], wv[3]);
            hi = make_uint4(wv[4], wv[5], wv[6], wv[7]);
          }
          uint8_t* core = tile + (size_t)((2 * ch) * 16 + g) * 128 + (row & 7) * 16;
          *reinterpret_cast<uint4*>(core) = lo;
          *reinterpret_cast<uint4*>(core + 16 * 128) = hi;     // kg + 1: 16 row groups further
        }
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&sh.tile_full[tb.idx]));
      tb.next(kTiles);
    }
    cp_async_wait<0>();
  } else if (warp == kMmaWarp) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      // kind::f16, D f32, A = B = f16 K-major, M = 128, N = npad
      const uint32_t idesc = (1u << 4) | ((uint32_t)(npad >> 3) << 17) | ((uint32_t)(kRowsM >> 4) << 24);
      Ring tb, acc, last;
      int in_period = 0, periods = 0;
      bool ok = true;
      for (int s = 0;; ++s) {
        if (*stop) {
          ok = false;
          break;
        }
        ok = mbar_wait(smem_u32(&sh.tile_full[tb.idx]), tb.phase);
        if (!ok) break;
        if (s >= sh.kend) break;             // the converters handed on the end
        if (in_period == 0 && periods >= 2) {
          ok = mbar_wait(smem_u32(&sh.acc_empty[acc.idx]), acc.phase ^ 1u);
          if (!ok) break;
        }
        fence_after();
        const unsigned base = smem_u32(tiles + tb.idx * kTileBytes);
        const unsigned dt = tbase + (unsigned)(acc.idx * 128);
        for (int ks = 0; ks < kKst / 16; ++ks) {
          const uint64_t d = smem_desc(base + (unsigned)ks * 4096u, 2048u, 128u);
          mma_f16(dt, d, d, idesc, (in_period > 0 || ks > 0) ? 1u : 0u);
        }
        mma_commit(smem_u32(&sh.tile_free[tb.idx]));
        tb.next(kTiles);
        if (++in_period == kStepsPerDrain) {
          mma_commit(smem_u32(&sh.acc_full[acc.idx]));
          sh.dflag[acc.idx] = 1;
          mbar_arrive(smem_u32(&sh.acc_full[acc.idx]));
          last = acc;
          acc.next(2);
          ++periods;
          in_period = 0;
        }
      }
      if (ok && in_period > 0) {             // the last, partial period
        mma_commit(smem_u32(&sh.acc_full[acc.idx]));
        sh.dflag[acc.idx] = 1;
        mbar_arrive(smem_u32(&sh.acc_full[acc.idx]));
        last = acc;
        acc.next(2);
        ++periods;
      }
      if (ok && periods >= 2) ok = mbar_wait(smem_u32(&sh.acc_empty[acc.idx]), acc.phase ^ 1u);
      if (ok) {                              // stop marker for the drain warps
        sh.dflag[acc.idx] = 0;
        mbar_arrive2(smem_u32(&sh.acc_full[acc.idx]));
      } else {
        raise_timeout(a.status, stop);
      }
      // no MMA may write tensor memory once it is freed
      if (periods > 0) mbar_wait(smem_u32(&sh.acc_full[last.idx]), last.phase);
    }
  } else {
    // ---------------- drain (warps 0..7) ----------------
    const int lq = warp & 3, half = warp >> 2;
    const int cols = npad / 2;                       // multiple of 8, <= 64
    const int col0 = half * cols;
    long long sum[8][8];
#pragma unroll
    for (int pc = 0; pc < 8; ++pc)
#pragma unroll
      for (int i = 0; i < 8; ++i) sum[pc][i] = 0;
    Ring acc;
    for (;;) {
      if (*stop) break;
      int ok = 1;
      if (lane == 0) ok = mbar_wait(smem_u32(&sh.acc_full[acc.idx]), acc.phase);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) raise_timeout(a.status, stop);
        break;
      }
      if (!sh.dflag[acc.idx]) break;
      fence_after();
      const unsigned taddr = tbase + ((unsigned)(32 * lq) << 16) + (unsigned)(acc.idx * 128 + col0);
#pragma unroll
      for (int pc = 0; pc < 8; ++pc) {
        if (8 * pc < cols) {
          unsigned v[8];
          tmem_ld8_nowait(taddr + 8 * pc, v);
          tmem_ld_wait();
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            asm volatile("" : "+r"(v[i]));
            sum[pc][i] += (long long)__float2int_rn(__uint_as_float(v[i]));
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&sh.acc_empty[acc.idx]));
      acc.next(2);
    }
    // this CTA's partial G' (rows and columns 0 .. c; row/column c = sums)
    const int row = 32 * lq + lane;
    long long* P = a.partials + (int64_t)blockIdx.x * kRowsM * kRowsM;
#pragma unroll
    for (int pc = 0; pc < 8; ++pc)
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int col = col0 + 8 * pc + i;
        if (8 * pc < cols && row <= c && col <= kt) P[(int64_t)row * kRowsM + col] = sum[pc][i];
      }
  }
  __syncthreads();
  fence_after();
  __syncwarp();
  if (warp == kMmaWarp) tmem_dealloc(tbase, kTmemCols);
}

// G_ij = G'_ij + 128 (s_i + s_j) + 128^2 n from the per-CTA partials, for
// every tile row i (one block each) and target j (threads), written to both
// G[i][j] and G[j][i] at the physical slots.
__global__ void reset_sched_kernel(unsigned* sched) { sched[0] = 0u; }   // ready for the next launch

__global__ void gram_full_finish_kernel(GramFullArgs a, int ctas) {
  __shared__ long long si_n[2];
  const int i = blockIdx.x, kt = a.k;
  if (i == kt) return;                   // the ones row
  if (threadIdx.x < 2) {                 // s_i = G'_i,kt and n = G'_kt,kt
    const int rw = (threadIdx.x == 0) ? i : kt;
    long long s = 0;
    for (int b = 0; b < ctas; ++b) s += a.partials[((int64_t)b * kRowsM + rw) * kRowsM + kt];
    si_n[threadIdx.x] = s;
  }
  __syncthreads();
  const long long si = si_n[0], n = si_n[1];
  const int ti = (i < kt) ? a.t_tgt + i : a.t_old + (i - kt - 1);
  const int pi = (a.start + ti) % a.m;
  for (int j = threadIdx.x; j < kt; j += blockDim.x) {
    long long g = 0, sj = 0;
    for (int b = 0; b < ctas; ++b) {
      const long long* P = a.partials + (int64_t)b * kRowsM * kRowsM;
      g += P[(int64_t)i * kRowsM + j];
      sj += P[(int64_t)j * kRowsM + kt];
    }
    const long long v = g + 128LL * (si + sj) + 16384LL * n;
    const int pj = (a.start + a.t_tgt + j) % a.m;
    a.G[(int64_t)pi * a.m + pj] = v;
    a.G[(int64_t)pj * a.m + pi] = v;
  }
}

}  // namespace

cudaError_t launch_gram_full_tc(const GramFullArgs& base, int* ctas_out, cudaStream_t st) {
  const int c = base.c, k = base.k;
  if (c < 1 || c > SDMD_MAX_M || k < 1 || k > c) return cudaErrorNotSupported;
  {
    const cudaError_t e = smem_optin(reinterpret_cast<const void*>(gram_full_tc_kernel), kSmemBytes);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms < 1) sms = 1;
  const int ctas = sms < kGramFullMaxCtas ? sms : kGramFullMaxCtas;
  // targets = window time indices c - k .. c - 1 in groups of at most 64,
  // newest first; each group against the older snapshots 0 .. lo - 1 in
  // blocks of 127 - kg rows. A window of at most 127 fits one tile: one
  // launch whatever k.
  const int gmax = (c + 1 <= kRowsM) ? k : kGramFullMaxTargets;
  for (int hi = c; hi > c - k;) {
    const int lo = (hi - gmax > c - k) ? hi - gmax : c - k;
    const int kg = hi - lo;
    const int blk = kRowsM - 1 - kg;
    int o = 0;
    do {
      GramFullArgs a = base;
      a.t_tgt = lo;
      a.k = kg;
      a.t_old = o;
      a.nold = (lo - o < blk) ? lo - o : blk;
      gram_full_tc_kernel<<<ctas, kThreads, kSmemBytes, st>>>(a);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      gram_full_finish_kernel<<<a.k + 1 + a.nold, 128, 0, st>>>(a, ctas);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      reset_sched_kernel<<<1, 1, 0, st>>>(a.sched);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      o += a.nold;
    } while (o < lo);
    hi = lo;
  }
  if (ctas_out) *ctas_out = ctas;
  return cudaSuccess;
}

}  // namespace sdmd
