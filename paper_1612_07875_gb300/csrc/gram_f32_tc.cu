// Gram rows and columns of FP32 snapshots on the 5th-generation tensor cores
// in BF16x3 split precision: the multi-column catch-up and the full-window
// rebuild of Algorithm 1's first step (Sec. 2.1, Eq. 3) with one read of the
// window per block of target columns instead of one pass per column.
//
// Split. Every value is written as three bf16 terms, x = b0 + b1 + b2 + r:
// b0 = bf16(x), b1 = bf16(x - b0), b2 = bf16(x - b0 - b1) (round to nearest;
// each remainder is exact in FP32), |b1| <= 2^-8 |x|, |b2| <= 2^-16 |x| and
// |r| <= 2^-24 |x|. A product x y is taken as the six products b_i c_j with
// i + j <= 2; the dropped ones and the remainders are below 2^-22 |x y|.
//
// Two-term variant (split = 2): x = b0 + b1 + r2 with |r2| <= 2^-16 |x|, the
// three products with i + j <= 1; the dropped b1 c1 and remainders are about
// 2^-16 |x y| (the bf16x3 of three bf16 GEMMs).
//
// Accumulation. One accumulation period is one K-step of 64 positions: its
// cross-term MMAs (i + j >= 1, smallest first) run first, from a zeroed
// accumulator, then the 4 b0 c0 MMAs, so the FP32 tensor-memory accumulator
// rounds about 4 times at full magnitude per period. Every period is drained into
// compensated FP32 sums (hi + lo, error-free two-sum per value) per CTA, and
// the per-CTA sums are added in FP64 in a fixed order. Chunks are assigned to
// CTAs statically, so the result is the same on every run. Bound used by the
// tests: |G_ij - <x_i, x_j>| <= 1e-6 sum_p |x_ip x_jp|.
//
// GEMM. Tile rows (M = 128): first the k target snapshots (k <= 64), then a
// block of older snapshots. D[128 x N] += T_a T_b^T over the six term pairs,
// with T_b the first N = k (rounded up to 16) rows of the same term tiles, so
// D holds <x_i, x_j> for every tile row i and target j. Each term tile is
// K-major bf16, 128 rows x 64 positions in the 128-byte swizzle: row r is 128
// bytes at r * 128 and its 16-byte chunk c (positions 8 c .. 8 c + 7) sits at
// chunk c ^ (r & 7); eight rows form one 1024-byte atom (SBO 1024 B), and the
// K-slice of positions 16 j .. 16 j + 15 starts 32 j bytes into the tile.
//
// Roles (544 threads):
//   warps 9..16  load + split: warp-private row groups, cp.async 16-byte
//                copies (a half warp = one row's 256 contiguous bytes) into a
//                4-deep staging ring (16-byte chunk c of row r at chunk
//                c ^ (r & 7): conflict-free reads), bulk L2 prefetch of every row 2 KiB
//                ahead, then the three-term split into a 2-deep ring of term
//                tiles;
//   warp 8       lane 0 issues the 24 MMAs of a K-step into one of four TMEM
//                accumulators (128 x 64 FP32 each) and commits;
//   warps 0..7   drain: 32 TMEM lanes x N/2 columns each, two-sum into
//                registers; at the end the CTA's sums go to a partial array.
// A second kernel adds the partials over CTAs and writes G (physical slots).
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
constexpr int kConvWarps = 8;
constexpr int kGroupsPerWarp = 16 / kConvWarps;   // row groups of 8 per converter warp
constexpr int kThreads = 32 * (kConvWarp0 + kConvWarps);   // 544
constexpr int kRowsM = 128;          // MMA M
constexpr int kKst = 64;             // positions per K-step (= accumulation period)
constexpr int kStepsPerChunk = 16;   // scheduling unit: 1024 positions, 4 KiB per row
constexpr int kStages = 4;           // staging ring (fp32): three K-steps in flight
constexpr int kStagesStk = 3;        // ... with the stacked B tiles (two K-steps in flight)
constexpr int kStkMaxT = 32;         // targets (rounded to 16) for the stacked B tiles
constexpr int kTiles = 2;            // ring of term tiles
constexpr int kRowBytes = kKst * 4;                        // 256 B of a row per K-step
constexpr int kTermBytes = kRowsM * kKst * 2;              // 16384
constexpr int kTileBytes = 3 * kTermBytes;                 // 49152
constexpr int kStageBytes = kRowsM * kRowBytes;            // 32768
constexpr int kAcc = 4;              // TMEM accumulators
constexpr int kAccCols = kGramF32MaxTargets;               // 64 (the partials' row stride)
constexpr int kAccColsStk = 3 * kStkMaxT;                  // 96: three column groups
constexpr int kStkBytes = 3 * kStkMaxT * 128;              // stacked B tile: three terms' target rows

struct F32Shared {
  unsigned long long tile_full[kTiles];   // tile split (converter warps)
  unsigned long long tile_free[kTiles];   // MMAs reading the tile done (commit)
  unsigned long long acc_full[kAcc];      // period's MMAs done (commit)
  unsigned long long acc_empty[kAcc];     // accumulator drained (drain warps)
  int stop;
  unsigned tmem_base;
  int64_t tab[kRowsM];                    // ring byte offset of tile row i
};

template <bool kStk>
struct F32Layout {
  static constexpr int kSt = kStk ? kStagesStk : kStages;
  static constexpr int kStkOff = kTiles * kTileBytes;                  // 1024-aligned
  static constexpr int kStgOff = kStkOff + (kStk ? kTiles * kStkBytes : 0);
  static constexpr int kShOff = kStgOff + kSt * kStageBytes;
  static constexpr int kBytes = kShOff + (int)sizeof(F32Shared);
  static constexpr int kAccStride = kStk ? kAccColsStk : kAccCols;  // TMEM columns per accumulator
  static constexpr int kTmem = kStk ? 512 : 256;
};


__device__ __forceinline__ void raise_timeout(int* status, volatile int* stop) {
  atomicOr(status, kDevTimeout);
  *stop = 1;
}

// two FP32 values -> bf16x2 (first value in the low half), round to nearest
__device__ __forceinline__ unsigned bf16x2(float lo, float hi) {
  unsigned d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;\n" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
__device__ __forceinline__ float bf16_lo(unsigned p) { return __uint_as_float(p << 16); }
__device__ __forceinline__ float bf16_hi(unsigned p) { return __uint_as_float(p & 0xFFFF0000u); }

// (x0, x1) -> the three bf16x2 terms
__device__ __forceinline__ void split3(float x0, float x1, unsigned& t0, unsigned& t1, unsigned& t2) {
  t0 = bf16x2(x0, x1);
  const float r0 = __fsub_rn(x0, bf16_lo(t0)), r1 = __fsub_rn(x1, bf16_hi(t0));
  t1 = bf16x2(r0, r1);
  const float s0 = __fsub_rn(r0, bf16_lo(t1)), s1 = __fsub_rn(r1, bf16_hi(t1));
  t2 = bf16x2(s0, s1);
}

// error-free two-sum: hi + lo += v
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float v) {
  const float s = __fadd_rn(hi, v);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
  hi = s;
  lo = __fadd_rn(lo, e);
}

// kStk (targets rounded to 16 at most 32): the target rows of the three
// terms are also written, stacked, into a small B tile, so that one MMA per
// A term and K-slice covers all its B terms (N = 3, 2, 1 x npad): 12 MMAs per
// K-step instead of 24. The products b_i c_j then land in column group j;
// every group starts from zero (the drain writes zeros back after reading),
// takes its small terms first, and the drain adds the groups.
template <bool kStk>
__global__ void __launch_bounds__(kThreads, 1) gram_f32_tc_kernel(GramF32Args a) {
  using Lay = F32Layout<kStk>;
  constexpr int kSt = Lay::kSt;
  constexpr int kAccStride = Lay::kAccStride;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* tiles = smem;
  uint8_t* stk = smem + Lay::kStkOff;
  uint8_t* stg = smem + Lay::kStgOff;
  F32Shared& sh = *reinterpret_cast<F32Shared*>(smem + Lay::kShOff);
  volatile int* stop = &sh.stop;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kt = a.k;                          // targets: tile rows 0 .. kt - 1
  const int rows = a.k + a.nold;               // tile rows in use
  const int npad = ((kt + 15) / 16) * 16;
  const int64_t nchunks = (a.n + (int64_t)kKst * kStepsPerChunk - 1) / ((int64_t)kKst * kStepsPerChunk);
  const int64_t my_chunks = (nchunks > blockIdx.x) ? (nchunks - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t nsteps = my_chunks * kStepsPerChunk;

  if (tid == 0) {
    for (int b = 0; b < kTiles; ++b) {
      mbar_init(smem_u32(&sh.tile_full[b]), kConvWarps);
      mbar_init(smem_u32(&sh.tile_free[b]), 1);
    }
    for (int b = 0; b < kAcc; ++b) {
      mbar_init(smem_u32(&sh.acc_full[b]), 1);
      mbar_init(smem_u32(&sh.acc_empty[b]), kDrainWarps);
    }
    sh.stop = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == kMmaWarp) tmem_alloc(smem_u32(&sh.tmem_base), Lay::kTmem);
  for (int r = tid; r < rows; r += kThreads) {
    const int t = (r < kt) ? a.t_tgt + r : a.t_old + (r - kt);   // window time index of tile row r
    sh.tab[r] = (int64_t)((a.start + t) % a.m) * a.slot_bytes;
  }
  for (int idx = tid; idx < kSt * kStageBytes / 16; idx += kThreads)
    reinterpret_cast<uint4*>(stg)[idx] = make_uint4(0u, 0u, 0u, 0u);
  if (kStk)   // stacked B rows past the targets stay zero
    for (int idx = tid; idx < kTiles * kStkBytes / 16; idx += kThreads)
      reinterpret_cast<uint4*>(stk)[idx] = make_uint4(0u, 0u, 0u, 0u);
  // rows beyond `rows` stay zero in every term of both tiles
  for (int idx = tid; idx < kTiles * 3 * kRowsM * (kKst / 8); idx += kThreads) {
    const int tt = idx / (kRowsM * (kKst / 8)), rem = idx - tt * (kRowsM * (kKst / 8));
    const int row = rem / (kKst / 8), c = rem % (kKst / 8);
    if (row >= rows)
      *reinterpret_cast<uint4*>(tiles + tt * kTermBytes + row * 128 + c * 16) = make_uint4(0u, 0u, 0u, 0u);
  }
  fence_proxy_async();
  fence_before();
  __syncthreads();
  fence_after();
  const unsigned tbase = sh.tmem_base;
  if (kStk) {   // every accumulator starts at zero (the MMAs only accumulate)
    if (warp < kDrainWarps) {
      const int lq = warp & 3, half = warp >> 2;
      constexpr int kHalfCols = kAcc * kAccStride / 2;
      for (int c = 0; c < kHalfCols; c += 8)
        tmem_st8_zero(tbase + ((unsigned)(32 * lq) << 16) + (unsigned)(half * kHalfCols + c));
      tmem_st_wait();
    }
    fence_before();
    __syncthreads();
    fence_after();
  }

  if (warp >= kConvWarp0) {
    // ---------------- load + split ----------------
    // Warp cw owns row groups cw and cw + 8 (rows 8 g .. 8 g + 7). Loads: a
    // half warp copies one row's 256 bytes. Split: lane = (row in group,
    // quarter kq) converts positions 8 kq .. 8 kq + 7 and 8 kq + 32 .. + 39.
    // Staging rows past `rows` are never written and stay zero, so they
    // split into the zero rows the tiles need.
    const int cw = warp - kConvWarp0;
    const unsigned stg0 = smem_u32(stg);
    const uint8_t* src[kGroupsPerWarp][4];
    bool ld_ok[kGroupsPerWarp][4];
    unsigned ld_dst[kGroupsPerWarp][4];
    bool grp_ok[kGroupsPerWarp];
#pragma unroll
    for (int gi = 0; gi < kGroupsPerWarp; ++gi) {
      const int g = cw + gi * kConvWarps;
      grp_ok[gi] = 8 * g < rows;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int row = 8 * g + 2 * t + (lane >> 4), ch = lane & 15;
        ld_ok[gi][t] = row < rows;
        src[gi][t] = a.ring + (row < rows ? sh.tab[row] : 0) + 16 * ch;
        ld_dst[gi][t] = (unsigned)(row * kRowBytes + 16 * (ch ^ (row & 7)));
      }
    }
    const int rsub = lane & 7, kq = lane >> 3;
    // first position of this CTA's K-step s (chunks b, b + grid, ...)
    auto step_pos = [&](int64_t s) -> int64_t {
      const int64_t ck = blockIdx.x + (s / kStepsPerChunk) * (int64_t)gridDim.x;
      return (ck * kStepsPerChunk + s % kStepsPerChunk) * kKst;
    };
    auto prefetch_half = [&](int64_t s) {      // K-steps s .. s + 7: 2 KiB of every row
      const int q = cw * 32 + lane;
      if (s < nsteps && q < rows) bulk_prefetch_l2(a.ring + sh.tab[q] + step_pos(s) * 4, 8 * kKst * 4);
    };
    auto load = [&](int64_t s) {
      if (s < nsteps) {
        const int64_t off = step_pos(s) * 4;
        const unsigned dst = stg0 + (unsigned)((s % kSt) * kStageBytes);
#pragma unroll
        for (int gi = 0; gi < kGroupsPerWarp; ++gi)
#pragma unroll
          for (int t = 0; t < 4; ++t)
            if (ld_ok[gi][t]) cp_async16(dst + ld_dst[gi][t], src[gi][t] + off);
      }
      cp_async_commit();                       // one group per K-step, empty past the end
    };
    prefetch_half(0);
    for (int s = 0; s < kSt - 1; ++s) load(s);
    for (int64_t s = 0; s < nsteps && !*stop; ++s) {
      if (s % 8 == 0) prefetch_half(s + 8);
      load(s + kSt - 1);
      cp_async_wait<kSt - 1>();                // this lane's copies of K-step s have landed
      __syncwarp();                            // ... and those of the other lanes
      const int tb = (int)(s % kTiles);
      const bool ok = s < kTiles || mbar_wait(smem_u32(&sh.tile_free[tb]), (unsigned)(((s / kTiles) & 1) ^ 1));
      if (!ok) {
        if (lane == 0) raise_timeout(a.status, stop);
        break;
      }
      const int64_t p0 = step_pos(s);
      const bool tail = p0 + kKst > a.n;       // positions past n contribute nothing
      const uint8_t* sb = stg + (s % kSt) * kStageBytes;
      uint8_t* tile = tiles + tb * kTileBytes;
#pragma unroll
      for (int gi = 0; gi < kGroupsPerWarp; ++gi) {
        if (!grp_ok[gi]) continue;
        const int g = cw + gi * kConvWarps;
        const uint8_t* rp = sb + (8 * g + rsub) * kRowBytes;
        float4 x[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)            // chunks 2 kq, 2 kq + 1, 2 kq + 8, 2 kq + 9 (swizzled)
          x[q] = *reinterpret_cast<const float4*>(rp + 16 * ((2 * kq + (q & 1) + 8 * (q >> 1)) ^ rsub));
        if (tail) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int64_t pos = p0 + 8 * kq + 32 * (q >> 1) + 4 * (q & 1);
            if (pos >= a.n) x[q].x = 0.f;
            if (pos + 1 >= a.n) x[q].y = 0.f;
            if (pos + 2 >= a.n) x[q].z = 0.f;
            if (pos + 3 >= a.n) x[q].w = 0.f;
          }
        }
        uint8_t* trow = tile + (8 * g + rsub) * 128;
#pragma unroll
        for (int h = 0; h < 2; ++h) {          // positions 8 kq .. (h = 0) and 8 kq + 32 .. (h = 1)
          uint4 t0, t1, t2;
          split3(x[2 * h].x, x[2 * h].y, t0.x, t1.x, t2.x);
          split3(x[2 * h].z, x[2 * h].w, t0.y, t1.y, t2.y);
          split3(x[2 * h + 1].x, x[2 * h + 1].y, t0.z, t1.z, t2.z);
          split3(x[2 * h + 1].z, x[2 * h + 1].w, t0.w, t1.w, t2.w);
          uint8_t* cp = trow + 16 * ((kq + 4 * h) ^ rsub);
          *reinterpret_cast<uint4*>(cp) = t0;
          *reinterpret_cast<uint4*>(cp + kTermBytes) = t1;
          *reinterpret_cast<uint4*>(cp + 2 * kTermBytes) = t2;
          if (kStk && 8 * g < kt) {            // a target row: also into the stacked B tile
            // term t's target rows at t * npad * 128 (1024-aligned: the same swizzle phase)
            uint8_t* bp = stk + tb * kStkBytes + (8 * g + rsub) * 128 + 16 * ((kq + 4 * h) ^ rsub);
            *reinterpret_cast<uint4*>(bp) = t0;
            *reinterpret_cast<uint4*>(bp + npad * 128) = t1;
            *reinterpret_cast<uint4*>(bp + 2 * npad * 128) = t2;
          }
        }
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&sh.tile_full[tb]));
    }
    cp_async_wait<0>();
  } else if (warp == kMmaWarp) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      // kind::f16, D f32, A = B = bf16 K-major, M = 128, N = npad
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(npad >> 3) << 17) |
                             ((uint32_t)(kRowsM >> 4) << 24);
      // (A term, B term): the cross terms first, b0 c0 last
      // (A term, B term), smallest first: three terms take all six pairs
      // (i + j <= 2), two terms the last three (i + j <= 1); b0 c0 is last
      constexpr int kPairs = 6;
      const int pa[kPairs] = {1, 2, 0, 1, 0, 0};
      const int pb[kPairs] = {1, 0, 2, 0, 1, 0};
      const int pr0 = (a.split == 2) ? 3 : 0;
      bool ok = true;
      int64_t s = 0;
      for (; s < nsteps; ++s) {
        if (*stop) {
          ok = false;
          break;
        }
        const int tb = (int)(s % kTiles), ac = (int)(s % kAcc);
        ok = mbar_wait(smem_u32(&sh.tile_full[tb]), (unsigned)((s / kTiles) & 1));
        if (!ok) break;
        if (s >= kAcc) {
          ok = mbar_wait(smem_u32(&sh.acc_empty[ac]), (unsigned)(((s / kAcc) & 1) ^ 1));
          if (!ok) break;
        }
        fence_after();
        const unsigned base = smem_u32(tiles + tb * kTileBytes);
        const unsigned dt = tbase + (unsigned)(ac * kAccStride);
        if (kStk) {
          // A term i against the stacked B terms 0 .. G - 1 - i (G = split):
          // smallest products first; every MMA accumulates onto the zeroed groups
          const unsigned sbase = smem_u32(stk + tb * kStkBytes);
          const int G = (a.split == 2) ? 2 : 3;
          for (int i = G - 1; i >= 0; --i) {
            const int nb = G - i;                      // B terms 0 .. nb - 1
            const uint32_t idn = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)((nb * npad) >> 3) << 17) |
                                 ((uint32_t)(kRowsM >> 4) << 24);
#pragma unroll
            for (int ks = 0; ks < kKst / 16; ++ks) {
              const uint64_t da = smem_desc_sw128(base + (unsigned)(i * kTermBytes + ks * 32));
              const uint64_t db = smem_desc_sw128(sbase + (unsigned)(ks * 32));
              mma_f16(dt, da, db, idn, 1u);
            }
          }
        } else {
          int first = 1;
#pragma unroll
          for (int pr = 0; pr < kPairs; ++pr) {
            if (pr < pr0) continue;
#pragma unroll
            for (int ks = 0; ks < kKst / 16; ++ks) {
              const uint64_t da = smem_desc_sw128(base + (unsigned)(pa[pr] * kTermBytes + ks * 32));
              const uint64_t db = smem_desc_sw128(base + (unsigned)(pb[pr] * kTermBytes + ks * 32));
              mma_f16(dt, da, db, idesc, first ? 0u : 1u);
              first = 0;
            }
          }
        }
        mma_commit(smem_u32(&sh.tile_free[tb]));
        mma_commit(smem_u32(&sh.acc_full[ac]));
      }
      if (!ok) raise_timeout(a.status, stop);
      // no MMA may write tensor memory once it is freed
      if (s > 0) mbar_wait(smem_u32(&sh.acc_full[(s - 1) % kAcc]), (unsigned)(((s - 1) / kAcc) & 1));
    }
  } else {
    // ---------------- drain (warps 0..7) ----------------
    const int lq = warp & 3, half = warp >> 2;
    const int cols = npad / 2;                         // multiple of 8, <= 32
    const int col0 = half * cols;
    constexpr int kDc = kStk ? kStkMaxT / 2 : 32;       // target columns per drain warp, at most
    float hi[kDc], lo[kDc];
#pragma unroll
    for (int i = 0; i < kDc; ++i) hi[i] = lo[i] = 0.f;
    for (int64_t s = 0; s < nsteps; ++s) {
      if (*stop) break;
      const int ac = (int)(s % kAcc);
      const bool ok = mbar_wait(smem_u32(&sh.acc_full[ac]), (unsigned)((s / kAcc) & 1));
      if (!ok) {
        if (lane == 0) raise_timeout(a.status, stop);
        break;
      }
      fence_after();
      const unsigned taddr = tbase + ((unsigned)(32 * lq) << 16) + (unsigned)(ac * kAccStride + col0);
#pragma unroll
      for (int pc = 0; pc < kDc / 8; ++pc) {
        if (8 * pc < cols) {
          unsigned v[8];
          tmem_ld8_nowait(taddr + 8 * pc, v);
          tmem_ld_wait();
          if (kStk) {
            // column groups 1 and 2 (B terms 1, 2) of the same targets; then
            // all three back to zero for the accumulator's next use
            unsigned v1[8], v2[8];
            tmem_ld8_nowait(taddr + npad + 8 * pc, v1);
            if (a.split != 2) tmem_ld8_nowait(taddr + 2 * npad + 8 * pc, v2);
            tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const float g12 = (a.split != 2) ? __uint_as_float(v1[i]) + __uint_as_float(v2[i]) : __uint_as_float(v1[i]);
              two_sum_add(hi[8 * pc + i], lo[8 * pc + i], __uint_as_float(v[i]) + g12);
            }
            tmem_st8_zero(taddr + 8 * pc);
            tmem_st8_zero(taddr + npad + 8 * pc);
            if (a.split != 2) tmem_st8_zero(taddr + 2 * npad + 8 * pc);
          } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) two_sum_add(hi[8 * pc + i], lo[8 * pc + i], __uint_as_float(v[i]));
          }
        }
      }
      if (kStk) tmem_st_wait();
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&sh.acc_empty[ac]));
    }
    // this CTA's sums for tile row `row` and targets col0 .. col0 + cols - 1
    const int row = 32 * lq + lane;
    float2* P = a.partials + (int64_t)blockIdx.x * kRowsM * kAccCols;
#pragma unroll
    for (int i = 0; i < kDc; ++i) {
      const int col = col0 + i;
      if (i < cols && row < rows && col < kt) P[(int64_t)row * kAccCols + col] = make_float2(hi[i], lo[i]);
    }
  }
  __syncthreads();
  fence_after();
  __syncwarp();
  if (warp == kMmaWarp) tmem_dealloc(tbase, Lay::kTmem);
}

// G for every tile row i (one block each) and target j (threads): the sum of
// the per-CTA partials in FP64, CTA order fixed. Pairs of two targets are
// taken from the entry with i >= j and written to both G[i][j] and G[j][i].
__global__ void gram_f32_finish_kernel(GramF32Args a, int ctas) {
  const int i = blockIdx.x, kt = a.k;
  const int ti = (i < kt) ? a.t_tgt + i : a.t_old + (i - kt);
  const int pi = (a.start + ti) % a.m;
  for (int j = threadIdx.x; j < kt; j += blockDim.x) {
    if (i < kt && i < j) continue;
    double g = 0.0;
    for (int b = 0; b < ctas; ++b) {
      const float2 v = a.partials[((int64_t)b * kRowsM + i) * kAccCols + j];
      g += (double)v.x + (double)v.y;
    }
    const int pj = (a.start + a.t_tgt + j) % a.m;
    a.G[(int64_t)pi * a.m + pj] = g;
    a.G[(int64_t)pj * a.m + pi] = g;
  }
}

cudaError_t launch_one(const GramF32Args& a, int ctas, cudaStream_t st) {
  if (((a.k + 15) / 16) * 16 <= kStkMaxT)
    gram_f32_tc_kernel<true><<<ctas, kThreads, F32Layout<true>::kBytes, st>>>(a);
  else
    gram_f32_tc_kernel<false><<<ctas, kThreads, F32Layout<false>::kBytes, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  gram_f32_finish_kernel<<<a.k + a.nold, 64, 0, st>>>(a, ctas);
  return cudaGetLastError();
}

}  // namespace

int gram_f32_tc_ctas(int64_t n, int num_sms) {
  const int64_t nchunks = (n + (int64_t)kKst * kStepsPerChunk - 1) / ((int64_t)kKst * kStepsPerChunk);
  int ctas = num_sms < kGramF32MaxCtas ? num_sms : kGramF32MaxCtas;
  if (nchunks < ctas) ctas = (int)nchunks;
  return ctas < 1 ? 1 : ctas;
}

// Targets = window time indices c - k .. c - 1, taken in groups of at most 64
// from the newest; each group is paired with every older snapshot, in blocks
// of 128 - (group size) rows, one launch per block (a group with nothing
// older gets one launch of its own). Pairs inside a group are recomputed by
// each of its launches, with the same result.
cudaError_t launch_gram_f32_tc(const GramF32Args& base, int c, int k, int num_sms, int* launches,
                               cudaStream_t st) {
  if (c < 1 || k < 1 || k > c) return cudaErrorNotSupported;
  {
    cudaError_t e = smem_optin(reinterpret_cast<const void*>(gram_f32_tc_kernel<false>), F32Layout<false>::kBytes);
    if (e == cudaSuccess) e = smem_optin(reinterpret_cast<const void*>(gram_f32_tc_kernel<true>), F32Layout<true>::kBytes);
    if (e != cudaSuccess) return e;
  }
  const int ctas = gram_f32_tc_ctas(base.n, num_sms);
  int count = 0;
  for (int hi = c; hi > c - k;) {
    const int lo = (hi - kGramF32MaxTargets > c - k) ? hi - kGramF32MaxTargets : c - k;
    const int kg = hi - lo;
    const int blk = kRowsM - kg;
    int o = 0;
    do {
      GramF32Args a = base;
      a.t_tgt = lo;
      a.k = kg;
      a.t_old = o;
      a.nold = (lo - o < blk) ? lo - o : blk;
      cudaError_t e = launch_one(a, ctas, st);
      if (e != cudaSuccess) return e;
      ++count;
      o += a.nold;
    } while (o < lo);
    hi = lo;
  }
  if (launches) *launches = count;
  return cudaSuccess;
}

}  // namespace sdmd
