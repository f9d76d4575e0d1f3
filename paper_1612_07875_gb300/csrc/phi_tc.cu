// Exact DMD modes Phi = X' (V Sigma^-1 W) (Sec. 2.2, Eq. 9) for uint8
// snapshots on the 5th-generation tensor cores (tcgen05, accumulators in
// tensor memory).
//
// GEMM shape per tile: D[128 positions x 96] = A[128 x K] * B[K x 96] with
//   A = X' for 128 consecutive positions, K = p window slots padded to 16.
//       Pixels are exact in fp16; A is stored MN-major (positions contiguous,
//       as they are in the ring), so converting a pixel pair takes one byte
//       permute that builds fp16 (1024 + b) and one f16x2 subtraction of 1024.
//   B = the p x 32 real matrix M = V Sigma^-1 W (re/im of 16 modes), each
//       column scaled by a power of two into fp16 range and split into three
//       fp16 terms M0 + M1 + M2 (~33 bits); the terms sit side by side along
//       N, so one MMA per 16 slots reads the A tile once and the epilogue
//       sums the three FP32 column groups. Products b * Mt are exact in FP32.
// Core-matrix layouts (8 rows x 16 bytes, no swizzle): A core (mg, kg) =
// positions 8 mg .. 8 mg + 7 (a row) x slots 8 kg .. 8 kg + 7 (the 8 rows) at
// (kg * 16 + mg) * 128 bytes: 2048 B between K neighbours (leading offset),
// 128 B between position groups (stride offset). B core (ng, kg) is K-major
// at (kg * 12 + ng) * 128 bytes: LBO 1536 B, SBO 128 B.
//
// Scheduling: persistent CTAs take chunks of 8 consecutive tiles from a
// per-pass global counter (atomicAdd), so a CTA that starts late (its SM
// busy with another stream's kernel) just finds less work; the last CTA to
// finish zeroes the counters for the next launch. Tile indices travel from
// the converters to the MMA issuer and the epilogue through a 16-entry ring
// in shared memory, ordered by the same mbarriers as the data; index -1 ends
// every role's loop. Staging rows (128 bytes, one tile) have their 16-byte
// chunks XOR-swizzled by the slot's low three bits (conflict-free copies
// and reads).
//
// Warp roles in a persistent CTA of up to 12 warps (one CTA per SM):
//   warps 5..   load + convert (K / 16, K / 32 or 4 warps: 4, 8 or 16 units
//               per lane per tile). Warp-private units: per tile and step j
//               a warp owns 8 slots x 64 positions; it copies them with
//               cp.async (16 B, L2 only; a quarter warp reads two whole
//               64-byte row pieces, since 16-byte accesses coalesce only
//               within a quarter warp) and, after cp.async.wait_group and
//               __syncwarp, every lane converts one 16-byte chunk of eight
//               different slots, so its A-tile stores hit distinct banks.
//               A tiles go into a ring of up to 4 buffers;
//   warp 4      lane 0 issues the K/16 MMAs of a tile into one of four TMEM
//               accumulators and commits them to mbarriers;
//   warps 0..3  epilogue: tcgen05.ld of their 32 TMEM lanes, sum and scale,
//               complex64 stores of Phi (coalesced per mode).
// The A and accumulator rings are deep because a tile is small: the
// hand-offs between the roles take longer than the work of one tile.
// Every mbarrier wait is bounded (about one second): on expiry the kernel
// raises kDevTimeout, every role stops at its next step, the converters
// drain their copies in flight, the MMA issuer waits (bounded) for its last
// commit, and the tensor memory is freed before exit.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sdmd_internal.cuh"
#include "tc_util.cuh"

namespace sdmd {

namespace {

using namespace tc;

constexpr int kEpiWarps = 4;         // warps 0..3
constexpr int kMmaWarp = 4;
constexpr int kConvWarp0 = 5;        // converter warps 5 .. 5 + K / (4 kIpt) - 1
constexpr int kMaxThreads = 32 * (kConvWarp0 + 7);
constexpr int kTileM = 128;          // positions per tile (MMA M)
constexpr int kMaxModes = 16;        // modes per pass, at most (gridDim.y covers r)
constexpr int kMaxCols = 2 * kMaxModes;
constexpr int kSplits = 3;
constexpr int kMaxN = kSplits * kMaxCols;   // 96 accumulator columns per tile, at most
// A pass of kMd modes: 2 kMd re/im columns per fp16 term, the three terms
// side by side along N, N rounded up to a multiple of 16 (kMd = 10: N = 64)
template <int kMd>
struct PassShape {
  static constexpr int kCols = 2 * kMd;
  static constexpr int kN = ((kSplits * kCols + 15) / 16) * 16;
  static constexpr int kLoad = ((kN + 31) / 32) * 32;   // tensor-memory columns read per tile
};
constexpr int kAcc = 4;              // TMEM accumulators (ring)
constexpr int kMaxA = 4;             // A-tile buffers (ring)
constexpr int kTmemCols = 512;       // kAcc x kN <= 384, power of two
constexpr int kMaxRows = 256;        // K padded (p <= 255)
constexpr int kChunk = 8;            // tiles per scheduling grab
constexpr int kTix = 16;             // tile-index ring

// Instruction descriptor, kind::f16: D f32, A and B f16, A MN-major, B K-major.
__host__ __device__ constexpr uint32_t idesc_f16_amn(int M, int N) {
  return (1u << 4)                 // D format: f32
         | (0u << 7)               // A format: f16
         | (0u << 10)              // B format: f16
         | (1u << 15)              // A major: MN
         | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Two pixels (bytes `sel` of w) -> f16x2 (b0, b1): the permute builds the
// fp16 bit patterns 0x64bb = 1024 + b (exact: the ulp at 1024 is 1), and
// the subtraction of 1024 is exact.
__device__ __forceinline__ unsigned f16x2_of_bytes(unsigned w, unsigned sel) {
  const unsigned t = __byte_perm(w, 0x64u, sel);
  unsigned d;
  asm("sub.rn.f16x2 %0, %1, %2;\n" : "=r"(d) : "r"(t), "r"(0x64006400u));
  return d;
}

struct TcShared {
  unsigned long long a_full[kMaxA];       // A buffer converted
  unsigned long long a_free[kMaxA];       // MMAs reading the A buffer done
  unsigned long long acc_full[kAcc];      // accumulator complete (MMA commit + issuer's release)
  unsigned long long acc_empty[kAcc];     // accumulator drained
  unsigned tmem_base;
  int stop;
  unsigned long long chunk_bar[2];        // chunk start published (by chunk parity)
  int chunk[2];                           // tile chunks grabbed by the converter leader (by parity)
  int tix[kTix];                          // tile index of iteration it at it % kTix, -1: no more
  int expo[kMaxCols];                     // per-column power-of-two scaling of M
};

// Dynamic shared memory: A ring, B, staging ring, slot offsets, state.
struct TcLayout {
  int a_bytes, b_off, b_bytes, st_off, st_bytes, tab_off, xn_off, gs_off, sh_off, total;
};

constexpr int kMaxConvWarps = 7;

// kb: 128-position MMA blocks per tile (a tile is what one iteration of the
// roles hands on: its A buffer holds kb blocks, its staging rows kb x 128
// bytes). fuse: add a private copy of the new snapshot's tile per converter
// warp and stage and the CTA's Gram sums
__host__ __device__ inline TcLayout tc_layout(int kpad, int n_a, int stages, int fuse = 0, int kb = 1) {
  TcLayout L;
  L.a_bytes = kb * kTileM * kpad * 2;            // multiple of 4096
  L.b_off = n_a * L.a_bytes;
  L.b_bytes = kMaxN * kpad * 2;                  // multiple of 3072 (room for 16 modes)
  L.st_off = L.b_off + L.b_bytes;                // 16-byte aligned (cp.async destination)
  L.st_bytes = kpad * kTileM * kb;
  L.tab_off = L.st_off + stages * L.st_bytes;    // window slot offsets (int64)
  L.xn_off = L.tab_off + kMaxRows * 8;
  L.gs_off = L.xn_off + (fuse ? stages * kMaxConvWarps * kTileM * kb : 0);
  L.sh_off = L.gs_off + (fuse ? kMaxRows * 8 : 0);
  L.total = L.sh_off + (int)sizeof(TcShared);
  return L;
}

// Position in a ring of `size` buffers and the parity of the current use.
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

__device__ __forceinline__ void raise_timeout(const PhiArgs& a, volatile int* stop) {
  atomicOr(a.status, kDevTimeout);
  *stop = 1;
}

template <int kIpt, int kMd, int kB>
__global__ void __launch_bounds__(kMaxThreads, 1) phi_tc_u8_kernel(PhiArgs a, int kpad, int n_a, int stages) {
  constexpr int kT = kB * kTileM;        // positions per tile (kB MMA blocks)
  constexpr int kU = kT;                 // staging row bytes
  constexpr int kSeg = 2 * kB;           // 64-position segments per tile
  constexpr int kCols = PassShape<kMd>::kCols;
  constexpr int kN = PassShape<kMd>::kN;
  constexpr int kAccT = (kB * kN * 4 <= kTmemCols) ? 4 : 2;   // accumulator sets (kB x kN columns each)
  constexpr int kChunkT = kChunk / kB;   // tiles per scheduling grab (1024 positions)
  extern __shared__ __align__(1024) uint8_t smem[];
  const TcLayout L = tc_layout(kpad, n_a, stages, a.fuse, kB);
  const int a_blk = kTileM * kpad * 2;   // one block of an A buffer
  // fused Gram row: only the first mode pass computes it
  const bool dots = a.fuse && blockIdx.y == 0;
  const int krows = dots ? a.ktot : a.p;  // staged rows
  unsigned long long* gsum = reinterpret_cast<unsigned long long*>(smem + L.gs_off);
  uint8_t* abuf = smem;
  uint8_t* bbuf = smem + L.b_off;
  uint8_t* stg = smem + L.st_off;
  int64_t* tab = reinterpret_cast<int64_t*>(smem + L.tab_off);
  TcShared& sh = *reinterpret_cast<TcShared*>(smem + L.sh_off);
  volatile int* stop = &sh.stop;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nthreads = blockDim.x;
  const int conv_warps = (nthreads >> 5) - kConvWarp0;   // = kpad kB / (4 kIpt)
  const int k0 = blockIdx.y * kMd;
  const int nks = kpad / 16;
  const int ntiles = (int)((a.n + kT - 1) / kT);

  if (tid == 0) {
    for (int b = 0; b < kMaxA; ++b) {
      mbar_init(smem_u32(&sh.a_full[b]), (unsigned)conv_warps);
      mbar_init(smem_u32(&sh.a_free[b]), 1);
    }
    for (int b = 0; b < 2; ++b) mbar_init(smem_u32(&sh.chunk_bar[b]), 1);
    for (int b = 0; b < kAccT; ++b) {
      mbar_init(smem_u32(&sh.acc_full[b]), 2);
      mbar_init(smem_u32(&sh.acc_empty[b]), kEpiWarps);
    }
    sh.stop = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&sh.tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  for (int q = tid; q < krows; q += nthreads) tab[q] = (int64_t)((a.start + 1 + q) % a.m) * a.slot_bytes;
  if (dots)
    for (int q = tid; q < kMaxRows; q += nthreads) gsum[q] = 0ull;
  if (tid < kCols) {
    // column scale: the largest |M| of the column lands in [2^14, 2^15)
    const int mode = k0 + tid / 2;
    float mx = 0.f;
    if (mode < a.r)
      for (int k = 0; k < a.p; ++k) mx = fmaxf(mx, fabsf(a.Mf[(int64_t)k * 2 * a.r + 2 * mode + (tid & 1)]));
    int e = 0;
    if (mx > 0.f) {
      int ex;
      frexpf(mx, &ex);
      e = 15 - ex;
    }
    sh.expo[tid] = e;
  }
  // B columns past the three terms (kMd = 10: 60 .. 63) are zero
  for (int idx = tid; idx < (kN - kSplits * kCols) * kpad; idx += nthreads) {
    const int nn = kSplits * kCols + idx / kpad, k = idx % kpad;
    *reinterpret_cast<unsigned short*>(bbuf + ((k >> 3) * (kN / 8) + (nn >> 3)) * 128 + (nn & 7) * 16 + (k & 7) * 2) = 0;
  }
  __syncthreads();
  // B: three fp16 terms of the scaled M, K-major cores, zero padded
  for (int idx = tid; idx < kCols * kpad; idx += nthreads) {
    const int c = idx / kpad, k = idx - c * kpad;
    const int mode = k0 + c / 2;
    float x = 0.f;
    if (k < a.p && mode < a.r) x = ldexpf(a.Mf[(int64_t)k * 2 * a.r + 2 * mode + (c & 1)], sh.expo[c]);
    const __half h0 = __float2half_rn(x);
    const float r1 = x - __half2float(h0);          // exact
    const __half h1 = __float2half_rn(r1);
    const float r2 = r1 - __half2float(h1);         // exact
    const __half h2 = __float2half_rn(r2);
    const unsigned short hs[kSplits] = {__half_as_ushort(h0), __half_as_ushort(h1), __half_as_ushort(h2)};
#pragma unroll
    for (int t = 0; t < kSplits; ++t) {
      const int nn = t * kCols + c;
      const int off = ((k >> 3) * (kN / 8) + (nn >> 3)) * 128 + (nn & 7) * 16 + (k & 7) * 2;
      *reinterpret_cast<unsigned short*>(bbuf + off) = hs[t];
    }
  }
  fence_proxy_async();
  fence_before();
  __syncthreads();
  fence_after();
  const unsigned tbase = sh.tmem_base;

  if (warp >= kConvWarp0) {
    // ---------------- load + convert ----------------
    // step j of converter warp cw covers u = cw + conv_warps j: slot group
    // kg = u / kSeg (slots 8 kg .. 8 kg + 7) and positions 64 h .. 64 h + 63
    // (h = u % kSeg) of a tile; every (kg, h) is covered exactly once.
    // Staging rows hold the tile's kU bytes of a slot in 16-byte chunks;
    // within each 128-byte half the chunk index is XORed with the slot's low
    // three bits (conflict-free copies and reads)
    const int cw = warp - kConvWarp0;
    int64_t src[kIpt];                      // copy source in the ring (without tile)
    unsigned ldo[kIpt];                     // copy destination in a stage (first tile's segment)
    unsigned sto[kIpt], ao[kIpt];           // conversion source in a stage, A-tile destination
#pragma unroll
    for (int j = 0; j < kIpt; ++j) {
      const int u = cw + conv_warps * j;
      const int kg = u / kSeg, h = u % kSeg;
      // copy: lane -> slot 8 kg + lr, chunk pl (a quarter warp: slots r and r + 4, 4 chunks each)
      const int lr = (lane >> 3) + 4 * ((lane >> 2) & 1), pl = 4 * h + (lane & 3);
      const int ql = 8 * kg + lr;
      // rows past the staged ones (K padding) copy the last staged row's bytes
      // again (L2 hits: the same tile reads that row), so every lane issues
      // the same copies with no branch; B is zero on those rows and their
      // dots are dropped
      src[j] = tab[(ql < krows) ? ql : krows - 1] + 16 * pl;
      ldo[j] = (unsigned)(ql * kU + 16 * ((pl & ~7) | ((pl & 7) ^ lr)));
      // conversion: lane -> slot 8 kg + kr, chunk pc (a quarter warp: 8 slots, one chunk)
      const int kr = lane & 7, pc = 4 * h + (lane >> 3);
      sto[j] = (unsigned)((8 * kg + kr) * kU + 16 * ((pc & ~7) | ((pc & 7) ^ kr)));
      // block pc / 8 of the A buffer, core (2 (pc % 8), kg), row kr
      ao[j] = (unsigned)((pc >> 3) * a_blk + (kg * 16 + 2 * (pc & 7)) * 128 + kr * 16);
    }
    // tile sequence: chunk c (iterations 8 c .. 8 c + 7 of this CTA) starts
    // at the tile index the leader grabbed and published through chunk_bar
    // (by chunk parity: the A ring keeps every converter warp within a few
    // tiles of the leader, so a slot is rewritten only after all have read
    // it); an index is fixed when its copies are issued, kStages - 1
    // iterations before the tile is converted
    const int ct = tid - 32 * kConvWarp0;
    int ld_count = 0;                        // tiles whose index is fixed
    bool ended = false;                      // an index past the last tile was seen
    int nvalid = 0;                          // (once ended) iterations 0 .. nvalid - 1 have tiles
    int cbase = 0;                           // start of the chunk being fixed
    auto fix_next = [&]() -> int {           // all converter threads, in step
      int t = -1;
      if (!ended) {
        const int c = ld_count / kChunkT, o = ld_count % kChunkT;
        if (o == 0) {
          const unsigned bar = smem_u32(&sh.chunk_bar[c & 1]);
          if (ct == 0) {
            sh.chunk[c & 1] = (int)atomicAdd(&a.sched[blockIdx.y], (unsigned)kChunkT);
            mbar_arrive(bar);
          }
          int ok = 1;
          if (lane == 0) ok = mbar_wait(bar, (unsigned)((c >> 1) & 1));
          ok = __shfl_sync(0xffffffffu, ok, 0);
          __syncwarp();
          if (ok) {
            cbase = sh.chunk[c & 1];
          } else {
            if (lane == 0) raise_timeout(a, stop);
            cbase = ntiles;                  // end the sequence here
          }
        }
        t = cbase + o;
        if (t >= ntiles) {
          t = -1;
          ended = true;
          nvalid = ld_count;
        }
      }
      if (ct == 0) sh.tix[ld_count % kTix] = t;
      ++ld_count;
      return t;
    };
    const unsigned stg0 = smem_u32(stg);
    // fused Gram row: this warp's private copy of the new snapshot's tile
    // (lanes 0 .. 8 kB - 1, 16 bytes each) per stage, and per step j the exact sum of
    // <x_slot, x_new> over this lane's 16 positions (computed for every lane,
    // branch-free, in two independent DP4A chains; lanes whose slot is not in
    // the new window drop their sums at the end)
    uint8_t* xnw = smem + L.xn_off + cw * kT;           // stage s at + s * kMaxConvWarps * kT
    const int64_t xsrc = dots ? tab[a.ktot - 1] + 16 * (lane & (8 * kB - 1)) : 0;
    unsigned long long gacc[kIpt];
    bool gslot[kIpt];
#pragma unroll
    for (int j = 0; j < kIpt; ++j) {
      gacc[j] = 0ull;
      const int u = cw + conv_warps * j;
      const int sl = 8 * (u / kSeg) + (lane & 7);
      gslot[j] = dots && sl >= a.g0 && sl < a.ktot;
    }
    int ld_stage = 0;
    auto load_next = [&]() {
      const int t = fix_next();
      if (t >= 0) {
        const unsigned dst = stg0 + (unsigned)(ld_stage * L.st_bytes);
        const uint8_t* tsrc = a.ring + (int64_t)t * kT;
#pragma unroll
        for (int j = 0; j < kIpt; ++j)
          cp_async16(dst + ldo[j], tsrc + src[j]);
        if (dots && lane < 8 * kB)
          cp_async16(smem_u32(xnw + ld_stage * kMaxConvWarps * kT + 16 * lane), tsrc + xsrc);
      }
      ld_stage = (ld_stage + 1 == stages) ? 0 : ld_stage + 1;
    };
    for (int st = 0; st < stages - 1; ++st) {
      load_next();
      cp_async_commit();
    }
    int stage = 0;
    Ring ab;                                 // A buffer of the current tile
    for (int it = 0; !*stop; ++it) {
      const bool valid = !(ended && it >= nvalid);   // tile `it` exists
      load_next();
      cp_async_commit();
      cp_async_wait_pending(stages - 1);     // this lane's copies of tile `it` have landed
      __syncwarp();                          // ... and those of the other lanes of the warp
      const uint8_t* sb = stg + stage * L.st_bytes;
      const uint8_t* xb = xnw + stage * kMaxConvWarps * kT;
      stage = (stage + 1 == stages) ? 0 : stage + 1;
      {
        int ok = 1;
        if (lane == 0 && it >= n_a) ok = mbar_wait(smem_u32(&sh.a_free[ab.idx]), ab.phase ^ 1u);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          if (lane == 0) raise_timeout(a, stop);
          break;
        }
        if (!valid) {                        // past the last tile: hand the end on and stop
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&sh.a_full[ab.idx]));
          break;
        }
        uint8_t* abt = abuf + (size_t)ab.idx * L.a_bytes;
        uint4 w[kIpt];
#pragma unroll
        for (int j = 0; j < kIpt; ++j) w[j] = *reinterpret_cast<const uint4*>(sb + sto[j]);
        if (dots) {
          const uint8_t* xl = xb + 16 * (lane >> 3);
#pragma unroll
          for (int j = 0; j < kIpt; ++j) {
            const uint4 xv = *reinterpret_cast<const uint4*>(xl + 64 * ((cw + conv_warps * j) % kSeg));
            unsigned d0 = __dp4a(w[j].x, xv.x, 0u);
            unsigned d1 = __dp4a(w[j].y, xv.y, 0u);
            d0 = __dp4a(w[j].z, xv.z, d0);
            d1 = __dp4a(w[j].w, xv.w, d1);
            gacc[j] += (unsigned long long)(d0 + d1);
          }
        }
#pragma unroll
        for (int j = 0; j < kIpt; ++j) {
          uint4 lo, hi;
          lo.x = f16x2_of_bytes(w[j].x, 0x4140u);
          lo.y = f16x2_of_bytes(w[j].x, 0x4342u);
          lo.z = f16x2_of_bytes(w[j].y, 0x4140u);
          lo.w = f16x2_of_bytes(w[j].y, 0x4342u);
          hi.x = f16x2_of_bytes(w[j].z, 0x4140u);
          hi.y = f16x2_of_bytes(w[j].z, 0x4342u);
          hi.z = f16x2_of_bytes(w[j].w, 0x4140u);
          hi.w = f16x2_of_bytes(w[j].w, 0x4342u);
          *reinterpret_cast<uint4*>(abt + ao[j]) = lo;
          *reinterpret_cast<uint4*>(abt + ao[j] + 128) = hi;
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&sh.a_full[ab.idx]));
        ab.next(n_a);
      }
    }
    cp_async_wait<0>();                      // no copy lands after the CTA exits
    if (dots) {                              // lanes kr, kr + 8, kr + 16, kr + 24 share a slot
#pragma unroll
      for (int j = 0; j < kIpt; ++j) {
        unsigned long long v = gacc[j];
        v += __shfl_xor_sync(0xffffffffu, v, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 16);
        if (lane < 8 && gslot[j]) atomicAdd(&gsum[8 * ((cw + conv_warps * j) / kSeg) + lane], v);
      }
    }
  } else if (warp == kMmaWarp) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = idesc_f16_amn(kTileM, kN);
      // K step ks advances A by 4096 bytes and B by 2 (kN / 8) 128 bytes: the
      // descriptors' start-address field (bytes / 16) by 256 and by 16 kN / 8
      const uint64_t bd0 = smem_desc(smem_u32(bbuf), (kN / 8) * 128u, 128u);
      constexpr uint64_t kBStep = 2u * (kN / 8) * 128u / 16u;
      Ring ab, acc, last;
      int issued = 0;
      for (int it = 0;; ++it) {
        if (*stop) break;
        bool ok = mbar_wait(smem_u32(&sh.a_full[ab.idx]), ab.phase);
        if (ok && it >= kAccT) ok = mbar_wait(smem_u32(&sh.acc_empty[acc.idx]), acc.phase ^ 1u);
        if (!ok) {
          raise_timeout(a, stop);
          break;
        }
        if (sh.tix[it % kTix] < 0) {         // no more tiles: hand the end to the epilogue
          mbar_arrive2(smem_u32(&sh.acc_full[acc.idx]));
          break;
        }
        fence_after();
        const unsigned abase = smem_u32(abuf + (size_t)ab.idx * L.a_bytes);
#pragma unroll
        for (int blk = 0; blk < kB; ++blk) {   // block blk of the tile into accumulator columns (acc, blk)
          const uint64_t ad0 = smem_desc(abase + (unsigned)(blk * a_blk), 2048u, 128u);
          const unsigned dt = tbase + (unsigned)((acc.idx * kB + blk) * kN);
          mma_f16(dt, ad0, bd0, idesc, 0u);
          for (int ks = 1; ks < nks; ++ks) mma_f16(dt, ad0 + 256u * ks, bd0 + kBStep * ks, idesc, 1u);
        }
        mma_commit(smem_u32(&sh.a_free[ab.idx]));
        mma_commit(smem_u32(&sh.acc_full[acc.idx]));
        mbar_arrive(smem_u32(&sh.acc_full[acc.idx]));   // release: the epilogue sees tix[]
        issued = it + 1;
        last = acc;
        ab.next(n_a);
        acc.next(kAccT);
      }
      // no MMA may still write tensor memory when it is freed
      if (issued > 0) mbar_wait(smem_u32(&sh.acc_full[last.idx]), last.phase);
    }
  } else {
    // ---------------- epilogue (warps 0..3 own TMEM lanes 32w .. 32w + 31) ----------------
    float sc[kCols];
#pragma unroll
    for (int c = 0; c < kCols; ++c) sc[c] = ldexpf(1.f, -sh.expo[c]);
    float2* out = reinterpret_cast<float2*>(a.phi) + (int64_t)k0 * a.n;
    const int nq = (a.r - k0 < kMd) ? a.r - k0 : kMd;      // modes of this pass
    Ring acc;
    for (int it = 0;; ++it) {
      if (*stop) break;
      int ok = 1;
      if (lane == 0) ok = mbar_wait(smem_u32(&sh.acc_full[acc.idx]), acc.phase);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) raise_timeout(a, stop);
        break;
      }
      const int t = sh.tix[it % kTix];
      if (t < 0) break;                      // no more tiles
      fence_after();
#pragma unroll 1
      for (int blk = 0; blk < kB; ++blk) {   // the tile's blocks one after the other
        const int64_t i = (int64_t)t * kT + blk * kTileM + 32 * warp + lane;
        unsigned v[PassShape<kMd>::kLoad];
        const unsigned taddr = tbase + ((unsigned)(32 * warp) << 16) + (unsigned)((acc.idx * kB + blk) * kN);
        if constexpr (PassShape<kMd>::kLoad == 64)
          tmem_ld64_wait(taddr, v);
        else
          tmem_ld96_wait(taddr, v);
        if (blk + 1 == kB) {                 // every block of the set read: hand it back
          fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&sh.acc_empty[acc.idx]));
        }
        if (i < a.n) {
          float2* o = out + i;
#pragma unroll
          for (int q = 0; q < kMd; ++q) {
            if (nq == kMd || q < nq) {
              const float re = (__uint_as_float(v[2 * q]) + __uint_as_float(v[kCols + 2 * q])) +
                               __uint_as_float(v[2 * kCols + 2 * q]);
              const float im = (__uint_as_float(v[2 * q + 1]) + __uint_as_float(v[kCols + 2 * q + 1])) +
                               __uint_as_float(v[2 * kCols + 2 * q + 1]);
              *o = make_float2(re * sc[2 * q], im * sc[2 * q + 1]);
            }
            o += a.n;
          }
        }
      }
      acc.next(kAccT);
    }
  }
  __syncthreads();
  fence_after();
  __syncwarp();
  if (warp == kMmaWarp)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tbase), "r"(kTmemCols) : "memory");
  if (dots)                                  // this CTA's sums (every CTA writes all of them)
    for (int q = a.g0 + tid; q < a.ktot; q += nthreads)
      a.gpart[(int64_t)(q - a.g0) * kFusedMaxCtas + blockIdx.x] = (long long)gsum[q];
  // the last CTA out (all grabs are done) zeroes the counters for the next launch
  if (tid == 0) {
    __threadfence();
    const unsigned total = gridDim.x * gridDim.y;
    if (atomicAdd(&a.sched[kPhiSchedPasses], 1u) == total - 1u) {
      for (unsigned y = 0; y < gridDim.y; ++y) a.sched[y] = 0u;
      a.sched[kPhiSchedPasses] = 0u;
      __threadfence();
    }
  }
}

template <int kIpt, int kMd, int kB>
cudaError_t launch_cfg(const PhiArgs& a, cudaStream_t st, int kpad, int n_a, int stages, size_t smem, int* ctas) {
  {
    const cudaError_t e = smem_optin(reinterpret_cast<const void*>(phi_tc_u8_kernel<kIpt, kMd, kB>), smem);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms < 1) sms = 1;
  const int64_t ntiles = (a.n + kB * kTileM - 1) / (kB * kTileM);
  const int ky = (a.r + kMd - 1) / kMd;
  int64_t bx = ((int64_t)sms + ky - 1) / ky;
  if (bx > ntiles) bx = ntiles;
  if (bx < 1) bx = 1;
  if (a.fuse && bx > kFusedMaxCtas) bx = kFusedMaxCtas;
  // the fused pass runs beside the other frames' eigensolvers (one whole SM
  // each, about 1.1 ms per 0.29 ms step: four at a time); leaving them their
  // SMs measured 264 instead of 271 us per pass
  if (a.fuse && bx > sms - kFusedReserveSms && sms - kFusedReserveSms >= 1) bx = sms - kFusedReserveSms;
  const int threads = 32 * (kConvWarp0 + kpad * kB / (4 * kIpt));
  phi_tc_u8_kernel<kIpt, kMd, kB><<<dim3((unsigned)bx, (unsigned)ky), threads, smem, st>>>(a, kpad, n_a, stages);
  if (ctas) *ctas = (int)bx;
  return cudaGetLastError();
}

// one pass of 10 modes when r <= 10 (N = 64), else passes of 16 (N = 96)
template <int kIpt, int kB>
cudaError_t launch_modes(const PhiArgs& a, cudaStream_t st, int kpad, int n_a, int stages, size_t smem, int* ctas) {
  if (a.fit_modes && a.r <= 10) return launch_cfg<kIpt, 10, kB>(a, st, kpad, n_a, stages, smem, ctas);
  return launch_cfg<kIpt, 16, kB>(a, st, kpad, n_a, stages, smem, ctas);
}

// G's new row and column from the per-CTA sums (exact int64): one block per
// window slot jj, its CTA sums contiguous at gpart + jj * kFusedMaxCtas
__global__ void __launch_bounds__(128) fused_gram_finish_kernel(const long long* gpart, int ctas, long long* G, int gm,
                                                                 int s_new, int slot0) {
  __shared__ long long red[4];
  const int jj = blockIdx.x;
  long long s = 0;
  for (int b = threadIdx.x; b < ctas; b += blockDim.x) s += gpart[(int64_t)jj * kFusedMaxCtas + b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    const long long v = red[0] + red[1] + red[2] + red[3];
    const int j = (slot0 + jj) % gm;
    G[(int64_t)s_new * gm + j] = v;
    G[(int64_t)j * gm + s_new] = v;
  }
}

cudaError_t launch_phi_tc_impl(const PhiArgs& a, cudaStream_t st, int* ctas) {
  if (a.dtype != SDMD_U8 || a.p < 1 || a.p >= kMaxRows || a.sched == nullptr) return cudaErrorNotSupported;
  const int rows = a.fuse ? a.ktot : a.p;
  if (a.fuse && (rows >= kMaxRows || a.g0 < 0 || a.g0 >= rows || a.gpart == nullptr)) return cudaErrorNotSupported;
  // K padding and units per converter lane, at most 7 converter warps:
  // K <= 112: 4 units (K / 16 warps); K <= 224: K to a multiple of 32 and
  // 8 units (K / 32 warps); else K = 256 and 16 units (4 warps)
  int kpad = ((rows + 15) / 16) * 16, ipt = 4;
  if (kpad > 112) {
    kpad = ((rows + 31) / 32) * 32;
    ipt = 8;
    if (kpad > 224) {
      kpad = 256;
      ipt = 16;
    }
  }
  const int kLimit = 227 * 1024;
  // at least 116 KiB of shared memory: one of these CTAs per SM, so its 512
  // tensor-memory columns are always free
  auto smem_of = [](const TcLayout& L) { return L.total < 116 * 1024 ? (size_t)116 * 1024 : (size_t)L.total; };
  // K <= 112 with fitted shapes: tiles of two 128-position blocks (every
  // role hands on 256 positions at a time, eight units per converter lane,
  // the same converter warps), when two A buffers and three stages fit
  if (ipt == 4 && a.fit_modes) {
    static const int kConfigs2[][2] = {{2, 4}, {2, 3}};
    for (const auto& cf : kConfigs2) {
      const TcLayout L = tc_layout(kpad, cf[0], cf[1], a.fuse, 2);
      if (L.total > kLimit) continue;
      return launch_modes<8, 2>(a, st, kpad, cf[0], cf[1], smem_of(L), ctas);
    }
  }
  // deepest A ring first, then the deepest staging ring, within 227 KiB
  static const int kConfigs[][2] = {{4, 6}, {4, 5}, {4, 4}, {3, 5}, {3, 4}, {2, 6}, {2, 4}, {2, 3}, {1, 4}, {1, 3}};
  for (const auto& cf : kConfigs) {
    const TcLayout L = tc_layout(kpad, cf[0], cf[1], a.fuse);
    if (L.total > kLimit) continue;
    if (ipt == 4) return launch_modes<4, 1>(a, st, kpad, cf[0], cf[1], smem_of(L), ctas);
    if (ipt == 8) return launch_modes<8, 1>(a, st, kpad, cf[0], cf[1], smem_of(L), ctas);
    return launch_modes<16, 1>(a, st, kpad, cf[0], cf[1], smem_of(L), ctas);
  }
  return cudaErrorNotSupported;
}

}  // namespace

// Tensor-core Phi for uint8 windows. Returns cudaErrorNotSupported when the
// shape is outside what this kernel handles (the caller then uses the SIMT
// kernel).
cudaError_t launch_phi_tc(const PhiArgs& a, cudaStream_t st) {
  PhiArgs b = a;
  b.fuse = 0;
  return launch_phi_tc_impl(b, st, nullptr);
}

cudaError_t launch_phi_fused(const PhiArgs& a, long long* G, int32_t gm, int32_t s_new, int32_t slot0,
                             cudaStream_t st) {
  if (!a.fuse) return cudaErrorInvalidValue;
  int ctas = 0;
  cudaError_t e = launch_phi_tc_impl(a, st, &ctas);
  if (e != cudaSuccess) return e;
  fused_gram_finish_kernel<<<a.ktot - a.g0, 128, 0, st>>>(a.gpart, ctas, G, gm, s_new, slot0);
  return cudaGetLastError();
}

}  // namespace sdmd
