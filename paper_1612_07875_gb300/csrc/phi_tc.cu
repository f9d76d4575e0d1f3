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
// Warp roles in a persistent CTA of 9 warps (one CTA per SM):
//   warps 4..7  load + convert: each thread owns fixed 16-byte chunks of the
//               tile (one window slot x 16 positions) and streams them with
//               cp.async (16 B, L2 only) through a private 4-deep staging
//               ring (row pitch 144 B: the 16-byte reads of eight consecutive
//               slots by a quarter warp hit distinct banks); it converts only
//               chunks it loaded itself, so stages need no barrier, then
//               writes the fp16 A tile (double-buffered);
//   warp 8      lane 0 issues the K/16 MMAs of a tile into one of two TMEM
//               accumulators and commits them to mbarriers;
//   warps 0..3  epilogue: tcgen05.ld of their 32 TMEM lanes, sum and scale,
//               complex64 stores of Phi (coalesced per mode).
// Every mbarrier wait is bounded (about one second): on expiry the kernel
// raises kDevTimeout, every role stops at its next step, the converters
// drain their copies in flight, the MMA issuer waits (bounded) for its last
// commit, and the tensor memory is freed before exit.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sdmd_internal.cuh"

namespace sdmd {

namespace {

constexpr int kEpiWarps = 4;         // warps 0..3
constexpr int kMmaWarp = 4;
constexpr int kConvWarp0 = 5;        // converter warps 5 .. 5 + K / (4 kIpt) - 1
constexpr int kMaxThreads = 32 * (kConvWarp0 + 7);
constexpr int kTileM = 128;          // positions per tile (MMA M)
constexpr int kModes = 16;           // modes per pass (gridDim.y covers r)
constexpr int kCols = 2 * kModes;    // re/im columns of one fp16 term
constexpr int kSplits = 3;
constexpr int kN = kSplits * kCols;  // 96 accumulator columns per tile
constexpr int kTmemCols = 256;       // two accumulators, power of two
constexpr int kPitch = 144;          // staging row pitch, bytes
constexpr int kMaxRows = 256;        // K padded (p <= 255)
constexpr long long kWaitCycles = 2000000000LL;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
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

__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

__device__ __forceinline__ void cp_async16(unsigned dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// tcgen05 shared-memory matrix descriptor, no swizzle: `lbo` is the byte
// distance between core matrices adjacent along K, `sbo` along M or N.
__device__ __forceinline__ uint64_t smem_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;          // descriptor version of the tcgen05 family
  return d;
}

// Instruction descriptor, kind::f16: D f32, A and B f16, A MN-major, B K-major.
__host__ __device__ constexpr uint32_t idesc_f16_amn(int M, int N) {
  return (1u << 4)                 // D format: f32
         | (0u << 7)               // A format: f16
         | (0u << 10)              // B format: f16
         | (1u << 15)              // A major: MN
         | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(unsigned dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        unsigned accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(unsigned mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld32_nowait(unsigned taddr, unsigned (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

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
  unsigned long long a_full[2];           // A buffer converted
  unsigned long long a_free[2];           // MMAs reading the A buffer done
  unsigned long long acc_full[2];         // accumulator complete
  unsigned long long acc_empty[2];        // accumulator drained
  unsigned tmem_base;
  int stop;
  int expo[kCols];                        // per-column power-of-two scaling of M
};

struct TcLayout {
  int a_bytes, b_off, b_bytes, st_off, st_bytes, tab_off, sh_off, total;
};

__host__ __device__ inline TcLayout tc_layout(int kpad, int n_a, int stages) {
  TcLayout L;
  L.a_bytes = kTileM * kpad * 2;                 // multiple of 4096
  L.b_off = n_a * L.a_bytes;
  L.b_bytes = kN * kpad * 2;                     // multiple of 3072
  L.st_off = L.b_off + L.b_bytes;                // 16-byte aligned (bulk copy destination)
  L.st_bytes = kpad * kPitch;
  L.tab_off = L.st_off + stages * L.st_bytes;    // window slot offsets (int64)
  L.sh_off = L.tab_off + kMaxRows * 8;
  L.total = L.sh_off + (int)sizeof(TcShared);
  return L;
}

template <int kStages, int kIpt>
__global__ void __launch_bounds__(kMaxThreads, 1) phi_tc_u8_kernel(PhiArgs a, int kpad, int n_a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const TcLayout L = tc_layout(kpad, n_a, kStages);
  uint8_t* abuf = smem;
  uint8_t* bbuf = smem + L.b_off;
  uint8_t* stg = smem + L.st_off;
  int64_t* tab = reinterpret_cast<int64_t*>(smem + L.tab_off);
  TcShared& sh = *reinterpret_cast<TcShared*>(smem + L.sh_off);
  volatile int* stop = &sh.stop;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nthreads = blockDim.x;
  const int conv_warps = (nthreads >> 5) - kConvWarp0;   // = kpad / (4 kIpt)
  const int k0 = blockIdx.y * kModes;
  const int nks = kpad / 16;
  const int64_t ntiles = (a.n + kTileM - 1) / kTileM;
  const int64_t first = blockIdx.x, stride = gridDim.x;
  const int64_t mine = (first < ntiles) ? (ntiles - first + stride - 1) / stride : 0;

  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&sh.a_full[b]), (unsigned)conv_warps);
      mbar_init(smem_u32(&sh.a_free[b]), 1);
      mbar_init(smem_u32(&sh.acc_full[b]), 1);
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
  for (int q = tid; q < a.p; q += nthreads) tab[q] = (int64_t)((a.start + 1 + q) % a.m) * a.slot_bytes;
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
    // chunk j of this thread is item ct + j T of the tile's K x 8 items
    // (T = converter threads): slot row q = 8 kg + kr, positions 16 pc ..
    // 16 pc + 15; every thread owns exactly kIpt chunks
    const int ct = tid - 32 * kConvWarp0;
    const int T = 32 * conv_warps;
    int64_t src[kIpt];                      // byte offset in the ring (without the tile), -1: row >= p
    unsigned sto[kIpt], ao[kIpt];           // staging and A-tile byte offsets
#pragma unroll
    for (int j = 0; j < kIpt; ++j) {
      const int item = ct + j * T;
      const int kr = item & 7, pc = (item >> 3) & 7, kg = item >> 6;
      const int q = 8 * kg + kr;
      src[j] = (q < a.p) ? tab[q] + 16 * pc : -1;
      sto[j] = (unsigned)(q * kPitch + 16 * pc);
      ao[j] = (unsigned)((kg * 16 + 2 * pc) * 128 + kr * 16);   // core (2 pc, kg), row kr
    }
    const unsigned stg0 = smem_u32(stg);
    auto load_tile = [&](int64_t it) {
      const int64_t i0 = (first + it * stride) * kTileM;
      const unsigned dst = stg0 + (unsigned)((it % kStages) * L.st_bytes);
#pragma unroll
      for (int j = 0; j < kIpt; ++j)
        if (src[j] >= 0) cp_async16(dst + sto[j], a.ring + src[j] + i0);
    };
#pragma unroll
    for (int st = 0; st < kStages - 1; ++st) {
      if (st < mine) load_tile(st);
      cp_async_commit();
    }
    for (int64_t it = 0; it < mine; ++it) {
      if (*stop) break;
      if (it + kStages - 1 < mine) load_tile(it + kStages - 1);
      cp_async_commit();
      cp_async_wait<kStages - 1>();          // this thread's chunks of tile `it` have landed
      const int b = (int)(it % n_a);
      int ok = 1;
      if (lane == 0 && it >= n_a) ok = mbar_wait(smem_u32(&sh.a_free[b]), (unsigned)(((it / n_a) - 1) & 1));
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) {
          atomicOr(a.status, kDevTimeout);
          *stop = 1;
        }
        break;
      }
      const uint8_t* sb = stg + (size_t)(it % kStages) * L.st_bytes;
      uint8_t* ab = abuf + (size_t)b * L.a_bytes;
      uint4 w[kIpt];
#pragma unroll
      for (int j = 0; j < kIpt; ++j) w[j] = *reinterpret_cast<const uint4*>(sb + sto[j]);
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
        *reinterpret_cast<uint4*>(ab + ao[j]) = lo;
        *reinterpret_cast<uint4*>(ab + ao[j] + 128) = hi;
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&sh.a_full[b]));
    }
    cp_async_wait<0>();                      // no copy lands after the CTA exits
  } else if (warp == kMmaWarp) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = idesc_f16_amn(kTileM, kN);
      const unsigned bbase = smem_u32(bbuf);
      int64_t commits = 0;
      for (int64_t it = 0; it < mine; ++it) {
        if (*stop) break;
        const int b = (int)(it % n_a), ab = (int)(it & 1);
        bool ok = mbar_wait(smem_u32(&sh.a_full[b]), (unsigned)((it / n_a) & 1));
        if (ok && it >= 2) ok = mbar_wait(smem_u32(&sh.acc_empty[ab]), (unsigned)(((it >> 1) - 1) & 1));
        if (!ok) {
          atomicOr(a.status, kDevTimeout);
          *stop = 1;
          break;
        }
        fence_after();
        const unsigned abase = smem_u32(abuf + (size_t)b * L.a_bytes);
        for (int ks = 0; ks < nks; ++ks) {
          const uint64_t ad = smem_desc(abase + (unsigned)ks * 4096u, 2048u, 128u);
          const uint64_t bd = smem_desc(bbase + (unsigned)ks * 2u * (kN / 8) * 128u, (kN / 8) * 128u, 128u);
          mma_f16(tbase + (unsigned)(ab * kN), ad, bd, idesc, ks > 0 ? 1u : 0u);
        }
        mma_commit(smem_u32(&sh.a_free[b]));
        mma_commit(smem_u32(&sh.acc_full[ab]));
        commits = it + 1;
      }
      // no MMA may still write tensor memory when it is freed
      if (commits > 0) mbar_wait(smem_u32(&sh.acc_full[(commits - 1) & 1]), (unsigned)(((commits - 1) >> 1) & 1));
    }
  } else {
    // ---------------- epilogue (warps 0..3 own TMEM lanes 32w .. 32w + 31) ----------------
    float sc[kCols];
#pragma unroll
    for (int c = 0; c < kCols; ++c) sc[c] = ldexpf(1.f, -sh.expo[c]);
    float2* out = reinterpret_cast<float2*>(a.phi);
    for (int64_t it = 0; it < mine; ++it) {
      if (*stop) break;
      const int ab = (int)(it & 1);
      int ok = 1;
      if (lane == 0) ok = mbar_wait(smem_u32(&sh.acc_full[ab]), (unsigned)((it >> 1) & 1));
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) {
          atomicOr(a.status, kDevTimeout);
          *stop = 1;
        }
        break;
      }
      fence_after();
      unsigned v0[32], v1[32], v2[32];
      const unsigned taddr = tbase + ((unsigned)(32 * warp) << 16) + (unsigned)(ab * kN);
      tmem_ld32_nowait(taddr, v0);
      tmem_ld32_nowait(taddr + kCols, v1);
      tmem_ld32_nowait(taddr + 2 * kCols, v2);
      tmem_ld_wait();
#pragma unroll
      for (int q = 0; q < 32; ++q) {     // uses of the loaded registers stay after the wait
        asm volatile("" : "+r"(v0[q]));
        asm volatile("" : "+r"(v1[q]));
        asm volatile("" : "+r"(v2[q]));
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&sh.acc_empty[ab]));
      const int64_t i = (first + it * stride) * kTileM + 32 * warp + lane;
      if (i < a.n) {
#pragma unroll
        for (int q = 0; q < kModes; ++q) {
          if (k0 + q < a.r) {
            const float re = (__uint_as_float(v0[2 * q]) + __uint_as_float(v1[2 * q])) + __uint_as_float(v2[2 * q]);
            const float im =
                (__uint_as_float(v0[2 * q + 1]) + __uint_as_float(v1[2 * q + 1])) + __uint_as_float(v2[2 * q + 1]);
            out[(int64_t)(k0 + q) * a.n + i] = make_float2(re * sc[2 * q], im * sc[2 * q + 1]);
          }
        }
      }
    }
  }
  __syncthreads();
  fence_after();
  __syncwarp();
  if (warp == kMmaWarp)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tbase), "r"(kTmemCols) : "memory");
}

template <int kStages, int kIpt>
cudaError_t launch_cfg(const PhiArgs& a, cudaStream_t st, int kpad, int n_a, size_t smem) {
  static size_t attr = 0;
  if (smem > attr) {
    cudaError_t e = cudaFuncSetAttribute(phi_tc_u8_kernel<kStages, kIpt>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = smem;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms < 1) sms = 1;
  const int64_t ntiles = (a.n + kTileM - 1) / kTileM;
  const int ky = (a.r + kModes - 1) / kModes;
  int64_t bx = ((int64_t)sms + ky - 1) / ky;
  if (bx > ntiles) bx = ntiles;
  if (bx < 1) bx = 1;
  const int threads = 32 * (kConvWarp0 + kpad / (4 * kIpt));
  phi_tc_u8_kernel<kStages, kIpt><<<dim3((unsigned)bx, (unsigned)ky), threads, smem, st>>>(a, kpad, n_a);
  return cudaGetLastError();
}

}  // namespace

// Tensor-core Phi for uint8 windows. Returns cudaErrorNotSupported when the
// shape is outside what this kernel handles (the caller then uses the SIMT
// kernel).
cudaError_t launch_phi_tc(const PhiArgs& a, cudaStream_t st) {
  if (a.dtype != SDMD_U8 || a.p < 1 || a.p >= kMaxRows) return cudaErrorNotSupported;
  // K padding and chunks per converter thread, at most 7 converter warps:
  // K <= 112: 4 chunks (K / 16 warps); K <= 224: K to a multiple of 32 and
  // 8 chunks (K / 32 warps); else K = 256 and 16 chunks (4 warps)
  int kpad = ((a.p + 15) / 16) * 16, ipt = 4;
  if (kpad > 112) {
    kpad = ((a.p + 31) / 32) * 32;
    ipt = 8;
    if (kpad > 224) {
      kpad = 256;
      ipt = 16;
    }
  }
  // the deepest copy ring and double-buffered A that fit in 227 KiB
  static const int kConfigs[4][2] = {{2, 6}, {2, 3}, {1, 6}, {1, 3}};
  const int kLimit = 227 * 1024;
  for (const auto& cf : kConfigs) {
    const TcLayout L = tc_layout(kpad, cf[0], cf[1]);
    if (L.total > kLimit) continue;
    // at least 80 KiB: at most two of these CTAs share an SM, so their tensor
    // memory (256 columns each) always fits the SM's 512 columns
    const size_t smem = L.total < 80 * 1024 ? 80 * 1024 : (size_t)L.total;
    // instantiated combinations: K <= 112 always fits (2, 6); K = 256 only
    // fits (1, 3)
    const bool deep = cf[1] == 6;
    if (ipt == 4 && deep) return launch_cfg<6, 4>(a, st, kpad, cf[0], smem);
    if (ipt == 8) return deep ? launch_cfg<6, 8>(a, st, kpad, cf[0], smem) : launch_cfg<3, 8>(a, st, kpad, cf[0], smem);
    if (ipt == 16 && !deep) return launch_cfg<3, 16>(a, st, kpad, cf[0], smem);
  }
  return cudaErrorNotSupported;
}

}  // namespace sdmd
