// Small dense algebra of the exact DMD step (Sec. 2.1 Eqs. 3-4, Sec. 2.2
// Eqs. 7-9; Algorithm 1's eig/sort and Algorithm 2's vsi, A~, eig, vsi*W),
// one CTA of 256 threads per call.
//
// Precision plan. GB300 executes FP64 at about 1/64 of the FP32 rate, and an
// FP64 instruction costs the same whether one lane or 32 are active. So the
// O(p^3) and O(p^2 r) parts run in double-float ("df64", csrc/df64.cuh:
// hi + lo float pairs, ~48 bits) on the FP32 pipes, and the sequential,
// latency-bound parts run in FP32 and are then refined in df64 by steps whose
// result does not depend on the FP32 error to first order:
//
//  0. gather  G_X = G[0:p, 0:p], G_XY = G[0:p, 1:p+1] in time order from the
//     ring-indexed physical G (p = c-1), converted to df64 and scaled by an
//     exact power of two so that the largest diagonal entry is in [0.5, 1).
//  1. Householder tridiagonalisation of G_X in df64: Q^T G_X Q = T (d, e),
//     reflectors kept down the columns of G_X's storage, one block barrier
//     per Householder step (the rank-2 update deferred into the next step).
//  2. the r largest eigenvalues of T by Sturm-count multisection in FP32
//     (one warp per eigenvalue, 32 points per round): shifts accurate to
//     ~eps32 * |T|.
//  3. df64 inverse iteration on T with those shifts (one thread per vector,
//     LU with partial pivoting), classical Gram-Schmidt over all wanted
//     vectors after every solve, then a Rayleigh-Ritz step (Z^T T Z
//     diagonalised by parallel cyclic Jacobi in df64); a second round uses
//     the Ritz values as shifts. Clusters of close eigenvalues are resolved
//     by the Gram-Schmidt / Rayleigh-Ritz steps.
//  4. back-transform z -> Q z in df64 (warp per vector) = columns of V.
//  5. numerical rank, sigma = sqrt(lambda), vsi = V Sigma^-1.
//  6. A~ = vsi^T (G_XY vsi) in df64.
//  7. eig(A~): FP32 complex Householder-Hessenberg, shifted QR (Wilkinson
//     shifts) to Schur form on warp 0, right and left eigenvectors by
//     triangular solves; each eigenvalue is then replaced by the two-sided
//     Rayleigh quotient u^H A~ w / u^H w evaluated in df64, whose error is
//     second order in the FP32 eigenvector errors. W = unit-norm right
//     eigenvectors; eigenpairs ordered by descending |lambda| then angle.
//  8. M = vsi W in df64, written in FP32 (scaled back) for the Phi kernel;
//     lambda, sigma and V written out in FP64.
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <stdint.h>

#include "df64.cuh"
#include "sdmd_internal.cuh"

namespace sdmd {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr double kEps = 2.220446049250313e-16;   // 2^-52 (rank rule, as the oracle)
constexpr double kRankRtol = 64.0;               // rank threshold factor (times p * eps)
constexpr float kEps32 = 5.9604645e-8f;          // 2^-24
constexpr int kInvIters = 2;                     // inverse-iteration solves per vector and round
constexpr int kMsRounds = 8;                     // FP32 multisection rounds (33-way each)
constexpr int kJacobiSweeps = 12;                // Rayleigh-Ritz Jacobi sweep cap
constexpr int kSmemMaxP = 144;                   // G_X kept in shared memory up to this p
constexpr int kRRMax = 32;                       // Rayleigh-Ritz matrices in smem up to this r
constexpr int kClusterExt = 8;                   // eigenvalues added to close a cluster at the boundary
constexpr int kEigMaxR = 48;                     // FP32 eig workspace in smem up to this r

// ------------------------------------------------------------ helpers ----
__device__ __forceinline__ dd shfl_dd(dd v, int o) {
  return {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}
// xor-butterfly sum; dd_add is commutative bit for bit, so all lanes agree
__device__ __forceinline__ dd warp_sum_dd(dd v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = dd_add(v, shfl_dd(v, o));
  return v;
}
__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ dd dd_sel(bool c, dd a, dd b) { return {c ? a.hi : b.hi, c ? a.lo : b.lo}; }

struct CF {
  float re, im;
};
__device__ __forceinline__ CF cadd(CF a, CF b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ CF csub(CF a, CF b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ CF cmul(CF a, CF b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ CF cconj(CF a) { return {a.re, -a.im}; }
__device__ __forceinline__ CF cscale(CF a, float s) { return {a.re * s, a.im * s}; }
__device__ __forceinline__ float cabs2(CF a) { return a.re * a.re + a.im * a.im; }
__device__ __forceinline__ float cabs(CF a) { return hypotf(a.re, a.im); }
// a / b by Smith's method (no overflow or underflow of |b|^2)
__device__ __forceinline__ CF cdiv(CF a, CF b) {
  if (fabsf(b.re) >= fabsf(b.im)) {
    const float r = b.im / b.re, den = b.re + b.im * r;
    return {(a.re + a.im * r) / den, (a.im - a.re * r) / den};
  }
  const float r = b.re / b.im, den = b.re * r + b.im;
  return {(a.re * r + a.im) / den, (a.im * r - a.re) / den};
}
__device__ __forceinline__ CF csqrt(CF z) {
  const float m = cabs(z);
  if (m == 0.f) return {0.f, 0.f};
  const float re = sqrtf(0.5f * (m + fabsf(z.re)));
  const float im = z.im / (2.f * re);
  if (z.re >= 0.f) return {re, im};
  return {fabsf(im), copysignf(re, z.im)};
}

struct WS {
  dd *GXYd, *Ad, *Z, *Y, *lu;
  double *V, *sig, *lamout, *bamp;
  float* Mf;
  long long* clk;
};

__device__ WS carve(double* base, const ModesLayout& L) {
  WS w;
  w.GXYd = reinterpret_cast<dd*>(base + L.GXY);
  w.Ad = reinterpret_cast<dd*>(base + L.A);
  w.Z = reinterpret_cast<dd*>(base + L.Z);
  w.Y = reinterpret_cast<dd*>(base + L.Y);
  w.lu = reinterpret_cast<dd*>(base + L.lu);
  w.V = base + L.V;
  w.sig = base + L.sig;
  w.lamout = base + L.lamout;
  w.bamp = base + L.bamp;
  w.Mf = reinterpret_cast<float*>(base + L.Mf);
  w.clk = reinterpret_cast<long long*>(base + L.clk);
  return w;
}

// ---------------------------------------------------------------- phase 1 --
// df64 Householder reduction of the symmetric p x p matrix A (row-major,
// full storage) to tridiagonal form (d, e). Reflector k is I - 2 v v^T on
// indices k+1..p-1 with v unit (zero if column k is already reduced); it is
// stored down column k, A[k+1..p-1][k].
//
// One block barrier per step. Step k's rank-2 update A -= v w^T + w v^T
// (w = 2 (A v - (v^T A v) v)) is not applied in step k: step k+1 applies it
// while it reads the trailing block for its own product A u, so the block is
// read and written once per step. Warp w owns trailing rows w, w + 8, ...
// and lane l columns l, l + 32, ...; as the block is symmetric, the row sums
// of A u are also its column sums, so each lane sums its columns over its
// warp's rows, and u^T A u comes from the same column sums. After the
// barrier every warp adds the eight warps' parts for its lanes' columns and
// forms v, A v and w itself, then the next pivot row, its norm and the
// reflector's scalars: the same operations in the same order in every warp,
// so all warps hold the same bits without a second barrier. The block stays
// exactly symmetric: the update term of (i, j) is formed from the same
// products, added in an order-free way, as that of (j, i).
//
// Workspace tw (8-byte units): part[2][kWarps][P] (per-warp column sums by
// step parity), u, v, w [kWarps][P] (each warp's copy, indexed by row, of
// the current reflector's u and of the pending reflector's v and w),
// dot[2][kWarps] (per-warp parts of u^T A_sub u).
constexpr int kTriCols = 8;   // columns per lane: p <= 8 * 32
constexpr int kTriUnitsPerP = 5 * kWarps;

// a*b as an unevaluated (hi, lo) pair whose bits do not depend on the operand order
__device__ __forceinline__ dd dd_mul_sym(dd a, dd b) {
  const float ph = a.hi * b.hi;
  const float pe = fmaf(a.hi, b.hi, -ph);
  return {ph, pe + __fadd_rn(__fmul_rn(a.hi, b.lo), __fmul_rn(a.lo, b.hi))};   // no fma contraction
}
// a - (v_i w_j + w_i v_j); the same bits for (i, j) and (j, i)
__device__ __forceinline__ dd dd_rank2_sub(dd a, dd vi, dd wi, dd vj, dd wj) {
  const dd p1 = dd_mul_sym(vi, wj), p2 = dd_mul_sym(wi, vj);
  const dd s = two_sum(p1.hi, p2.hi);
  const float c = (p1.lo + p2.lo) + s.lo;
  const dd r = two_sum(a.hi, -s.hi);
  return quick_two_sum(r.hi, (a.lo - c) + r.lo);
}
// running sum (s, c) += a * b, c collecting the rounding errors (Dot2-style)
__device__ __forceinline__ void dot2_acc(float& s, float& c, dd a, dd b) {
  const float ph = a.hi * b.hi;
  float pe = fmaf(a.hi, b.hi, -ph);
  pe = fmaf(a.hi, b.lo, pe);
  pe = fmaf(a.lo, b.hi, pe);
  const dd t = two_sum(s, ph);
  s = t.hi;
  c += t.lo + pe;
}
// (hi, lo) pairs added without renormalising the tail (Dot2-style): the
// exact error of the leading parts is kept, the tails are added in FP32
__device__ __forceinline__ dd pair_add(dd a, dd b) {
  const dd t = two_sum(a.hi, b.hi);
  return {t.hi, (a.lo + b.lo) + t.lo};
}
// the eight per-warp parts x[0], x[st], ..., x[7 st] summed as a fixed tree
__device__ __forceinline__ dd dd_sum8(const dd* x, int64_t st) {
  const dd a = pair_add(x[0], x[st]), b = pair_add(x[2 * st], x[3 * st]);
  const dd c = pair_add(x[4 * st], x[5 * st]), f = pair_add(x[6 * st], x[7 * st]);
  const dd r = pair_add(pair_add(a, b), pair_add(c, f));
  return quick_two_sum(r.hi, r.lo);
}
static_assert(kWarps == 8, "dd_sum8 adds one part per warp");

__device__ void tridiagonalize(dd* A, int p, dd* d, dd* e, dd* tw, int64_t P) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  dd* part = tw;                                            // [2][kWarps][P]
  dd* uw = tw + (2 * kWarps + warp) * P;                    // this warp's u, v, w by row
  dd* vw = tw + (3 * kWarps + warp) * P;
  dd* ww = tw + (4 * kWarps + warp) * P;
  dd* dotp = tw + (int64_t)kTriUnitsPerP * P;               // [2][kWarps]
  // pending reflector's v, w at g = k + lane + 32c (from the previous step's combine)
  dd vr[kTriCols], wr[kTriCols];
#pragma unroll
  for (int c = 0; c < kTriCols; ++c) {
    vr[c] = {0.f, 0.f};
    wr[c] = {0.f, 0.f};
  }
  for (int k = 0; k + 2 < p; ++k) {
    const int L = p - k - 1;
    const int par = k & 1;
    const bool pend = (k > 0);
    // pivot row k of the updated matrix, x_g for g = k..p-1 (lane g - k + 32c)
    const dd vk = {__shfl_sync(0xffffffffu, vr[0].hi, 0), __shfl_sync(0xffffffffu, vr[0].lo, 0)};
    const dd wk = {__shfl_sync(0xffffffffu, wr[0].hi, 0), __shfl_sync(0xffffffffu, wr[0].lo, 0)};
    float ts = 0.f, tc = 0.f;
    dd xk[kTriCols];
#pragma unroll
    for (int c = 0; c < kTriCols; ++c) {
      xk[c] = {0.f, 0.f};
      if (32 * c > L) break;             // warp-uniform: no slot beyond the row
      const int g = k + lane + 32 * c;
      dd x = {0.f, 0.f};
      if (g < p) {
        x = A[(int64_t)k * p + g];
        if (pend) x = dd_rank2_sub(x, vk, wk, vr[c], wr[c]);
        if (g >= k + 2) dot2_acc(ts, tc, x, x);
      }
      xk[c] = x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {   // xor butterfly: all lanes end with the same bits
      const float so = __shfl_xor_sync(0xffffffffu, ts, o), co = __shfl_xor_sync(0xffffffffu, tc, o);
      const dd q = two_sum(ts, so);
      ts = q.hi;
      tc = (tc + co) + q.lo;
    }
    const dd t = quick_two_sum(ts, tc);
    const dd x0 = {__shfl_sync(0xffffffffu, xk[0].hi, 1), __shfl_sync(0xffffffffu, xk[0].lo, 1)};
    dd inv = {0.f, 0.f}, u0 = x0, ek = x0;
    if (t.hi != 0.f) {
      const dd nrm = dd_sqrt(dd_fma(x0, x0, t));
      const dd alpha = (x0.hi >= 0.f) ? dd_neg(nrm) : nrm;
      u0 = dd_sub(x0, alpha);                       // same sign as x0: no cancellation
      inv = dd_recip(dd_sqrt(dd_fma(u0, u0, t)));
      ek = alpha;
    }
    // this warp's copy of u (u_{k+1} = x0 - alpha, u_g = x_g beyond)
#pragma unroll
    for (int c = 0; c < kTriCols; ++c) {
      if (32 * c > L) break;
      const int g = k + lane + 32 * c;
      if (g > k && g < p) uw[g] = (g == k + 1) ? u0 : xk[c];
    }
    if (warp == 0 && lane == 0) {
      d[k] = xk[0];
      e[k] = ek;
    }
    __syncwarp();
    // trailing block rows/cols k+1..p-1: apply the pending update, store, and
    // sum a_ij u_i down this lane's columns j over this warp's rows i
    dd vc[kTriCols], wc[kTriCols];
    float cs[kTriCols], cc[kTriCols];
#pragma unroll
    for (int c = 0; c < kTriCols; ++c) {
      const int gj = k + 1 + lane + 32 * c;
      vc[c] = {0.f, 0.f};
      wc[c] = {0.f, 0.f};
      cs[c] = 0.f;
      cc[c] = 0.f;
      if (32 * c >= L) continue;
      if (pend && gj < p) {
        vc[c] = vw[gj];
        wc[c] = ww[gj];
      }
    }
    // four rows per iteration: their loads, updates and sums interleave
    for (int i0 = warp; i0 < L; i0 += 4 * kWarps) {
      dd ui[4], vi[4], wi[4];
      dd* rp[4];
      bool ok[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = i0 + q * kWarps;
        ok[q] = i < L;
        const int gi = ok[q] ? k + 1 + i : k + 1;
        ui[q] = ok[q] ? uw[gi] : dd{0.f, 0.f};
        vi[q] = (pend && ok[q]) ? vw[gi] : dd{0.f, 0.f};
        wi[q] = (pend && ok[q]) ? ww[gi] : dd{0.f, 0.f};
        rp[q] = A + (int64_t)gi * p + (k + 1);
      }
#pragma unroll
      for (int c = 0; c < kTriCols; ++c) {
        if (32 * c >= L) break;
        const int j = lane + 32 * c;
        if (j < L) {
          dd av[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) av[q] = ok[q] ? rp[q][j] : dd{0.f, 0.f};
          if (pend) {
#pragma unroll
            for (int q = 0; q < 4; ++q) av[q] = dd_rank2_sub(av[q], vi[q], wi[q], vc[c], wc[c]);
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (ok[q]) rp[q][j] = av[q];
          }
#pragma unroll
          for (int q = 0; q < 4; ++q)   // rows past L add zero products
            dot2_acc(cs[c], cc[c], av[q], ui[q]);
        }
      }
    }
    // column parts, and this warp's part of u^T A_sub u
    dd* pp = part + (int64_t)par * kWarps * P;
    float us = 0.f, uc = 0.f;
#pragma unroll
    for (int c = 0; c < kTriCols; ++c) {
      if (32 * c >= L) break;
      const int gj = k + 1 + lane + 32 * c;
      if (gj < p) {
        const dd T = quick_two_sum(cs[c], cc[c]);
        pp[(int64_t)warp * P + gj] = T;
        dot2_acc(us, uc, uw[gj], T);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float so = __shfl_xor_sync(0xffffffffu, us, o), co = __shfl_xor_sync(0xffffffffu, uc, o);
      const dd q = two_sum(us, so);
      us = q.hi;
      uc = (uc + co) + q.lo;
    }
    if (lane == 0) dotp[par * kWarps + warp] = quick_two_sum(us, uc);
    __syncthreads();
    // every warp: A_sub u for its lanes' rows, v = u inv, pv = A_sub v,
    // K = v^T pv = inv^2 u^T A_sub u, w = 2 (pv - K v); reflector k down column k
    const dd kv = dd_mul(dd_mul(dd_sum8(dotp + par * kWarps, 1), inv), inv);
#pragma unroll
    for (int c = 0; c < kTriCols; ++c) {
      if (32 * c >= L) break;
      const int g = k + 1 + lane + 32 * c;
      if (g < p) {
        const dd pvg = dd_mul(dd_sum8(pp + g, P), inv);
        const dd vg = dd_mul(uw[g], inv);
        const dd wg = dd_scale(dd_sub(pvg, dd_mul(kv, vg)), 2.f);
        vw[g] = vg;
        ww[g] = wg;
        vr[c] = vg;
        wr[c] = wg;
        if (warp == 0) A[(int64_t)g * p + k] = vg;
      }
    }
    __syncwarp();
  }
  if (threadIdx.x == 0) {
    if (p >= 3) {   // the last reflector's update of the final 2 x 2 block
      const int k = p - 2;
      const dd v0 = vw[k], v1 = vw[k + 1], w0 = ww[k], w1 = ww[k + 1];
      d[k] = dd_rank2_sub(A[(int64_t)k * p + k], v0, w0, v0, w0);
      d[k + 1] = dd_rank2_sub(A[(int64_t)(k + 1) * p + k + 1], v1, w1, v1, w1);
      e[k] = dd_rank2_sub(A[(int64_t)k * p + k + 1], v0, w0, v1, w1);
    } else if (p == 2) {
      d[0] = A[0];
      d[1] = A[3];
      e[0] = A[1];
    } else {
      d[0] = A[0];
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- phase 2 --
// Number of eigenvalues of the FP32 tridiagonal (d, e^2) below x. The
// divisions use the fast reciprocal (about 2 ulp): the counts only place
// FP32 shifts, which the df64 inverse iteration refines.
__device__ int sturm32(const float* d, const float* e2, int p, float x, float pivmin) {
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  int cnt = (q < 0.f);
  for (int i = 1; i < p; ++i) {
    q = (d[i] - x) - __fdividef(e2[i - 1], q);   // |q| >= pivmin keeps e2 / q below 2^126
    if (fabsf(q) < pivmin) q = -pivmin;
    cnt += (q < 0.f);
  }
  return cnt;
}

// Number of eigenvalues of the df64 tridiagonal (d, e) below x (pivots kept
// at least pivmin away from zero): the df64 counterpart of sturm32, for the
// missed-eigenvalue check and the df64 multisection of phase 3'.
__device__ int sturm_below_dd(const dd* d, const dd* e, int p, dd x, float pivmin) {
  dd q = dd_sub(d[0], x);
  if (fabsf(q.hi) < pivmin) q = dd_make(-pivmin);
  int below = q.hi < 0.f;
  for (int i = 1; i < p; ++i) {
    q = dd_sub(dd_sub(d[i], x), dd_mul(dd_mul(e[i - 1], e[i - 1]), dd_recip(q)));
    if (fabsf(q.hi) < pivmin) q = dd_make(-pivmin);
    below += q.hi < 0.f;
  }
  return below;
}

// ---------------------------------------------------------------- phase 3 --
// LU with partial pivoting of the df64 tridiagonal T - mu I. Row i of U has
// (1/u0, u1, u2) on columns (i, i+1, i+2) (diagonal stored as reciprocal);
// mult / piv (0 or 1) describe L. Pivots below `tiny` are raised to it.
// Branch-free (selects), so the lanes of a warp that factor different shifts
// never diverge.
__device__ void tri_lu_dd(const dd* __restrict__ d, const dd* __restrict__ e, int p, dd mu, float tiny,
                          dd* __restrict__ u0, dd* __restrict__ u1, dd* __restrict__ u2, dd* __restrict__ mult,
                          dd* __restrict__ piv) {
  dd cd = dd_sub(d[0], mu), c1 = (p > 1) ? e[0] : dd{0.f, 0.f};
  for (int i = 0; i + 1 < p; ++i) {
    const dd sub = e[i];
    const dd nd = dd_sub(d[i + 1], mu);
    const dd n1 = (i + 2 < p) ? e[i + 1] : dd{0.f, 0.f};
    const bool sw = fabsf(cd.hi) < fabsf(sub.hi);   // row i+1 becomes the pivot row
    dd pv = dd_sel(sw, sub, cd);
    const dd num = dd_sel(sw, cd, sub);
    if (fabsf(pv.hi) < tiny) pv = {copysignf(tiny, pv.hi), 0.f};
    const dd rp = dd_recip(pv);
    const dd m = (pv.hi != 0.f) ? dd_mul(num, rp) : dd{0.f, 0.f};
    u0[i] = rp;
    u1[i] = dd_sel(sw, nd, c1);
    u2[i] = dd_sel(sw, n1, dd{0.f, 0.f});
    piv[i] = {sw ? 1.f : 0.f, 0.f};
    mult[i] = m;
    // no swap: row i+1 - m row i = (nd - m c1, n1); swap: row i - m row i+1 = (c1 - m nd, -m n1)
    cd = dd_sub(dd_sel(sw, c1, nd), dd_mul(m, dd_sel(sw, nd, c1)));
    c1 = sw ? dd_neg(dd_mul(m, n1)) : n1;
  }
  dd last = cd;
  if (fabsf(last.hi) < tiny) last = {copysignf(tiny, last.hi), 0.f};
  u0[p - 1] = dd_recip(last);
  u1[p - 1] = {0.f, 0.f};
  u2[p - 1] = {0.f, 0.f};
}

__device__ void tri_solve_dd(int p, const dd* __restrict__ u0inv, const dd* __restrict__ u1,
                             const dd* __restrict__ u2, const dd* __restrict__ mult, const dd* __restrict__ piv,
                             dd* __restrict__ b) {
  dd bi = b[0];
  for (int i = 0; i + 1 < p; ++i) {   // forward, branch-free: b_i is carried in registers
    const bool sw = piv[i].hi != 0.f;
    const dd bn = b[i + 1];
    const dd keep = dd_sel(sw, bn, bi), elim = dd_sel(sw, bi, bn);
    b[i] = keep;
    bi = dd_sub(elim, dd_mul(mult[i], keep));
  }
  b[p - 1] = bi;
  dd x1 = {0.f, 0.f}, x2 = {0.f, 0.f};   // x_{i+1}, x_{i+2}
  for (int i = p - 1; i >= 0; --i) {
    dd s = dd_sub(b[i], dd_mul(u2[i], x2));
    s = dd_sub(s, dd_mul(u1[i], x1));
    const dd x = dd_mul(s, u0inv[i]);
    b[i] = x;
    x2 = x1;
    x1 = x;
  }
}

// Orthonormalise vectors Z[i*p ..], i < rw, in order (classical Gram-Schmidt,
// `passes` times). The vectors stay unnormalised until the end: vector i is
// projected with coefficients ((z_j . z_i) / |z_j|) / |z_j|, the dots of one pass
// (and the vector's own norm) taken together, one vector per warp and the
// positions over its lanes; one final pass scales every vector. A vector that
// lies (to working precision) in the span of the earlier ones -- inverse
// iteration with shifts inside a cluster closer than the shifts' resolution --
// is replaced by a fixed pseudo-random vector and projected twice, so the set
// stays a basis of the cluster's subspace. rn: rw reciprocal norms 1 / |z_j|
// (not 1 / |z_j|^2: after a solve |z|^2 reaches ~1e30, and the low word of
// its reciprocal would sit in FP32's denormal range).
__device__ dd block_sum_dd(dd v, dd* red) {   // every thread gets the same sum
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  v = warp_sum_dd(v);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  dd t = red[0];
  for (int w = 1; w < kWarps; ++w) t = dd_add(t, red[w]);
  __syncthreads();
  return t;
}

// one projection pass of z_i against z_0..z_{i-1}; with `self` also z_i . z_i
// (before the projection) into *self_out
__device__ void cgs_pass(dd* Z, int i, int p, const dd* rn, dd* coef, dd* self_out) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const dd* zi = Z + (int64_t)i * p;
  const int nj = self_out ? i + 1 : i;
  for (int j = warp; j < nj; j += kWarps) {
    const dd* zj = Z + (int64_t)j * p;
    dd acc = {0.f, 0.f};   // full df64 sums: the basis must be orthonormal to df64 resolution
    for (int q = lane; q < p; q += 32) acc = dd_fma(zj[q], zi[q], acc);
    acc = warp_sum_dd(acc);
    if (lane == 0) {
      const dd dt = acc;
      if (j < i)
        coef[j] = dd_mul(dd_mul(dt, rn[j]), rn[j]);
      else
        *self_out = dt;
    }
  }
  __syncthreads();
  dd* zw = Z + (int64_t)i * p;
  for (int q = tid; q < p; q += kThreads) {
    dd s = zw[q];
    for (int j = 0; j < i; ++j) s = dd_sub(s, dd_mul(coef[j], Z[(int64_t)j * p + q]));
    zw[q] = s;
  }
  __syncthreads();
}

__device__ void cgs_dd(dd* Z, int rw, int p, int passes, dd* coef, dd* rn, dd* red, dd* sc) {
  const int tid = threadIdx.x;
  for (int i = 0; i < rw; ++i) {
    dd* zi = Z + (int64_t)i * p;
    for (int pass = 0; pass < passes && i > 0; ++pass) cgs_pass(Z, i, p, rn, coef, pass == 0 ? &sc[3] : nullptr);
    dd nn = {0.f, 0.f};
    for (int q = tid; q < p; q += kThreads) nn = dd_fma(zi[q], zi[q], nn);
    dd t = block_sum_dd(nn, red);
    if (i > 0 && !(t.hi > 1e-20f * sc[3].hi)) {   // collapsed: reseed and project twice
      for (int q = tid; q < p; q += kThreads) {
        const unsigned hsh = (unsigned)(q + 1) * 2654435761u ^ (unsigned)(i + 1) * 40503u;
        zi[q] = dd_make((float)((hsh >> 8) & 0xFFFFu) / 65536.f - 0.5f);
      }
      __syncthreads();
      for (int pass = 0; pass < 2; ++pass) cgs_pass(Z, i, p, rn, coef, nullptr);
      nn = {0.f, 0.f};
      for (int q = tid; q < p; q += kThreads) nn = dd_fma(zi[q], zi[q], nn);
      t = block_sum_dd(nn, red);
    }
    if (tid == 0) rn[i] = (t.hi > 0.f) ? dd_recip(dd_sqrt(t)) : dd{0.f, 0.f};
    __syncthreads();
  }
  for (int idx = tid; idx < rw * p; idx += kThreads) Z[idx] = dd_mul(Z[idx], rn[idx / p]);
  __syncthreads();
}

// Rayleigh-Ritz on the orthonormal vectors Z (rw x p, vector-major):
// H = Z^T T Z (df64) diagonalised by parallel cyclic Jacobi (circle-method
// pairing, disjoint rotations per round); Z <- Z R with columns ordered by
// descending Ritz value, lam <- those values. H, R: rw*rw; tz: rw*p scratch.
__device__ void rayleigh_ritz(dd* Z, int rw, int p, const dd* d, const dd* e, dd* H, dd* R, dd* tz, dd* lam,
                              dd* sc, int* ord) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int idx = tid; idx < rw * p; idx += kThreads) {
    const int i = idx / p, q = idx - i * p;
    const dd* z = Z + (int64_t)i * p;
    dd t = dd_mul(d[q], z[q]);
    if (q > 0) t = dd_fma(e[q - 1], z[q - 1], t);
    if (q + 1 < p) t = dd_fma(e[q], z[q + 1], t);
    tz[idx] = t;
  }
  __syncthreads();
  for (int pr = warp; pr < rw * rw; pr += kWarps) {
    const int a = pr / rw, b = pr - a * rw;
    if (b < a) continue;
    dd s = {0.f, 0.f};
    for (int q = lane; q < p; q += 32) s = dd_fma(Z[(int64_t)a * p + q], tz[(int64_t)b * p + q], s);
    s = warp_sum_dd(s);
    if (lane == 0) {
      H[a * rw + b] = s;
      H[b * rw + a] = s;
    }
  }
  for (int idx = tid; idx < rw * rw; idx += kThreads) R[idx] = {(idx / rw == idx % rw) ? 1.f : 0.f, 0.f};
  __syncthreads();
  const int n2 = rw + (rw & 1);
  for (int sweep = 0; sweep < kJacobiSweeps && rw > 1; ++sweep) {
    if (warp == 0) {    // converged when the off-diagonal is below df64 resolution
      float off = 0.f, dia = 0.f;
      for (int idx = lane; idx < rw * rw; idx += 32) {
        const float v = fabsf(H[idx].hi);
        if (idx / rw == idx % rw)
          dia = fmaxf(dia, v);
        else
          off = fmaxf(off, v);
      }
      off = warp_max_f(off);
      dia = warp_max_f(dia);
      if (lane == 0) sc[4] = {(off <= 1e-15f * dia) ? 1.f : 0.f, 0.f};
    }
    __syncthreads();
    if (sc[4].hi != 0.f) break;
    for (int round = 0; round < n2 - 1; ++round) {
      for (int k = tid; k < n2 / 2; k += kThreads) {
        int a = (k == 0) ? 0 : 1 + (k - 1 + round) % (n2 - 1);
        int b = 1 + (n2 - 2 - k + round) % (n2 - 1);
        if (a > b) {
          const int t = a;
          a = b;
          b = t;
        }
        dd c = {1.f, 0.f}, s = {0.f, 0.f};
        if (b < rw) {
          const dd hab = H[a * rw + b];
          if (hab.hi != 0.f) {
            const dd tau = dd_mul(dd_sub(H[b * rw + b], H[a * rw + a]), dd_recip(dd_scale(hab, 2.f)));
            // |tau| > 1e18 (or not finite: h_ab is a denormal): h_ab is below
            // 1e-18 of the diagonal gap, under df64 resolution, and the
            // rotation would be the identity to working precision; tau^2
            // would also leave the FP32 exponent range. Skip it.
            if (fabsf(tau.hi) <= 1e18f) {
              const dd root = dd_sqrt(dd_fma(tau, tau, dd_make(1.f)));
              dd t = dd_recip(dd_add(dd_abs(tau), root));
              if (tau.hi < 0.f) t = dd_neg(t);
              c = dd_recip(dd_sqrt(dd_fma(t, t, dd_make(1.f))));
              s = dd_mul(t, c);
            }
          }
        }
        ord[2 * k] = a;
        ord[2 * k + 1] = b;
        tz[2 * k] = c;
        tz[2 * k + 1] = s;
      }
      __syncthreads();
      for (int idx = tid; idx < (n2 / 2) * rw; idx += kThreads) {   // rows: H <- J^T H
        const int k = idx / rw, col = idx - k * rw;
        const int a = ord[2 * k], b = ord[2 * k + 1];
        if (b >= rw) continue;
        const dd c = tz[2 * k], s = tz[2 * k + 1];
        const dd ha = H[a * rw + col], hb = H[b * rw + col];
        H[a * rw + col] = dd_sub(dd_mul(c, ha), dd_mul(s, hb));
        H[b * rw + col] = dd_add(dd_mul(s, ha), dd_mul(c, hb));
      }
      __syncthreads();
      for (int idx = tid; idx < (n2 / 2) * rw * 2; idx += kThreads) {   // columns: H <- H J, R <- R J
        const int half = idx / ((n2 / 2) * rw);
        const int rem = idx - half * (n2 / 2) * rw;
        const int k = rem / rw, row = rem - k * rw;
        const int a = ord[2 * k], b = ord[2 * k + 1];
        if (b >= rw) continue;
        dd* M = half ? R : H;
        const dd c = tz[2 * k], s = tz[2 * k + 1];
        const dd ma = M[row * rw + a], mb = M[row * rw + b];
        M[row * rw + a] = dd_sub(dd_mul(c, ma), dd_mul(s, mb));
        M[row * rw + b] = dd_add(dd_mul(s, ma), dd_mul(c, mb));
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    for (int a = 0; a < rw; ++a) ord[a] = a;
    for (int a = 0; a < rw; ++a) {
      int best = a;
      for (int b = a + 1; b < rw; ++b)
        if (dd_lt(H[ord[best] * rw + ord[best]], H[ord[b] * rw + ord[b]])) best = b;
      const int t = ord[a];
      ord[a] = ord[best];
      ord[best] = t;
    }
  }
  __syncthreads();
  for (int a = tid; a < rw; a += kThreads) lam[a] = H[ord[a] * rw + ord[a]];
  for (int idx = tid; idx < rw * p; idx += kThreads) {   // tz <- Z R (permuted)
    const int a = idx / p, q = idx - a * p;
    const int col = ord[a];
    dd s = {0.f, 0.f};
    for (int b = 0; b < rw; ++b) s = dd_fma(Z[(int64_t)b * p + q], R[b * rw + col], s);
    tz[idx] = s;
  }
  __syncthreads();
  for (int idx = tid; idx < rw * p; idx += kThreads) Z[idx] = tz[idx];
  __syncthreads();
}

// ---------------------------------------------------------------- phase 7 --
// FP32 eigen-decomposition of the complex r x r matrix H (row-major) on one
// warp: Hessenberg reduction, shifted QR to Schur form with Q accumulated,
// right eigenvectors W and left eigenvectors U (columns, unit norm).
// Returns false if the QR iteration cap was reached.
// Complex Givens rotation [c s; -conj(s) c] taking (a, b) to (rho, 0). (a, b)
// are scaled by a power of two to a largest component in [1, 2) (c and s do
// not change), so the squared moduli neither underflow nor overflow; then c,
// s from one reciprocal square root.
__device__ __forceinline__ void givens32(CF a, CF b, float& c, CF& s) {
  const float mx = fmaxf(fmaxf(fabsf(a.re), fabsf(a.im)), fmaxf(fabsf(b.re), fabsf(b.im)));
  if (mx == 0.f) {
    c = 1.f;
    s = {0.f, 0.f};
    return;
  }
  const int be = min((__float_as_int(mx) >> 23) & 0xff, 253);
  const float sc = __int_as_float((254 - be) << 23);
  a = cscale(a, sc);
  b = cscale(b, sc);
  const float aa2 = cabs2(a), rho2 = aa2 + cabs2(b);
  if (aa2 < 1e-30f) {   // |a| negligible against |b| >= 1
    c = 0.f;
    s = {1.f, 0.f};
    return;
  }
  // k = 1 / (|a| rho): c = |a|^2 k, s = a conj(b) k; rsqrt plus one Newton
  // step (about 1 ulp), so c^2 + |s|^2 = 1 to FP32 rounding
  const float x = aa2 * rho2;
  float k = rsqrtf(x);
  k = k * fmaf(-0.5f * x * k, k, 1.5f);
  c = aa2 * k;
  s = cscale(cmul(a, cconj(b)), k);
}

__device__ bool warp_eig32(CF* H, CF* Q, CF* W, CF* U, CF* ycol, int r, float* cs, CF* sn) {
  const int lane = threadIdx.x & 31;
  for (int idx = lane; idx < r * r; idx += 32) {
    const int i = idx / r, j = idx - i * r;
    Q[idx] = {i == j ? 1.f : 0.f, 0.f};
  }
  __syncwarp();
  for (int j = 0; j + 2 < r; ++j) {
    const int L = r - j - 1;
    float tail = 0.f;
    for (int i = 1 + lane; i < L; i += 32) tail += cabs2(H[(j + 1 + i) * r + j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tail += __shfl_xor_sync(0xffffffffu, tail, o);
    const CF x0 = H[(j + 1) * r + j];
    __syncwarp();
    if (tail == 0.f) continue;
    const float ax0 = cabs(x0);
    const float nrm = sqrtf(ax0 * ax0 + tail);
    const CF ph = (ax0 > 0.f) ? cscale(x0, 1.f / ax0) : CF{1.f, 0.f};
    const CF alpha = cscale(ph, -nrm);
    const CF v0 = csub(x0, alpha);
    const float vn_inv = 1.f / sqrtf(cabs2(v0) + tail);
    for (int i = lane; i < L; i += 32) ycol[i] = cscale(i == 0 ? v0 : H[(j + 1 + i) * r + j], vn_inv);
    __syncwarp();
    for (int q = j + lane; q < r; q += 32) {
      CF s = {0.f, 0.f};
      for (int i = 0; i < L; ++i) s = cadd(s, cmul(cconj(ycol[i]), H[(j + 1 + i) * r + q]));
      for (int i = 0; i < L; ++i) H[(j + 1 + i) * r + q] = csub(H[(j + 1 + i) * r + q], cscale(cmul(ycol[i], s), 2.f));
    }
    __syncwarp();
    for (int q = lane; q < 2 * r; q += 32) {
      CF* M = (q < r) ? H : Q;
      const int row = (q < r) ? q : q - r;
      CF s = {0.f, 0.f};
      for (int i = 0; i < L; ++i) s = cadd(s, cmul(M[row * r + j + 1 + i], ycol[i]));
      for (int i = 0; i < L; ++i)
        M[row * r + j + 1 + i] = csub(M[row * r + j + 1 + i], cscale(cmul(s, cconj(ycol[i])), 2.f));
    }
    __syncwarp();
    for (int i = 2 + lane; i <= L; i += 32) H[(j + i) * r + j] = {0.f, 0.f};
    __syncwarp();
  }
  float hnorm = 0.f;
  for (int idx = lane; idx < r * r; idx += 32) hnorm = fmaxf(hnorm, cabs(H[idx]));
  hnorm = warp_max_f(hnorm);
  if (hnorm == 0.f) hnorm = 1.f;
  bool ok = true;
  int hi = r - 1, its = 0, total = 0;
  const int cap = 60 * r + 60;
  while (hi > 0) {
    // l = the largest i <= hi whose subdiagonal H[i][i-1] is negligible
    // (|h| <= eps32 (|a|^2 + |b|^2)^(1/2), in squares), else 0
    auto negligible = [&](int i) {
      const float sub2 = cabs2(H[i * r + i - 1]);
      float scale2 = cabs2(H[i * r + i]) + cabs2(H[(i - 1) * r + i - 1]);
      if (scale2 == 0.f) scale2 = hnorm * hnorm;
      return sub2 <= kEps32 * kEps32 * scale2;
    };
    int l = hi;
    if (r <= 32) {   // one subdiagonal per lane
      const unsigned neg = __ballot_sync(0xffffffffu, lane >= 1 && lane <= hi && negligible(lane));
      l = neg ? 31 - __clz(neg) : 0;
    } else {
      while (l > 0 && !negligible(l)) --l;
    }
    __syncwarp();
    if (l > 0 && lane == 0) H[l * r + l - 1] = {0.f, 0.f};
    __syncwarp();
    if (l == hi) {
      --hi;
      its = 0;
      continue;
    }
    if (total >= cap) {
      ok = false;
      break;
    }
    ++its;
    ++total;
    CF mu;
    {
      const CF a = H[(hi - 1) * r + hi - 1], b = H[(hi - 1) * r + hi], c = H[hi * r + hi - 1],
               dl = H[hi * r + hi];
      if (its % 11 == 10) {
        mu = cadd(dl, CF{0.75f * cabs(c), 0.f});
      } else {
        const CF half = cscale(csub(a, dl), 0.5f);
        const CF disc = csqrt(cadd(cmul(half, half), cmul(b, c)));
        const CF tr = cscale(cadd(a, dl), 0.5f);
        const CF m1 = cadd(tr, disc), m2 = csub(tr, disc);
        mu = (cabs(csub(m1, dl)) <= cabs(csub(m2, dl))) ? m1 : m2;
      }
    }
    for (int q = l + lane; q <= hi; q += 32) H[q * r + q] = csub(H[q * r + q], mu);
    __syncwarp();
    if (r <= 32) {
      // row rotations: lane q carries H[j][q] through rotations j = l..min(q, hi-1)
      // in registers; rotation j's pivot H[j][j] comes from lane j by shuffle
      const int q = lane;
      const bool col = q >= l && q < r;
      CF cur = col ? H[l * r + q] : CF{0.f, 0.f};
      for (int j = l; j < hi; ++j) {
        const CF a = {__shfl_sync(0xffffffffu, cur.re, j), __shfl_sync(0xffffffffu, cur.im, j)};
        const CF b = H[(j + 1) * r + j];   // row j+1 is untouched before rotation j
        float c;
        CF s;
        givens32(a, b, c, s);
        if (col && q >= j) {
          const CF h2 = H[(j + 1) * r + q];
          H[j * r + q] = cadd(cscale(cur, c), cmul(s, h2));
          cur = csub(cscale(h2, c), cmul(cconj(s), cur));
        }
        if (lane == 0) {
          cs[j] = c;
          sn[j] = s;
        }
      }
      if (col) H[(min(q, hi - 1) + 1) * r + q] = cur;
      __syncwarp();
      // column rotations: lane q applies rotations j >= max(l, q-1) to H's row
      // q (rows above j+1 only) and all of them to Q's row q, carrying column j
      if (q < r) {
        const int j0 = max(l, q - 1);
        const bool hrow = q <= hi;
        CF hc = hrow ? H[q * r + j0] : CF{0.f, 0.f};
        CF qc = Q[q * r + l];
        for (int j = l; j < hi; ++j) {
          const float c = cs[j];
          const CF s = sn[j];
          if (hrow && j >= j0) {
            const CF h2 = H[q * r + j + 1];
            H[q * r + j] = cadd(cscale(hc, c), cmul(h2, cconj(s)));
            hc = csub(cscale(h2, c), cmul(hc, s));
          }
          const CF q2 = Q[q * r + j + 1];
          Q[q * r + j] = cadd(cscale(qc, c), cmul(q2, cconj(s)));
          qc = csub(cscale(q2, c), cmul(qc, s));
        }
        if (hrow) H[q * r + hi] = hc;
        Q[q * r + hi] = qc;
      }
      __syncwarp();
    } else {
      for (int j = l; j < hi; ++j) {
        const CF a = H[j * r + j], b = H[(j + 1) * r + j];
        float c;
        CF s;
        givens32(a, b, c, s);
        __syncwarp();
        for (int q = j + lane; q < r; q += 32) {
          const CF h1 = H[j * r + q], h2 = H[(j + 1) * r + q];
          H[j * r + q] = cadd(cscale(h1, c), cmul(s, h2));
          H[(j + 1) * r + q] = csub(cscale(h2, c), cmul(cconj(s), h1));
        }
        if (lane == 0) {
          cs[j] = c;
          sn[j] = s;
        }
        __syncwarp();
      }
      for (int j = l; j < hi; ++j) {
        const float c = cs[j];
        const CF s = sn[j];
        for (int q = lane; q < r + (j + 2); q += 32) {
          CF* M = (q < j + 2) ? H : Q;
          const int row = (q < j + 2) ? q : q - (j + 2);
          if (q >= j + 2 && row >= r) continue;
          const CF h1 = M[row * r + j], h2 = M[row * r + j + 1];
          M[row * r + j] = cadd(cscale(h1, c), cmul(h2, cconj(s)));
          M[row * r + j + 1] = csub(cscale(h2, c), cmul(h1, s));
        }
        __syncwarp();
      }
    }
    for (int q = l + lane; q <= hi; q += 32) H[q * r + q] = cadd(H[q * r + q], mu);
    __syncwarp();
  }
  __syncwarp();
  float tnorm = 0.f;
  for (int idx = lane; idx < r * r; idx += 32) {
    const int i = idx / r, j = idx - i * r;
    if (j >= i) tnorm = fmaxf(tnorm, cabs(H[idx]));
  }
  tnorm = warp_max_f(tnorm);
  const float small = fmaxf(kEps32 * tnorm, FLT_MIN);
  // right eigenvectors: (T - l_k) y = 0 with y_k = 1, y_{>k} = 0; w = Q y
  for (int k = lane; k < r; k += 32) {
    CF* y = ycol + k * r;
    const CF lk = H[k * r + k];
    for (int i = k + 1; i < r; ++i) y[i] = {0.f, 0.f};
    y[k] = {1.f, 0.f};
    for (int i = k - 1; i >= 0; --i) {
      CF s = {0.f, 0.f};
      for (int j = i + 1; j <= k; ++j) s = cadd(s, cmul(H[i * r + j], y[j]));
      CF den = csub(H[i * r + i], lk);
      if (cabs(den) < small) den = {small, 0.f};
      y[i] = cdiv(cscale(s, -1.f), den);
    }
    float nn = 0.f;
    for (int q = 0; q < r; ++q) {
      CF w = {0.f, 0.f};
      for (int i = 0; i <= k; ++i) w = cadd(w, cmul(Q[q * r + i], y[i]));
      W[q * r + k] = w;
      nn += cabs2(w);
    }
    const float inv = 1.f / sqrtf(nn);
    for (int q = 0; q < r; ++q) W[q * r + k] = cscale(W[q * r + k], inv);
  }
  __syncwarp();
  // left eigenvectors: x^H T = l_k x^H with x_k = 1, x_{<k} = 0; u = Q x
  for (int k = lane; k < r; k += 32) {
    CF* x = ycol + k * r;
    const CF lk = H[k * r + k];
    for (int i = 0; i < k; ++i) x[i] = {0.f, 0.f};
    x[k] = {1.f, 0.f};
    for (int i = k + 1; i < r; ++i) {
      // column i of T^H x = conj(l_k) x: sum_{j<=i} conj(T[j][i]) x_j = conj(l_k) x_i
      CF s = {0.f, 0.f};
      for (int j = k; j < i; ++j) s = cadd(s, cmul(cconj(H[j * r + i]), x[j]));
      CF den = csub(cconj(H[i * r + i]), cconj(lk));
      if (cabs(den) < small) den = {small, 0.f};
      x[i] = cdiv(cscale(s, -1.f), den);
    }
    float nn = 0.f;
    for (int q = 0; q < r; ++q) {
      CF u = {0.f, 0.f};
      for (int i = k; i < r; ++i) u = cadd(u, cmul(Q[q * r + i], x[i]));
      U[q * r + k] = u;
      nn += cabs2(u);
    }
    const float inv = 1.f / sqrtf(nn);
    for (int q = 0; q < r; ++q) U[q * r + k] = cscale(U[q * r + k], inv);
  }
  __syncwarp();
  return ok;
}

// Shared-memory plan (dynamic), in 8-byte units.
struct SmemPlan {
  int a_in_smem;
  int rr_in_smem;
  int eig_in_smem;
  int inv_in_smem;       // inverse-iteration LU, Ritz scratch and vectors Z in shared memory
  int rr_dim;            // Rayleigh-Ritz size limit: r plus the cluster extension
  int64_t P, vec_units, rr_units, big_units, inv_units;
};

// Dynamic shared memory the plan may use (8-byte units): the SM's 227 KiB
// less the kernel's static arrays, with margin.
constexpr int64_t kSmemDynUnits = (220 * 1024) / 8;

__host__ __device__ inline SmemPlan smem_plan(int p, int r) {
  SmemPlan s;
  s.P = (p + 3) & ~3;
  // d, e, vs, pv, wv, lam (df64) + part (one df64 per thread) + d32, e2_32 (float) + 32 df64 scalars
  s.vec_units = 6 * s.P + kThreads + s.P + 32;
  s.rr_dim = (r + kClusterExt < p) ? r + kClusterExt : p;
  s.rr_in_smem = (s.rr_dim <= kRRMax);
  s.rr_units = s.rr_in_smem ? 2 * (int64_t)s.rr_dim * s.rr_dim : 0;
  // the tridiagonalisation's workspace (phase 1 only) shares its region with
  // the inverse iteration's working set (phase 3 on)
  const int64_t tri = (int64_t)kTriUnitsPerP * s.P + 2 * kWarps;
  s.a_in_smem = (p <= kSmemMaxP) && (s.vec_units + s.rr_units + (int64_t)p * p + tri <= kSmemDynUnits);
  s.eig_in_smem = (r <= kEigMaxR);
  const int64_t a = s.a_in_smem ? (int64_t)p * p : 0;
  const int64_t g = s.eig_in_smem ? (int64_t)5 * r * r : 0;   // H, Q, W, U, y (complex float)
  s.big_units = a > g ? a : g;
  // the inverse iteration's working set (per vector: LU 5p, Ritz scratch p,
  // the vector p) on chip when it fits: its tridiagonal recurrences are
  // chains of dependent loads and stores
  const int64_t inv = (int64_t)s.rr_dim * 7 * p;
  s.inv_in_smem = (s.vec_units + s.rr_units + s.big_units + (inv > tri ? inv : tri) <= kSmemDynUnits);
  s.inv_units = s.inv_in_smem ? (inv > tri ? inv : tri) : tri;
  return s;
}

__device__ __forceinline__ void modes_small_body(const ModesArgs& a, const ModesLayout& L) {
  extern __shared__ double smem_d[];
  __shared__ dd red[kWarps];
  __shared__ float cs[SDMD_MAX_M];
  __shared__ CF sn[SDMD_MAX_M];
  __shared__ int ord[SDMD_MAX_M];
  __shared__ dd coef[SDMD_MAX_M];
  __shared__ int sh_int[4];
  __shared__ float sh_f[4];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  WS w = carve(a.ws, L);
  // embed_cx: the 2pc x 2pc real embedding of a complex pc x pc G_X
  const int m = a.m, pc = a.c - 1, p = a.embed_cx ? 2 * pc : pc;
  const int rw = min(a.r_req, p);
  const SmemPlan plan = smem_plan(p, a.r_req);
  const int64_t P = plan.P;
  dd* base = reinterpret_cast<dd*>(smem_d);
  dd* d = base;
  dd* e = d + P;
  dd* vs = e + P;
  dd* pv = vs + P;
  dd* wv = pv + P;
  dd* lam = wv + P;
  dd* part = lam + P;
  float* d32 = reinterpret_cast<float*>(part + kThreads);
  float* e2_32 = d32 + P;
  dd* sc = reinterpret_cast<dd*>(e2_32 + P);
  dd* rrH = plan.rr_in_smem ? base + plan.vec_units : w.Y;
  dd* rrR = rrH + (int64_t)plan.rr_dim * plan.rr_dim;
  dd* big = base + plan.vec_units + plan.rr_units;
  dd* A = plan.a_in_smem ? big : w.Ad;
  // inverse iteration: LU factors + Ritz scratch (rr_dim x 6p) and the vectors
  // Z (rr_dim x p; later the eigenvectors, then vsi)
  dd* inv_base = big + plan.big_units;
  dd* LU = plan.inv_in_smem ? inv_base : w.lu;
  dd* Z = plan.inv_in_smem ? inv_base + (int64_t)plan.rr_dim * 6 * p : w.Z;
  if (tid == 0) w.clk[0] = clock64();

  // ---- 0. scale (exact power of two from the largest diagonal), gather, convert
  if (warp == 0) {
    int ex = -1000;
    for (int i = lane; i < p; i += 32) {
      const int si = (a.start + i) % m;
      int xe;
      if (a.embed_cx) {   // complex G: the real diagonal (as the complex kernel scales)
        const double g = static_cast<const double2*>(a.G)[(int64_t)((a.start + i % pc) % m) * m + (a.start + i % pc) % m].x;
        const int bits = (__double2hiint(g) >> 20) & 0x7ff;
        xe = (g > 0.0 && bits > 0) ? bits - 1023 : -1000;
      } else if (a.g_is_int) {
        const long long g = static_cast<const long long*>(a.G)[(int64_t)si * m + si];
        xe = (g > 0) ? 63 - __clzll(g) : -1000;
      } else {
        const double g = static_cast<const double*>(a.G)[(int64_t)si * m + si];
        const int bits = (__double2hiint(g) >> 20) & 0x7ff;
        xe = (bits > 0) ? bits - 1023 : -1000;
      }
      ex = max(ex, xe);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ex = max(ex, __shfl_xor_sync(0xffffffffu, ex, o));
    if (lane == 0) sh_int[0] = (ex == -1000) ? 0 : ex + 1;   // G / 2^s has max diag in [0.5, 1)
  }
  __syncthreads();
  const int s_exp = sh_int[0];
  // complex G_X = B0 + i B1 embedded as [[B0, -B1], [B1, B0]] (symmetric:
  // G_X is Hermitian, its diagonal imaginary parts taken as zero)
  for (int idx = tid; a.embed_cx && idx < p * p; idx += kThreads) {
    const int i = idx / p, j = idx - i * p;
    const int bi = i >= pc, bj = j >= pc, ii = i - bi * pc, jj = j - bj * pc;
    const double2 g = static_cast<const double2*>(a.G)[(int64_t)((a.start + ii) % m) * m + (a.start + jj) % m];
    const double v = (bi == bj) ? g.x : ((ii == jj) ? 0.0 : (bi ? g.y : -g.y));
    const dd gv = dd_from_double(v);
    A[idx] = {ldexpf(gv.hi, -s_exp), ldexpf(gv.lo, -s_exp)};
  }
  // G_X and G_XY entries, kGatherBatch per thread loaded before any is
  // converted and stored (the stores could alias G for the compiler, so a
  // plain loop waits a full memory latency per entry; beside a bandwidth-bound
  // pass that latency is long)
  constexpr int kGatherBatch = 8;
  for (int base = tid; !a.embed_cx && base < p * p; base += kThreads * kGatherBatch) {
    int64_t raw_x[kGatherBatch], raw_xy[kGatherBatch];   // the G words (int64 or the bits of an FP64)
#pragma unroll
    for (int u = 0; u < kGatherBatch; ++u) {
      const int idx = base + u * kThreads;
      raw_x[u] = raw_xy[u] = 0;
      if (idx < p * p) {
        const int i = idx / p, j = idx - i * p;
        int si = a.start + i, sj = a.start + j;
        if (si >= m) si -= m;
        if (sj >= m) sj -= m;
        const int sj1 = (sj + 1 == m) ? 0 : sj + 1;
        const long long* G = static_cast<const long long*>(a.G);
        raw_x[u] = G[(int64_t)si * m + sj];
        raw_xy[u] = G[(int64_t)si * m + sj1];
      }
    }
#pragma unroll
    for (int u = 0; u < kGatherBatch; ++u) {
      const int idx = base + u * kThreads;
      if (idx < p * p) {
        const dd gx = a.g_is_int ? dd_from_ll(raw_x[u]) : dd_from_double(__longlong_as_double(raw_x[u]));
        const dd gxy = a.g_is_int ? dd_from_ll(raw_xy[u]) : dd_from_double(__longlong_as_double(raw_xy[u]));
        A[idx] = {ldexpf(gx.hi, -s_exp), ldexpf(gx.lo, -s_exp)};
        w.GXYd[idx] = {ldexpf(gxy.hi, -s_exp), ldexpf(gxy.lo, -s_exp)};
      }
    }
  }
  __syncthreads();
  if (tid == 0) w.clk[1] = clock64();

  // ---- 1. tridiagonalise G_X (df64)
  tridiagonalize(A, p, d, e, inv_base, P);
  if (tid == 0) w.clk[2] = clock64();

  // ---- 2. FP32 multisection for the rw largest eigenvalues of T
  for (int i = tid; i < p; i += kThreads) {
    d32[i] = d[i].hi;
    e2_32[i] = (i + 1 < p) ? e[i].hi * e[i].hi : 0.f;
  }
  __syncthreads();
  if (tid == 0) {
    float gl = 0.f, gu = 0.f, em = 0.f;
    for (int i = 0; i < p; ++i) {
      const float rad = ((i > 0) ? fabsf(e[i - 1].hi) : 0.f) + ((i + 1 < p) ? fabsf(e[i].hi) : 0.f);
      gl = (i == 0) ? d32[0] - rad : fminf(gl, d32[i] - rad);
      gu = (i == 0) ? d32[0] + rad : fmaxf(gu, d32[i] + rad);
      if (i + 1 < p) em = fmaxf(em, e2_32[i]);
    }
    const float tn = fmaxf(fabsf(gl), fabsf(gu));
    sh_f[0] = gl - 4.f * kEps32 * tn * p - FLT_MIN;
    sh_f[1] = gu + 4.f * kEps32 * tn * p + FLT_MIN;
    sh_f[2] = tn;
    sh_f[3] = FLT_MIN * fmaxf(1.f, em) * 4.f;
  }
  __syncthreads();
  const float tnorm = sh_f[2];
  // eigenvalue number i (descending) of T to FP32 resolution, one warp
  auto multisect = [&](int i) -> float {
    const int target = p - 1 - i;
    float lo = sh_f[0], hi = sh_f[1];
    for (int round = 0; round < kMsRounds; ++round) {
      if (hi - lo <= 2.f * kEps32 * fmaxf(fabsf(lo), fabsf(hi)) + sh_f[3]) break;
      const float x = lo + (hi - lo) * (float)(lane + 1) / 33.f;
      const int cnt = sturm32(d32, e2_32, p, x, sh_f[3]);
      const unsigned above = __ballot_sync(0xffffffffu, cnt > target);
      const int f = above ? __ffs(above) - 1 : 32;
      const float xf = lo + (hi - lo) * (float)(f + 1) / 33.f;
      const float xp = lo + (hi - lo) * (float)f / 33.f;
      if (f < 32) hi = xf;
      lo = (f == 0) ? lo : xp;
    }
    return 0.5f * (lo + hi);
  };
  // the last pass's idle warps take the eigenvalues after the rw-th (the
  // cluster test below reads them instead of running more multisections)
  const int npre = min(p, ((rw + kWarps - 1) / kWarps) * kWarps);
  for (int i = warp; i < npre; i += kWarps) {
    const float v = multisect(i);
    if (lane == 0) lam[i] = dd_make(v);
  }
  __syncthreads();
  // A cluster that the FP32 values cannot resolve and that straddles the last
  // requested eigenvalue is taken in whole (up to kClusterExt more), so the
  // df64 inverse iteration and Rayleigh-Ritz below see its whole subspace;
  // only the rw largest Ritz pairs are kept. Eigenvalues under the rank
  // floor are dropped later anyway and do not extend the set.
  if (warp == 0) {
    int rwe = rw;
    const int cap = (rw + kClusterExt < p) ? rw + kClusterExt : p;
    const float floor_v = lam[0].hi * (float)(kRankRtol * (double)p * kEps);
    while (rwe < cap) {
      const float last = lam[rwe - 1].hi;
      if (!(last > floor_v)) break;
      const float v = (rwe < npre) ? lam[rwe].hi : multisect(rwe);
      if (fabsf(v - last) > 8.f * kEps32 * tnorm) break;
      if (lane == 0) lam[rwe] = dd_make(v);
      __syncwarp();
      ++rwe;
    }
    if (lane == 0) sh_int[2] = rwe;
  }
  __syncthreads();
  const int rwe = (rw > 0) ? sh_int[2] : 0;
  for (int i = tid; i < rwe; i += kThreads) pv[i] = lam[i];   // the FP32 values, for phase 3'
  if (tid == 0) w.clk[3] = clock64();

  // ---- 3. df64 inverse iteration + Gram-Schmidt + Rayleigh-Ritz, twice:
  //         round 0 shifts are the FP32 eigenvalues, round 1 shifts are the
  //         round-0 Ritz values (df64-accurate), which converges in one or two
  //         solves even for eigenvalues much closer than eps32 * |T|
  const float tiny = fmaxf(1e-13f * tnorm, FLT_MIN);
  for (int round = 0; round < 3; ++round) {
    if (round == 2) {
      // ---- 3'. missed-eigenvalue check: inverse iteration converges to the
      //          eigenvectors nearest its shifts, and inside a cluster below
      //          the FP32 multisection's resolution (eps32 |T|) those need not
      //          be the largest. A df64 Sturm count of the eigenvalues above
      //          the smallest kept Ritz value (less 1e-13 |T|) that exceeds rw
      //          sends the wanted eigenvalues through a df64 multisection
      //          (warp per eigenvalue, 33 points per round, bracketed by the
      //          FP32 value or else by Gershgorin) and one more round runs
      //          with those shifts.
      if (tid == 0) {
        const int below = sturm_below_dd(d, e, p, dd_sub(lam[rw - 1], dd_make(1e-13f * tnorm)), sh_f[3]);
        sh_int[3] = (p - below > rw) ? 1 : 0;
      }
      __syncthreads();
      // the embedding of a complex window leaves a failed check to the complex
      // kernel's FP64 Jacobi: for modes that far below lambda_1 its FP64
      // backward error keeps A~'s eigenvalues within 1e-9, df64 does not
      if (!sh_int[3] || a.embed_cx) break;
      for (int i = warp; i < rwe; i += kWarps) {
        const int target = p - 1 - i;
        const float W = 32.f * kEps32 * tnorm + sh_f[3];
        dd lo = dd_sub(pv[i], dd_make(W)), hi = dd_add(pv[i], dd_make(W));
        const int cb = (lane < 2) ? sturm_below_dd(d, e, p, lane ? hi : lo, sh_f[3]) : 0;
        const int c_lo = __shfl_sync(0xffffffffu, cb, 0), c_hi = __shfl_sync(0xffffffffu, cb, 1);
        if (!(c_lo <= target && c_hi >= target + 1)) {
          lo = dd_make(sh_f[0]);
          hi = dd_make(sh_f[1]);
        }
        for (int rnd = 0; rnd < 12; ++rnd) {
          const dd wd = dd_sub(hi, lo);
          if (wd.hi <= 1e-14f * tnorm) break;
          const dd x = dd_add(lo, dd_mul_f(wd, (float)(lane + 1) / 33.f));
          const int cnt = sturm_below_dd(d, e, p, x, sh_f[3]);
          const unsigned above = __ballot_sync(0xffffffffu, cnt > target);
          const int f = above ? __ffs(above) - 1 : 32;
          const dd xf = {__shfl_sync(0xffffffffu, x.hi, f & 31), __shfl_sync(0xffffffffu, x.lo, f & 31)};
          const dd xp = {__shfl_sync(0xffffffffu, x.hi, (f + 31) & 31), __shfl_sync(0xffffffffu, x.lo, (f + 31) & 31)};
          if (f < 32) hi = xf;
          if (f > 0) lo = xp;
        }
        if (lane == 0) lam[i] = dd_scale(dd_add(lo, hi), 0.5f);
      }
      __syncthreads();
    }
    const float sep = (round == 0) ? 2.f * kEps32 * tnorm : 1e-12f * tnorm;
    // vector i on lane i / 8 of warp i % 8: the factorisations and solves are
    // serial recurrences, so they are spread over all warps' issue slots
    for (int i = warp + kWarps * lane; i < rwe; i += kThreads) {
      dd* u0 = LU + (int64_t)i * 5 * p;
      dd shift = lam[i];
      for (int q = 0; q < i; ++q)    // (numerically) equal shifts: separate them slightly
        if (fabsf(lam[q].hi - shift.hi) <= sep) shift = dd_sub(shift, dd_make(sep));
      tri_lu_dd(d, e, p, shift, tiny, u0, u0 + p, u0 + 2 * p, u0 + 3 * p, u0 + 4 * p);
    }
    // rounds 0 and 2 start from fixed pseudo-random vectors: round 1 refines
    // round 0's, but round 2 follows a check that found an eigenvector round
    // 1 missed, whose component in round 1's vectors is at rounding level
    if (round != 1) {
      for (int idx = tid; idx < rwe * p; idx += kThreads) {
        const int i = idx / p, j = idx - i * p;
        Z[idx] = dd_make(1.f + 0.1f * (float)(((j + 1) * 7919 + (i + 1) * 104729) % 97) / 97.f);
      }
    }
    __syncthreads();
    for (int it = 0; it < kInvIters; ++it) {
      for (int i = warp + kWarps * lane; i < rwe; i += kThreads) {
        dd* u0 = LU + (int64_t)i * 5 * p;
        tri_solve_dd(p, u0, u0 + p, u0 + 2 * p, u0 + 3 * p, u0 + 4 * p, Z + (int64_t)i * p);
      }
      __syncthreads();
      cgs_dd(Z, rwe, p, (it + 1 == kInvIters) ? 2 : 1, coef, vs, red, sc);
    }
    rayleigh_ritz(Z, rwe, p, d, e, rrH, rrR, LU + (int64_t)rwe * 5 * p, lam, sc, ord);
  }
  if (tid == 0) w.clk[4] = clock64();

  // ---- 4. back-transform: v = H_0 H_1 ... H_{p-3} z  (half a warp per vector)
  for (int i0 = 2 * warp; i0 < rw; i0 += 2 * kWarps) {
    const int i = i0 + (lane >> 4), hl = lane & 15;
    const bool live = i < rw;
    dd* z = Z + (int64_t)(live ? i : i0) * p;
    for (int k = p - 3; k >= 0; --k) {
      const int Lk = p - k - 1;
      const dd* v = A + (int64_t)(k + 1) * p + k;   // down column k
      float ss = 0.f, sc2 = 0.f;
      if (live)
        for (int j = hl; j < Lk; j += 16) dot2_acc(ss, sc2, v[(int64_t)j * p], z[k + 1 + j]);
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {   // within each half warp
        const float so = __shfl_xor_sync(0xffffffffu, ss, o), co = __shfl_xor_sync(0xffffffffu, sc2, o);
        const dd q = two_sum(ss, so);
        ss = q.hi;
        sc2 = (sc2 + co) + q.lo;
      }
      const dd s = dd_scale(quick_two_sum(ss, sc2), -2.f);
      if (live)
        for (int j = hl; j < Lk; j += 16) z[k + 1 + j] = dd_fma(s, v[(int64_t)j * p], z[k + 1 + j]);
      __syncwarp();
    }
  }
  __syncthreads();
  if (tid == 0) w.clk[5] = clock64();
  if (a.embed_cx) {
    // hand the K = rw / 2 complex eigenpairs to the complex kernel: lambda_k
    // (unscaled, FP64) at the start of its A~ array, x_k = u + i v from the
    // pair's first Ritz vector [u; v] (unit norm) in its sorted-V array
    double* cxb = a.ws + L.cx;
    double* lam_h = cxb + 2 * 3 * (int64_t)pc * pc;   // A~ region
    double* vec_h = cxb + 2 * 5 * (int64_t)pc * pc;   // sorted-V region: vector k at k pc
    const int K = rw / 2;
    // Missed-eigenvalue check: inverse iteration finds the eigenvectors
    // nearest its shifts, and in a cluster below the FP32 multisection's
    // resolution (eps32 |T|) those need not be the largest. A df64 Sturm
    // count on T of the eigenvalues above the smallest kept Ritz value (less
    // 1e-13 |T|) must not exceed rw; lam_h[K] = 1 accepts the handoff, 0
    // sends the complex kernel to its Jacobi sweeps.
    if (tid == 0) {
      const int below = sturm_below_dd(d, e, p, dd_sub(lam[rw - 1], dd_make(1e-13f * tnorm)), sh_f[3]);
      lam_h[K] = (p - below <= rw) ? 1.0 : 0.0;
    }
    for (int k = tid; k < K; k += kThreads) lam_h[k] = ldexp(dd_to_double(lam[2 * k]), s_exp);
    for (int idx = tid; idx < K * pc; idx += kThreads) {
      const int k = idx / pc, i = idx - k * pc;
      const dd* z = Z + (int64_t)(2 * k) * p;
      vec_h[2 * idx] = dd_to_double(z[i]);
      vec_h[2 * idx + 1] = dd_to_double(z[pc + i]);
    }
    if (tid == 0) w.clk[6] = w.clk[7] = w.clk[8] = clock64();
    return;
  }

  // ---- 5. rank, sigma, V (FP64 out), vsi = V Sigma^-1 (df64, scaled units)
  if (tid == 0) {
    int k = 0;
    bool finite = true;                // a breakdown is reported, not returned as rank 0
    for (int i = 0; i < rw; ++i) finite = finite && isfinite(dd_to_double(lam[i]));
    if (!finite) atomicOr(a.status, kDevRank);
    const double lam0 = (rw > 0) ? dd_to_double(lam[0]) : 0.0;
    if (lam0 > 0.0) {
      const double thr = lam0 * kRankRtol * (double)p * kEps;
      while (k < rw && dd_to_double(lam[k]) > thr) ++k;
    }
    sh_int[1] = k;
  }
  __syncthreads();
  const int re = sh_int[1];
  for (int i = tid; i < a.r_req; i += kThreads) {
    w.sig[i] = (i < re) ? sqrt(ldexp(dd_to_double(lam[i]), s_exp)) : 0.0;
    if (i < re) coef[i] = dd_div(dd_make(1.f), dd_sqrt(lam[i]));
  }
  __syncthreads();
  for (int idx = tid; idx < a.r_req * p; idx += kThreads) {
    const int i = idx / p;
    const dd z = (i < re) ? Z[idx] : dd{0.f, 0.f};
    w.V[idx] = dd_to_double(z);
    if (i < re) Z[idx] = dd_mul(z, coef[i]);
  }
  __syncthreads();

  // ---- 6. A~ = vsi^T G_XY vsi (df64; independent of the scaling). G_XY is
  //         staged into A's region (free after the back-transform) and Y, A~
  //         into the inverse iteration's (free after phase 3) when on chip.
  const dd* GXY = w.GXYd;
  if (plan.a_in_smem) {
    for (int idx = tid; idx < p * p; idx += kThreads) big[idx] = w.GXYd[idx];
    GXY = big;
    __syncthreads();
  }
  dd* Yb = plan.inv_in_smem ? LU : w.Y;
  dd* At = plan.inv_in_smem ? LU + (int64_t)re * p : w.lu;   // re x re df64
  for (int idx = tid; idx < re * p; idx += kThreads) {
    const int k = idx / p, row = idx - k * p;
    const dd* g = GXY + (int64_t)row * p;
    const dd* v = Z + (int64_t)k * p;
    dd s0 = {0.f, 0.f}, s1 = {0.f, 0.f};
    int b = 0;
    for (; b + 1 < p; b += 2) {
      s0 = dd_fma(g[b], v[b], s0);
      s1 = dd_fma(g[b + 1], v[b + 1], s1);
    }
    if (b < p) s0 = dd_fma(g[b], v[b], s0);
    Yb[idx] = dd_add(s0, s1);
  }
  __syncthreads();
  CF* Hc = plan.eig_in_smem ? reinterpret_cast<CF*>(big) : reinterpret_cast<CF*>(w.lu + (int64_t)re * re);
  CF* Qc = Hc + re * re;
  CF* Wc = Qc + re * re;
  CF* Uc = Wc + re * re;
  CF* yc = Uc + re * re;
  for (int idx = tid; idx < re * re; idx += kThreads) {
    const int k = idx / re, l = idx - k * re;
    const dd* v = Z + (int64_t)k * p;
    const dd* y = Yb + (int64_t)l * p;
    dd s = {0.f, 0.f};
    for (int b = 0; b < p; ++b) s = dd_fma(v[b], y[b], s);
    At[idx] = s;
    Hc[idx] = {s.hi, 0.f};
  }
  __syncthreads();
  if (tid == 0) w.clk[6] = clock64();

  // ---- 7. eig(A~): FP32 Schur with left and right vectors, then df64
  //         two-sided Rayleigh quotients for the eigenvalues
  if (warp == 0 && re > 0) {
    const bool ok = warp_eig32(Hc, Qc, Wc, Uc, yc, re, cs, sn);
    if (!ok && lane == 0) atomicOr(a.status, kDevRank);
  }
  __syncthreads();
  double* lam_tmp = reinterpret_cast<double*>(w.Y);   // provisional order (Y is free)
  for (int k = tid; k < re; k += kThreads) {
    // lambda_k = (u^H A~ w) / (u^H w), A~ real df64, u and w promoted exactly
    dd nre = {0.f, 0.f}, nim = {0.f, 0.f}, dre = {0.f, 0.f}, dim = {0.f, 0.f};
    for (int i = 0; i < re; ++i) {
      dd awr = {0.f, 0.f}, awi = {0.f, 0.f};
      for (int j = 0; j < re; ++j) {
        const CF wj = Wc[j * re + k];
        awr = dd_fma(At[i * re + j], dd_make(wj.re), awr);
        awi = dd_fma(At[i * re + j], dd_make(wj.im), awi);
      }
      const CF ui = Uc[i * re + k];
      const CF wi = Wc[i * re + k];
      // conj(u_i) (aw_i) = (ur ar + ui ai) + i (ur ai - ui ar)
      nre = dd_fma(dd_make(ui.re), awr, dd_fma(dd_make(ui.im), awi, nre));
      nim = dd_sub(dd_fma(dd_make(ui.re), awi, nim), dd_mul(dd_make(ui.im), awr));
      dre = dd_add(dre, dd_add(two_prod(ui.re, wi.re), two_prod(ui.im, wi.im)));
      dim = dd_add(dim, dd_sub(two_prod(ui.re, wi.im), two_prod(ui.im, wi.re)));
    }
    const zd lk = zd_div({nre, nim}, {dre, dim});
    lam_tmp[2 * k] = dd_to_double(lk.re);
    lam_tmp[2 * k + 1] = dd_to_double(lk.im);
  }
  __syncthreads();
  if (tid == 0) {
    for (int k = 0; k < re; ++k) ord[k] = k;
    for (int k = 0; k < re; ++k) {
      int best = k;
      for (int q = k + 1; q < re; ++q) {
        const double br = lam_tmp[2 * ord[best]], bi = lam_tmp[2 * ord[best] + 1];
        const double qr = lam_tmp[2 * ord[q]], qi = lam_tmp[2 * ord[q] + 1];
        const double mb = br * br + bi * bi, mq = qr * qr + qi * qi;
        if (mq > mb || (mq == mb && atan2(qi, qr) < atan2(bi, br))) best = q;
      }
      const int t = ord[k];
      ord[k] = ord[best];
      ord[best] = t;
    }
  }
  __syncthreads();
  for (int k = tid; k < a.r_req; k += kThreads) {
    w.lamout[2 * k] = (k < re) ? lam_tmp[2 * ord[k]] : 0.0;
    w.lamout[2 * k + 1] = (k < re) ? lam_tmp[2 * ord[k] + 1] : 0.0;
  }
  __syncthreads();
  if (tid == 0) w.clk[7] = clock64();

  // ---- 8. M = vsi W (df64 accumulation of FP32 W), FP32 out, scaled back
  const int R = a.r_req;
  const float unscale = (float)exp2(-0.5 * s_exp);
  for (int idx = tid; idx < p * R; idx += kThreads) {
    const int row = idx / R, k = idx - row * R;
    dd sr = {0.f, 0.f}, si = {0.f, 0.f};
    if (k < re) {
      const int kk = ord[k];
      for (int l = 0; l < re; ++l) {
        const dd z = Z[(int64_t)l * p + row];
        const CF wv2 = Wc[l * re + kk];
        sr = dd_fma(z, dd_make(wv2.re), sr);
        si = dd_fma(z, dd_make(wv2.im), si);
      }
    }
    w.Mf[2 * idx] = (sr.hi + sr.lo) * unscale;
    w.Mf[2 * idx + 1] = (si.hi + si.lo) * unscale;
  }

  // ---- 9. amplitudes b = (W Lambda)^-1 alpha_1 (Sec. 3.3, Eq. 14a-e) with
  //         alpha_1 = Sigma V^H e_1 (the POD coefficients of x_1). The left
  //         eigenvectors give W^-1 = diag(1 / u_k^H w_k) U^H, so
  //         b_k = u_k^H alpha_1 / (lambda_k u_k^H w_k): O(r^2), no solve.
  //         Then the background index argmin_k |log lambda_k| (Algorithm 3,
  //         principal log).
  for (int k = tid; k < R; k += kThreads) {
    double br = 0.0, bi = 0.0;
    if (k < re) {
      const int kk = ord[k];
      double nr = 0.0, ni = 0.0, dr = 0.0, di = 0.0;
      for (int i = 0; i < re; ++i) {
        const CF u = Uc[i * re + kk], wv = Wc[i * re + kk];
        const double a1 = w.sig[i] * w.V[(int64_t)i * p];   // G_X real: V real
        nr += (double)u.re * a1;                            // conj(u_i) alpha_1[i]
        ni -= (double)u.im * a1;
        dr += (double)u.re * wv.re + (double)u.im * wv.im;  // conj(u_i) w_i
        di += (double)u.re * wv.im - (double)u.im * wv.re;
      }
      const double lr = w.lamout[2 * k], li = w.lamout[2 * k + 1];
      const double er = lr * dr - li * di, ei = lr * di + li * dr;
      const double q = er * er + ei * ei;
      if (q > 0.0) {
        br = (nr * er + ni * ei) / q;
        bi = (ni * er - nr * ei) / q;
      } else {
        atomicOr(a.status, kDevRank);
      }
    }
    w.bamp[2 * k] = br;
    w.bamp[2 * k + 1] = bi;
  }
  if (tid == 0) {
    int best = -1;
    double bv = 0.0;
    for (int k = 0; k < re; ++k) {
      const double lr = w.lamout[2 * k], li = w.lamout[2 * k + 1];
      const double lm = 0.5 * log(lr * lr + li * li), th = atan2(li, lr);
      const double v = lm * lm + th * th;
      if (best < 0 || v < bv) {
        best = k;
        bv = v;
      }
    }
    w.bamp[2 * (a.ws_m - 1 > 1 ? a.ws_m - 1 : 1)] = (double)best;   // fixed slot for any window length
  }
  __syncthreads();
  if (tid == 0) {
    *a.r_dev = re;
    w.clk[8] = clock64();
  }
}

__global__ void __launch_bounds__(kThreads, 1) modes_small_kernel(ModesArgs a, ModesLayout L) { modes_small_body(a, L); }

// One CTA per job: the eigensolvers of up to kMaxModesJobs windows (of any
// length) in one launch, each CTA on its own handle's G and workspace.
__global__ void __launch_bounds__(kThreads, 1) modes_batch_kernel(ModesBatch b) {
  const ModesArgs a = b.job[blockIdx.x];
  modes_small_body(a, modes_layout(a.ws_m));
}


// ------------------------------------------------------- complex windows --
// The small-matrix part of exact DMD for complex snapshots (dense complex64
// or Fourier-sparse handles: G is Hermitian complex128), Algorithms 1-2 with
// complex V: FP64 cyclic Jacobi for G_X (parallel round-robin rotations, a
// bounded number of sweeps), rank rule, sigma, vsi = V Sigma^-1, A~ = vsi^H
// G_XY vsi (FP64), eig(A~) by the FP32 complex Schur of phase 7 refined by
// FP64 two-sided Rayleigh quotients, M = vsi W, amplitudes and the
// background index as for real windows. Outputs go to the same workspace
// arrays (sig, lamout, Mf, bamp, r_dev); V (complex) to the cx region.
constexpr int kCThreads = 512;
constexpr int kCWarps = kCThreads / 32;
constexpr int kJacobiMaxSweeps = 40;

struct C64d {
  double re, im;
};
__device__ __forceinline__ C64d zmul(C64d a, C64d b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ C64d zcmul(C64d a, C64d b) {   // conj(a) b
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}

__device__ double block_sum_c(double v, double* red) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < kCWarps; ++w) t += red[w];
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(kCThreads, 1) modes_complex_kernel(ModesArgs a, ModesLayout L) {
  __shared__ double red[kCWarps];
  __shared__ double rc[SDMD_MAX_M / 2], rs[SDMD_MAX_M / 2], rpr[SDMD_MAX_M / 2], rpi[SDMD_MAX_M / 2];
  __shared__ int ri[SDMD_MAX_M / 2], rj[SDMD_MAX_M / 2];
  __shared__ int ord[SDMD_MAX_M];
  __shared__ double lam_s[SDMD_MAX_M];
  __shared__ float cs[SDMD_MAX_M];
  __shared__ CF sn[SDMD_MAX_M];
  __shared__ int sh_int[4];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m = a.m, p = a.c - 1;
  const int R = a.r_req;
  double* ws = a.ws;
  C64d* Ac = reinterpret_cast<C64d*>(ws + L.cx);   // p x p, row-major (later G_XY vsi)
  C64d* Vc = Ac + (int64_t)p * p;                  // p x p: V[i][k], column k = eigenvector k
  C64d* Bc = Vc + (int64_t)p * p;                  // G_XY
  C64d* At = Bc + (int64_t)p * p;                  // re x re
  C64d* vsi = At + (int64_t)p * p;                 // p x R
  C64d* Vo = vsi + (int64_t)p * p;                 // R vectors of length p (sorted V)
  const double2* G = static_cast<const double2*>(a.G);

  // ---- 0. scale by a power of two (largest diagonal), gather G_X, G_XY
  if (warp == 0) {
    int ex = -1000;
    for (int i = lane; i < p; i += 32) {
      const int si = (a.start + i) % m;
      const double g = G[(int64_t)si * m + si].x;
      const int bits = (__double2hiint(g) >> 20) & 0x7ff;
      ex = max(ex, (g > 0.0 && bits > 0) ? bits - 1023 : -1000);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ex = max(ex, __shfl_xor_sync(0xffffffffu, ex, o));
    if (lane == 0) sh_int[0] = (ex == -1000) ? 0 : ex + 1;
  }
  __syncthreads();
  const int s_exp = sh_int[0];
  for (int idx = tid; idx < p * p; idx += kCThreads) {
    const int i = idx / p, j = idx - i * p;
    const int si = (a.start + i) % m, sj = (a.start + j) % m, sj1 = (a.start + j + 1) % m;
    const double2 gx = G[(int64_t)si * m + sj], gxy = G[(int64_t)si * m + sj1];
    Ac[idx] = {ldexp(gx.x, -s_exp), (i == j) ? 0.0 : ldexp(gx.y, -s_exp)};
    Bc[idx] = {ldexp(gxy.x, -s_exp), ldexp(gxy.y, -s_exp)};
    Vc[idx] = {(i == j) ? 1.0 : 0.0, 0.0};
  }
  __syncthreads();

  // ---- 1. cyclic Jacobi: A <- J^H A J, V <- V J, J = diag(1, e^{-i phi}) R
  //         with R the real rotation that zeroes |a_ij| (round-robin pairs,
  //         all disjoint pairs of a step at once)
  const int P2 = p + (p & 1);
  const int npairs = P2 / 2;
  // the handoff of the embedded solve, if it passed its missed-eigenvalue check
  const bool pre = a.cx_pre && reinterpret_cast<const double*>(At)[min(R, p)] == 1.0;
  for (int sweep = 0; !pre && sweep < kJacobiMaxSweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int idx = tid; idx < p * p; idx += kCThreads) {
      const C64d v = Ac[idx];
      const double q = v.re * v.re + v.im * v.im;
      tot += q;
      if (idx / p != idx % p) off += q;
    }
    off = block_sum_c(off, red);
    tot = block_sum_c(tot, red);
    if (!(off > 1e-30 * tot)) break;
    for (int step = 0; step < P2 - 1; ++step) {
      if (tid < npairs) {
        int u = (tid == 0) ? P2 - 1 : (step + tid) % (P2 - 1);
        int v = (step - tid + (P2 - 1)) % (P2 - 1);
        if (tid == 0) v = step;
        const int i = min(u, v), j = max(u, v);
        double c = 1.0, sv = 0.0, pr = 1.0, pim = 0.0;
        if (j < p) {
          const C64d b = Ac[(int64_t)i * p + j];
          const double ab = hypot(b.re, b.im);
          if (ab > 0.0) {
            const double al = Ac[(int64_t)i * p + i].re, de = Ac[(int64_t)j * p + j].re;
            const double tau = (de - al) / (2.0 * ab);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            sv = t * c;
            pr = b.re / ab;                   // e^{i phi}
            pim = b.im / ab;
          }
        }
        ri[tid] = i;
        rj[tid] = (j < p) ? j : -1;
        rc[tid] = c;
        rs[tid] = sv;
        rpr[tid] = pr;
        rpi[tid] = pim;
      }
      __syncthreads();
      // columns: (a_ki, a_kj) <- (a_ki c - a_kj s e^{-i phi}, a_ki s + a_kj c e^{-i phi}); also V
      for (int w = tid; w < 2 * npairs * p; w += kCThreads) {
        const int which = w / (npairs * p);
        const int rem = w - which * npairs * p;
        const int q = rem / p, k = rem - q * p;
        const int j = rj[q];
        if (j < 0) continue;
        const int i = ri[q];
        C64d* X = which ? Vc : Ac;
        const C64d xi = X[(int64_t)k * p + i], xj = X[(int64_t)k * p + j];
        const C64d em = {rpr[q], -rpi[q]};
        const C64d xje = zmul(xj, em);
        const double c = rc[q], sv = rs[q];
        X[(int64_t)k * p + i] = {c * xi.re - sv * xje.re, c * xi.im - sv * xje.im};
        X[(int64_t)k * p + j] = {sv * xi.re + c * xje.re, sv * xi.im + c * xje.im};
      }
      __syncthreads();
      // rows: (a_ik, a_jk) <- (c a_ik - s e^{i phi} a_jk, s a_ik + c e^{i phi} a_jk)
      for (int w = tid; w < npairs * p; w += kCThreads) {
        const int q = w / p, k = w - q * p;
        const int j = rj[q];
        if (j < 0) continue;
        const int i = ri[q];
        const C64d xi = Ac[(int64_t)i * p + k], xj = Ac[(int64_t)j * p + k];
        const C64d ep = {rpr[q], rpi[q]};
        const C64d xje = zmul(ep, xj);
        const double c = rc[q], sv = rs[q];
        Ac[(int64_t)i * p + k] = {c * xi.re - sv * xje.re, c * xi.im - sv * xje.im};
        Ac[(int64_t)j * p + k] = {sv * xi.re + c * xje.re, sv * xi.im + c * xje.im};
      }
      __syncthreads();
    }
  }

  // ---- 1'. (cx_pre, check passed) the eigenpairs handed over by the real
  //          df64 solver of the embedding: lambda_k at the start of the A~
  //          array, x_k in the sorted-V array; the other diagonal entries sort
  //          last, below the rank threshold
  if (pre) {
    const int K = min(R, p);
    const double* lam_h = reinterpret_cast<const double*>(At);
    for (int idx = tid; idx < p * p; idx += kCThreads) {
      const int i = idx / p, k = idx - i * p;
      Vc[idx] = (k < K) ? Vo[(int64_t)k * p + i] : C64d{(i == k) ? 1.0 : 0.0, 0.0};
    }
    for (int i = tid; i < p; i += kCThreads) Ac[(int64_t)i * p + i].re = (i < K) ? ldexp(lam_h[i], -s_exp) : -1.0;
    __syncthreads();
  }

  // ---- 2. eigenvalues (real diagonal) sorted descending, rank, sigma, V, vsi
  for (int i = tid; i < p; i += kCThreads) lam_s[i] = Ac[(int64_t)i * p + i].re;
  __syncthreads();
  if (tid == 0) {
    for (int i = 0; i < p; ++i) ord[i] = i;
    for (int i = 0; i < p; ++i) {
      int best = i;
      for (int q = i + 1; q < p; ++q)
        if (lam_s[ord[q]] > lam_s[ord[best]]) best = q;
      const int t = ord[i];
      ord[i] = ord[best];
      ord[best] = t;
    }
    const int rw = min(R, p);
    int k = 0;
    const double l0 = lam_s[ord[0]];
    if (l0 > 0.0) {
      const double thr = l0 * kRankRtol * (double)p * kEps;
      while (k < rw && lam_s[ord[k]] > thr) ++k;
    }
    sh_int[1] = k;
  }
  __syncthreads();
  const int re = sh_int[1];
  for (int k = tid; k < R; k += kCThreads)
    ws[L.sig + k] = (k < re) ? sqrt(ldexp(lam_s[ord[k]], s_exp)) : 0.0;
  for (int idx = tid; idx < R * p; idx += kCThreads) {
    const int k = idx / p, i = idx - k * p;
    const C64d v = (k < re) ? Vc[(int64_t)i * p + ord[k]] : C64d{0.0, 0.0};
    Vo[idx] = v;
    const double inv = (k < re) ? 1.0 / sqrt(lam_s[ord[k]]) : 0.0;
    vsi[(int64_t)i * R + k] = {v.re * inv, v.im * inv};
  }
  __syncthreads();

  // ---- 3. A~ = vsi^H (G_XY vsi)
  for (int idx = tid; idx < p * re; idx += kCThreads) {
    const int i = idx / re, k = idx - i * re;
    C64d s = {0.0, 0.0};
    for (int j = 0; j < p; ++j) {
      const C64d t = zmul(Bc[(int64_t)i * p + j], vsi[(int64_t)j * R + k]);
      s.re += t.re;
      s.im += t.im;
    }
    Ac[(int64_t)i * R + k] = s;                  // Y = G_XY vsi, p x re (stride R)
  }
  __syncthreads();
  CF* Hc = reinterpret_cast<CF*>(ws + L.lu);
  CF* Qc = Hc + re * re;
  CF* Wc = Qc + re * re;
  CF* Uc = Wc + re * re;
  CF* yc = Uc + re * re;
  for (int idx = tid; idx < re * re; idx += kCThreads) {
    const int k = idx / re, l = idx - k * re;
    C64d s = {0.0, 0.0};
    for (int i = 0; i < p; ++i) {
      const C64d t = zcmul(vsi[(int64_t)i * R + k], Ac[(int64_t)i * R + l]);
      s.re += t.re;
      s.im += t.im;
    }
    At[idx] = s;
    Hc[idx] = {(float)s.re, (float)s.im};
  }
  __syncthreads();

  // ---- 4. eig(A~): FP32 complex Schur, then FP64 two-sided Rayleigh quotients
  if (warp == 0 && re > 0) {
    const bool ok = warp_eig32(Hc, Qc, Wc, Uc, yc, re, cs, sn);
    if (!ok && lane == 0) atomicOr(a.status, kDevRank);
  }
  __syncthreads();
  double* lam_tmp = ws + L.Y;
  for (int k = tid; k < re; k += kCThreads) {
    C64d num = {0.0, 0.0}, den = {0.0, 0.0};
    for (int i = 0; i < re; ++i) {
      C64d aw = {0.0, 0.0};
      for (int j = 0; j < re; ++j) {
        const CF wj = Wc[j * re + k];
        const C64d t = zmul(At[i * re + j], C64d{wj.re, wj.im});
        aw.re += t.re;
        aw.im += t.im;
      }
      const CF ui = Uc[i * re + k], wi = Wc[i * re + k];
      const C64d un = zcmul(C64d{ui.re, ui.im}, aw);
      const C64d ud = zcmul(C64d{ui.re, ui.im}, C64d{wi.re, wi.im});
      num.re += un.re;
      num.im += un.im;
      den.re += ud.re;
      den.im += ud.im;
    }
    const double q = den.re * den.re + den.im * den.im;
    lam_tmp[2 * k] = (q > 0.0) ? (num.re * den.re + num.im * den.im) / q : 0.0;
    lam_tmp[2 * k + 1] = (q > 0.0) ? (num.im * den.re - num.re * den.im) / q : 0.0;
  }
  __syncthreads();
  if (tid == 0) {
    for (int k = 0; k < re; ++k) ord[k] = k;
    for (int k = 0; k < re; ++k) {
      int best = k;
      for (int q = k + 1; q < re; ++q) {
        const double br = lam_tmp[2 * ord[best]], bi = lam_tmp[2 * ord[best] + 1];
        const double qr = lam_tmp[2 * ord[q]], qi = lam_tmp[2 * ord[q] + 1];
        const double mb = br * br + bi * bi, mq = qr * qr + qi * qi;
        if (mq > mb || (mq == mb && atan2(qi, qr) < atan2(bi, br))) best = q;
      }
      const int t = ord[k];
      ord[k] = ord[best];
      ord[best] = t;
    }
  }
  __syncthreads();
  for (int k = tid; k < R; k += kCThreads) {
    ws[L.lamout + 2 * k] = (k < re) ? lam_tmp[2 * ord[k]] : 0.0;
    ws[L.lamout + 2 * k + 1] = (k < re) ? lam_tmp[2 * ord[k] + 1] : 0.0;
  }
  __syncthreads();

  // ---- 5. M = vsi W, FP32 out in true units (vsi carries 2^{s/2})
  float* Mf = reinterpret_cast<float*>(ws + L.Mf);
  const double unscale = exp2(-0.5 * s_exp);
  for (int idx = tid; idx < p * R; idx += kCThreads) {
    const int row = idx / R, k = idx - row * R;
    C64d s = {0.0, 0.0};
    if (k < re) {
      const int kk = ord[k];
      for (int l = 0; l < re; ++l) {
        const CF wv = Wc[l * re + kk];
        const C64d t = zmul(vsi[(int64_t)row * R + l], C64d{wv.re, wv.im});
        s.re += t.re;
        s.im += t.im;
      }
    }
    Mf[2 * idx] = (float)(s.re * unscale);
    Mf[2 * idx + 1] = (float)(s.im * unscale);
  }

  // ---- 6. amplitudes b_k = u_k^H alpha_1 / (lambda_k u_k^H w_k), alpha_1[i] =
  //         sigma_i conj(V[0][i]); background index argmin |log lambda|
  for (int k = tid; k < R; k += kCThreads) {
    double br = 0.0, bi = 0.0;
    if (k < re) {
      const int kk = ord[k];
      C64d nu = {0.0, 0.0}, de = {0.0, 0.0};
      for (int i = 0; i < re; ++i) {
        const CF u = Uc[i * re + kk], wv = Wc[i * re + kk];
        const double sg = ws[L.sig + i];
        const C64d a1 = {sg * Vo[(int64_t)i * p].re, -sg * Vo[(int64_t)i * p].im};
        const C64d t1 = zcmul(C64d{u.re, u.im}, a1), t2 = zcmul(C64d{u.re, u.im}, C64d{wv.re, wv.im});
        nu.re += t1.re;
        nu.im += t1.im;
        de.re += t2.re;
        de.im += t2.im;
      }
      const double lr = ws[L.lamout + 2 * k], li = ws[L.lamout + 2 * k + 1];
      const C64d e = zmul(C64d{lr, li}, de);
      const double q = e.re * e.re + e.im * e.im;
      if (q > 0.0) {
        br = (nu.re * e.re + nu.im * e.im) / q;
        bi = (nu.im * e.re - nu.re * e.im) / q;
      } else {
        atomicOr(a.status, kDevRank);
      }
    }
    ws[L.bamp + 2 * k] = br;
    ws[L.bamp + 2 * k + 1] = bi;
  }
  __syncthreads();
  if (tid == 0) {
    int best = -1;
    double bv = 0.0;
    for (int k = 0; k < re; ++k) {
      const double lr = ws[L.lamout + 2 * k], li = ws[L.lamout + 2 * k + 1];
      const double lm = 0.5 * log(lr * lr + li * li), th = atan2(li, lr);
      const double v = lm * lm + th * th;
      if (best < 0 || v < bv) {
        best = k;
        bv = v;
      }
    }
    ws[L.bamp + 2 * (a.ws_m - 1 > 1 ? a.ws_m - 1 : 1)] = (double)best;
    *a.r_dev = re;
  }
}

}  // namespace

__host__ __device__ ModesLayout modes_layout(int m) {
  const int64_t p = m - 1 > 1 ? m - 1 : 1;
  const int64_t p2 = p * p;
  ModesLayout L;
  int64_t o = 0;
  auto take = [&](int64_t n) {
    const int64_t at = o;
    o += (n + 31) & ~int64_t(31);   // 256-byte aligned sub-arrays
    return at;
  };
  L.A = take(p2);           // df64 G_X when it does not fit in shared memory
  L.GXY = take(p2);         // df64 G_XY
  L.HV = 0;
  L.d = 0;
  L.e = 0;
  L.lam = 0;
  L.Z = take(p2);           // df64 vectors (rw x p)
  L.V = take(p2);           // FP64 V out
  L.Y = take(2 * p2);       // df64 G_XY vsi; Rayleigh-Ritz matrices when r > 32
  L.At = 0;
  L.Hc = 0;
  L.Qc = 0;
  L.Wc = 0;
  L.M = 0;
  L.Mf = take(p2);          // p x 2r floats
  L.sig = take(p);
  L.lamout = take(2 * p);
  L.tmp = 0;
  L.lu = take(6 * p2 + 64); // tridiagonal LU per vector (5 r p) + Ritz scratch (r p); A~ and eig fallback (6 r^2)
  L.clk = take(16);
  L.bamp = take(2 * p + 2);  // b (re, im) per mode, then [2p] = background index
  L.urec = take(p);          // 2p floats
  L.Mu = take((p2 + 1) / 2);  // p x r floats (r <= p)
  L.cx = take(12 * p2 + 64);  // complex windows: G_X, V, G_XY, A~, vsi, sorted V (complex128, p x p each)
  L.total = o;
  return L;
}

int64_t modes_ws_doubles(int m) { return modes_layout(m).total; }

bool modes_embed_ok(int c, int r) {
  const int pc = c - 1, K = (r < pc) ? r : pc, p = 2 * pc;
  const SmemPlan plan = smem_plan(p, 2 * K);
  if (!plan.a_in_smem || !plan.rr_in_smem) return false;
  if (plan.inv_in_smem) return true;
  // otherwise LU + Ritz scratch and Z go to the workspace laid out for pc
  const int64_t pp = (int64_t)pc * pc;
  return (int64_t)plan.rr_dim * 6 * p <= 6 * pp + 64 && (int64_t)plan.rr_dim * p <= pp;
}

cudaError_t launch_modes_small(const ModesArgs& a, cudaStream_t st) {
  const SmemPlan plan = smem_plan(a.embed_cx ? 2 * (a.c - 1) : a.c - 1, a.r_req);
  const size_t bytes = (size_t)(plan.vec_units + plan.rr_units + plan.big_units + plan.inv_units) * 8;
  const cudaError_t e = smem_optin(reinterpret_cast<const void*>(modes_small_kernel), bytes);
  if (e != cudaSuccess) return e;
  modes_small_kernel<<<1, kThreads, bytes, st>>>(a, modes_layout(a.ws_m));
  return cudaGetLastError();
}

cudaError_t launch_modes_batch(const ModesBatch& b, cudaStream_t st) {
  if (b.count < 1 || b.count > kMaxModesJobs) return cudaErrorInvalidValue;
  size_t bytes = 0;
  for (int i = 0; i < b.count; ++i) {
    const SmemPlan plan = smem_plan(b.job[i].c - 1, b.job[i].r_req);
    const size_t jb = (size_t)(plan.vec_units + plan.rr_units + plan.big_units + plan.inv_units) * 8;
    if (jb > bytes) bytes = jb;
  }
  const cudaError_t e = smem_optin(reinterpret_cast<const void*>(modes_batch_kernel), bytes);
  if (e != cudaSuccess) return e;
  modes_batch_kernel<<<b.count, kThreads, bytes, st>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_modes_complex(const ModesArgs& a, cudaStream_t st) {
  if (a.c - 1 > SDMD_MAX_M - 1) return cudaErrorNotSupported;
  modes_complex_kernel<<<1, kCThreads, 0, st>>>(a, modes_layout(a.ws_m));
  return cudaGetLastError();
}

}  // namespace sdmd
