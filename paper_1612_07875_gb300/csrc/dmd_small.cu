// Small dense FP64 algebra of the exact DMD step (Sec. 2.1 Eqs. 3-4, Sec. 2.2
// Eqs. 7-9; Algorithm 1's eig/sort and Algorithm 2's vsi, A~, eig, vsi*W).
// Everything here is O(m^3) on m <= 256 and runs in one CTA of 256 threads,
// in FP64. GB300 issues FP64 at about 2 FMA per clock per SM, so the kernel
// keeps G_X in shared memory (p <= 144), exploits symmetry in the rank-2
// updates, counts Sturm sign changes without divisions, runs the inverse
// iterations of all wanted vectors in parallel, and computes every scalar
// once (one thread) instead of redundantly in every lane.
//
// Steps (one kernel, phases separated by __syncthreads):
//  0. gather  G_X = G[0:p, 0:p], G_XY = G[0:p, 1:p+1] in time order from the
//     ring-indexed physical G (p = c-1).
//  1. Householder tridiagonalisation of G_X: Q^T G_X Q = T (d, e).
//  2. the r largest eigenvalues of T by Sturm-count bisection (one thread
//     per eigenvalue) to ~1e-11 relative.
//  3. their eigenvectors by inverse iteration on T (LU with partial
//     pivoting, one thread per vector), Gram-Schmidt over all wanted vectors
//     after every solve; Rayleigh quotients z^T T z give the final values.
//  4. back-transform z -> Q z (warp per vector) = columns of V.
//  5. numerical rank, sigma = sqrt(lambda), vsi = V Sigma^-1.
//  6. A~ = vsi^T (G_XY vsi).
//  7. eig of A~ (warp 0): complex Householder-Hessenberg, shifted complex QR
//     (Wilkinson shifts) to Schur form T = Q^H A~ Q, eigenvectors by
//     back-substitution on T, W = Q y normalised to unit 2-norm, eigenpairs
//     ordered by descending |lambda| then angle.
//  8. M = vsi W (complex), written in FP32 for the Phi kernel; lambda and
//     sigma written out.
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <stdint.h>

#include "sdmd_internal.cuh"

namespace sdmd {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr double kEps = 2.220446049250313e-16;   // 2^-52
constexpr double kRankRtol = 64.0;               // rank threshold factor (times p * eps)
constexpr int kInvIters = 3;                     // inverse-iteration solves per vector
constexpr int kBisectMax = 160;                  // bisection iteration cap
constexpr int kSmemMaxP = 144;                   // G_X kept in shared memory up to this p
constexpr int kSmemMaxR = 48;                    // eig(A~) workspace in shared memory up to this r

struct C2 {
  double re, im;
};
__device__ __forceinline__ C2 cadd(C2 a, C2 b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ C2 csub(C2 a, C2 b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ C2 cmul(C2 a, C2 b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__device__ __forceinline__ C2 cconj(C2 a) { return {a.re, -a.im}; }
__device__ __forceinline__ C2 cscale(C2 a, double s) { return {a.re * s, a.im * s}; }
__device__ __forceinline__ double cabs2(C2 a) { return a.re * a.re + a.im * a.im; }
__device__ __forceinline__ double cabs(C2 a) { return hypot(a.re, a.im); }
__device__ __forceinline__ C2 cdiv(C2 a, C2 b) {
  // Smith's algorithm
  if (fabs(b.re) >= fabs(b.im)) {
    const double r = b.im / b.re, den = b.re + b.im * r;
    return {(a.re + a.im * r) / den, (a.im - a.re * r) / den};
  }
  const double r = b.re / b.im, den = b.re * r + b.im;
  return {(a.re * r + a.im) / den, (a.im * r - a.re) / den};
}
__device__ __forceinline__ C2 csqrt(C2 z) {
  const double m = cabs(z);
  if (m == 0.0) return {0.0, 0.0};
  double re = sqrt(0.5 * (m + fabs(z.re)));
  double im = z.im / (2.0 * re);
  if (z.re >= 0.0) return {re, im};
  return {fabs(im), copysign(re, z.im)};
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct WS {
  double *A, *GXY, *d, *e, *lam, *Z, *V, *Y, *At, *Hc, *Qc, *Wc, *M, *sig, *lamout, *tmp, *lu, *clk;
  float* Mf;
};

__device__ WS carve(double* base, const ModesLayout& L) {
  WS w;
  w.A = base + L.A;
  w.GXY = base + L.GXY;
  w.d = base + L.d;
  w.e = base + L.e;
  w.lam = base + L.lam;
  w.Z = base + L.Z;
  w.V = base + L.V;
  w.Y = base + L.Y;
  w.At = base + L.At;
  w.Hc = base + L.Hc;
  w.Qc = base + L.Qc;
  w.Wc = base + L.Wc;
  w.M = base + L.M;
  w.sig = base + L.sig;
  w.lamout = base + L.lamout;
  w.tmp = base + L.tmp;
  w.lu = base + L.lu;
  w.clk = base + L.clk;
  w.Mf = reinterpret_cast<float*>(base + L.Mf);
  return w;
}

// ---------------------------------------------------------------- phase 3 --
// LU factorisation with partial pivoting of the tridiagonal T - lambda I.
// Row i of U has (u0, u1, u2) on columns (i, i+1, i+2); mult/piv describe L.
__device__ void tri_lu(const double* d, const double* e, int p, double lambda, double tiny,
                       double* u0, double* u1, double* u2, double* mult, double* piv) {
  double cd = d[0] - lambda, c1 = (p > 1) ? e[0] : 0.0, c2 = 0.0;
  for (int i = 0; i + 1 < p; ++i) {
    const double sub = e[i];
    const double nd = d[i + 1] - lambda;
    const double n1 = (i + 2 < p) ? e[i + 1] : 0.0;
    if (fabs(cd) >= fabs(sub)) {
      const double mu = (cd != 0.0) ? sub / cd : 0.0;
      u0[i] = cd;
      u1[i] = c1;
      u2[i] = c2;
      piv[i] = 0.0;
      mult[i] = mu;
      cd = nd - mu * c1;
      c1 = n1 - mu * c2;
      c2 = 0.0;
    } else {
      const double mu = cd / sub;
      u0[i] = sub;
      u1[i] = nd;
      u2[i] = n1;
      piv[i] = 1.0;
      mult[i] = mu;
      cd = c1 - mu * nd;
      c1 = c2 - mu * n1;
      c2 = 0.0;
    }
    if (fabs(u0[i]) < tiny) u0[i] = copysign(tiny, u0[i]);
  }
  u0[p - 1] = (fabs(cd) < tiny) ? copysign(tiny, cd) : cd;
  u1[p - 1] = 0.0;
  u2[p - 1] = 0.0;
}

__device__ void tri_solve(int p, const double* u0, const double* u1, const double* u2,
                          const double* mult, const double* piv, double* b) {
  for (int i = 0; i + 1 < p; ++i) {
    if (piv[i] != 0.0) {
      const double bi = b[i], bn = b[i + 1];
      b[i] = bn;
      b[i + 1] = bi - mult[i] * bn;
    } else {
      b[i + 1] -= mult[i] * b[i];
    }
  }
  for (int i = p - 1; i >= 0; --i) {
    double s = b[i];
    if (i + 1 < p) s -= u1[i] * b[i + 1];
    if (i + 2 < p) s -= u2[i] * b[i + 2];
    b[i] = s / u0[i];
  }
}

// ---------------------------------------------------------------- phase 7 --
// Eigen-decomposition of the complex r x r matrix H (row-major, C2) by one
// warp: Hessenberg reduction, shifted QR to Schur form with Q accumulated,
// eigenvectors W (columns, unit norm). Returns false if the QR iteration cap
// was reached.
__device__ bool warp_eig(C2* H, C2* Q, C2* W, C2* ycol, int r, double* cs, C2* sn) {
  const int lane = threadIdx.x & 31;
  for (int idx = lane; idx < r * r; idx += 32) {
    const int i = idx / r, j = idx - i * r;
    Q[idx] = {i == j ? 1.0 : 0.0, 0.0};
  }
  __syncwarp();
  // Householder to upper Hessenberg: for column j, reflect H[j+1..r-1][j].
  for (int j = 0; j + 2 < r; ++j) {
    const int L = r - j - 1;
    double tail = 0.0;
    for (int i = 1 + lane; i < L; i += 32) tail += cabs2(H[(j + 1 + i) * r + j]);
    tail = warp_sum(tail);
    const C2 x0 = H[(j + 1) * r + j];
    __syncwarp();
    if (tail == 0.0) continue;
    // reflector scalars on lane 0 only, then broadcast
    C2 v0 = {0.0, 0.0};
    double ivn = 0.0;
    if (lane == 0) {
      const double ax0 = cabs(x0);
      const double nrm = sqrt(ax0 * ax0 + tail);
      const C2 ph = (ax0 > 0.0) ? cscale(x0, 1.0 / ax0) : C2{1.0, 0.0};
      const C2 alpha = cscale(ph, -nrm);                 // -e^{i arg x0} |x|
      v0 = csub(x0, alpha);
      ivn = 1.0 / sqrt(cabs2(v0) + tail);
    }
    v0.re = __shfl_sync(0xffffffffu, v0.re, 0);
    v0.im = __shfl_sync(0xffffffffu, v0.im, 0);
    const double vn_inv = __shfl_sync(0xffffffffu, ivn, 0);
    // v stored in ycol[0..L-1]
    for (int i = lane; i < L; i += 32) ycol[i] = cscale(i == 0 ? v0 : H[(j + 1 + i) * r + j], vn_inv);
    __syncwarp();
    // H <- (I - 2 v v^H) H on rows j+1..r-1 (columns j..r-1)
    for (int q = j + lane; q < r; q += 32) {
      C2 s = {0.0, 0.0};
      for (int i = 0; i < L; ++i) s = cadd(s, cmul(cconj(ycol[i]), H[(j + 1 + i) * r + q]));
      for (int i = 0; i < L; ++i) H[(j + 1 + i) * r + q] = csub(H[(j + 1 + i) * r + q], cscale(cmul(ycol[i], s), 2.0));
    }
    __syncwarp();
    // H <- H (I - 2 v v^H) on columns j+1..r-1 (all rows); Q likewise
    for (int q = lane; q < 2 * r; q += 32) {
      C2* M = (q < r) ? H : Q;
      const int row = (q < r) ? q : q - r;
      C2 s = {0.0, 0.0};
      for (int i = 0; i < L; ++i) s = cadd(s, cmul(M[row * r + j + 1 + i], ycol[i]));
      for (int i = 0; i < L; ++i)
        M[row * r + j + 1 + i] = csub(M[row * r + j + 1 + i], cscale(cmul(s, cconj(ycol[i])), 2.0));
    }
    __syncwarp();
    for (int i = 2 + lane; i <= L; i += 32) H[(j + i) * r + j] = {0.0, 0.0};
    __syncwarp();
  }
  // Shifted QR on the Hessenberg matrix.
  double hnorm = 0.0;
  for (int idx = lane; idx < r * r; idx += 32) hnorm = fmax(hnorm, cabs(H[idx]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) hnorm = fmax(hnorm, __shfl_xor_sync(0xffffffffu, hnorm, o));
  if (hnorm == 0.0) hnorm = 1.0;
  bool ok = true;
  int hi = r - 1, its = 0, total = 0;
  const int cap = 60 * r + 60;
  while (hi > 0) {
    // deflation scan (lane 0), result broadcast
    int l = hi;
    if (lane == 0) {
      while (l > 0) {
        const double sub = cabs(H[l * r + l - 1]);
        double scale = cabs(H[l * r + l]) + cabs(H[(l - 1) * r + l - 1]);
        if (scale == 0.0) scale = hnorm;
        if (sub <= kEps * scale) break;
        --l;
      }
      if (l > 0) H[l * r + l - 1] = {0.0, 0.0};
    }
    l = __shfl_sync(0xffffffffu, l, 0);
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
    // Wilkinson shift from the trailing 2 x 2 of the active block (lane 0)
    C2 mu = {0.0, 0.0};
    if (lane == 0) {
      const C2 a = H[(hi - 1) * r + hi - 1], b = H[(hi - 1) * r + hi], c = H[hi * r + hi - 1],
               dd = H[hi * r + hi];
      if (its % 11 == 10) {
        mu = cadd(dd, C2{0.75 * cabs(c), 0.0});       // exceptional shift
      } else {
        const C2 half = cscale(csub(a, dd), 0.5);
        const C2 disc = csqrt(cadd(cmul(half, half), cmul(b, c)));
        const C2 tr = cscale(cadd(a, dd), 0.5);
        const C2 m1 = cadd(tr, disc), m2 = csub(tr, disc);
        mu = (cabs(csub(m1, dd)) <= cabs(csub(m2, dd))) ? m1 : m2;
      }
    }
    mu.re = __shfl_sync(0xffffffffu, mu.re, 0);
    mu.im = __shfl_sync(0xffffffffu, mu.im, 0);
    for (int q = l + lane; q <= hi; q += 32) H[q * r + q] = csub(H[q * r + q], mu);
    __syncwarp();
    // H - mu I = Q R by Givens rotations on rows j, j+1
    for (int j = l; j < hi; ++j) {
      double c = 1.0;
      C2 s = {0.0, 0.0};
      if (lane == 0) {
        const C2 a = H[j * r + j], b = H[(j + 1) * r + j];
        const double aa = cabs(a), rho = hypot(aa, cabs(b));
        if (rho == 0.0) {
          c = 1.0;
        } else if (aa == 0.0) {
          c = 0.0;
          s = {1.0, 0.0};
        } else {
          c = aa / rho;
          s = cscale(cmul(cscale(a, 1.0 / aa), cconj(b)), 1.0 / rho);
        }
      }
      c = __shfl_sync(0xffffffffu, c, 0);
      s.re = __shfl_sync(0xffffffffu, s.re, 0);
      s.im = __shfl_sync(0xffffffffu, s.im, 0);
      __syncwarp();
      for (int q = j + lane; q < r; q += 32) {
        const C2 h1 = H[j * r + q], h2 = H[(j + 1) * r + q];
        H[j * r + q] = cadd(cscale(h1, c), cmul(s, h2));
        H[(j + 1) * r + q] = csub(cscale(h2, c), cmul(cconj(s), h1));
      }
      if (lane == 0) {
        cs[j] = c;
        sn[j] = s;
      }
      __syncwarp();
    }
    // R Q + mu I: apply G_j^H on columns j, j+1 (rows 0..j+1); Q <- Q G_j^H
    for (int j = l; j < hi; ++j) {
      const double c = cs[j];
      const C2 s = sn[j];
      for (int q = lane; q < r + (j + 2); q += 32) {
        C2* M = (q < j + 2) ? H : Q;
        const int row = (q < j + 2) ? q : q - (j + 2);
        if (q >= j + 2 && row >= r) continue;
        const C2 h1 = M[row * r + j], h2 = M[row * r + j + 1];
        M[row * r + j] = cadd(cscale(h1, c), cmul(h2, cconj(s)));
        M[row * r + j + 1] = csub(cscale(h2, c), cmul(h1, s));
      }
      __syncwarp();
    }
    for (int q = l + lane; q <= hi; q += 32) H[q * r + q] = cadd(H[q * r + q], mu);
    __syncwarp();
  }
  __syncwarp();
  // Eigenvectors of the upper-triangular Schur factor, one per lane.
  double tnorm = 0.0;
  for (int idx = lane; idx < r * r; idx += 32) {
    const int i = idx / r, j = idx - i * r;
    if (j >= i) tnorm = fmax(tnorm, cabs(H[idx]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tnorm = fmax(tnorm, __shfl_xor_sync(0xffffffffu, tnorm, o));
  const double small = fmax(kEps * tnorm, DBL_MIN);
  for (int k = lane; k < r; k += 32) {
    C2* y = ycol + k * r;
    const C2 lk = H[k * r + k];
    for (int i = k + 1; i < r; ++i) y[i] = {0.0, 0.0};
    y[k] = {1.0, 0.0};
    for (int i = k - 1; i >= 0; --i) {
      C2 s = {0.0, 0.0};
      for (int j = i + 1; j <= k; ++j) s = cadd(s, cmul(H[i * r + j], y[j]));
      C2 den = csub(H[i * r + i], lk);
      if (cabs(den) < small) den = {small, 0.0};
      y[i] = cdiv(cscale(s, -1.0), den);
    }
    double nn = 0.0;
    for (int q = 0; q < r; ++q) {
      C2 w = {0.0, 0.0};
      for (int i = 0; i <= k; ++i) w = cadd(w, cmul(Q[q * r + i], y[i]));
      W[q * r + k] = w;
      nn += cabs2(w);
    }
    const double inv = 1.0 / sqrt(nn);
    for (int q = 0; q < r; ++q) W[q * r + k] = cscale(W[q * r + k], inv);
  }
  __syncwarp();
  return ok;
}

// ---------------------------------------------------------------- phase 1 --
// Householder reduction of the symmetric p x p matrix A (row-major, full
// storage) to tridiagonal form T = Q^T A Q (d, e). Reflector k is
// H_k = I - 2 v v^T on indices k+1..p-1 with v unit (zero when column k is
// already reduced); v is stored over row k, A[k][k+1..p-1], which holds no
// data any more once step k has run. Scalars are formed by one thread and
// shared through `sc`: on GB300 every FP64 lane-op counts, so no FP64 value
// is computed redundantly by all threads.
__device__ void tridiagonalize(double* A, int p, double* d, double* e, double* vs, double* pv,
                               double* wv, double* sc) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int k = 0; k + 2 < p; ++k) {
    const int L = p - k - 1;
    double* rowk = A + (int64_t)k * p + (k + 1);
    if (warp == 0) {
      double t = 0.0;
      for (int i = 1 + lane; i < L; i += 32) t = fma(rowk[i], rowk[i], t);
      t = warp_sum(t);
      if (lane == 0) {
        const double x0 = rowk[0];
        d[k] = A[(int64_t)k * p + k];
        if (t == 0.0) {
          sc[0] = 0.0;
          e[k] = x0;
        } else {
          const double nrm = sqrt(fma(x0, x0, t));
          const double alpha = (x0 >= 0.0) ? -nrm : nrm;
          const double v0 = x0 - alpha;                 // same sign as x0: no cancellation
          sc[0] = 1.0 / sqrt(fma(v0, v0, t));
          sc[1] = v0;
          e[k] = alpha;
        }
      }
    }
    __syncthreads();
    const double inv = sc[0];
    if (inv == 0.0) {
      for (int i = tid; i < L; i += kThreads) rowk[i] = 0.0;
      __syncthreads();
      continue;
    }
    const double v0 = sc[1];
    for (int i = tid; i < L; i += kThreads) vs[i] = (i == 0 ? v0 : rowk[i]) * inv;
    __syncthreads();
    // pv = A_sub v (column i of the symmetric A_sub read as row i); v -> row k
    double* As = A + (int64_t)(k + 1) * p + (k + 1);
    for (int i = tid; i < L; i += kThreads) {
      rowk[i] = vs[i];
      double s0 = 0.0, s1 = 0.0;
      int j = 0;
      for (; j + 1 < L; j += 2) {
        s0 = fma(As[(int64_t)j * p + i], vs[j], s0);
        s1 = fma(As[(int64_t)(j + 1) * p + i], vs[j + 1], s1);
      }
      if (j < L) s0 = fma(As[(int64_t)j * p + i], vs[j], s0);
      pv[i] = s0 + s1;
    }
    __syncthreads();
    if (warp == 0) {
      double t = 0.0;
      for (int i = lane; i < L; i += 32) t = fma(vs[i], pv[i], t);
      t = warp_sum(t);
      if (lane == 0) sc[2] = t;
    }
    __syncthreads();
    const double kv = sc[2];
    for (int i = tid; i < L; i += kThreads) wv[i] = 2.0 * fma(-kv, vs[i], pv[i]);
    __syncthreads();
    // A_sub -= v w^T + w v^T: lower triangle computed, mirrored to the upper;
    // thread t takes columns t and L-1-t (L+1 entries in all)
    const int half = (L + 1) / 2;
    for (int t = tid; t < half; t += kThreads) {
      for (int pass = 0; pass < 2; ++pass) {
        const int j = (pass == 0) ? t : L - 1 - t;
        if (pass == 1 && j == t) break;
        const double vj = vs[j], wj = wv[j];
        for (int i = j; i < L; ++i) {
          const double val = fma(-wv[i], vj, fma(-vs[i], wj, As[(int64_t)i * p + j]));
          As[(int64_t)i * p + j] = val;
          As[(int64_t)j * p + i] = val;
        }
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (p >= 2) {
      d[p - 2] = A[(int64_t)(p - 2) * p + (p - 2)];
      d[p - 1] = A[(int64_t)(p - 1) * p + (p - 1)];
      e[p - 2] = A[(int64_t)(p - 2) * p + (p - 1)];
    } else {
      d[0] = A[0];
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- phase 2 --
__device__ __forceinline__ int dexp_bits(double v) { return (__double2hiint(v) >> 20) & 0x7ff; }

// Sign of v (+1 / -1), or 0 for +-0, from the bit pattern (no FP64 compare).
__device__ __forceinline__ int dsign(double v) {
  const long long b = __double_as_longlong(v);
  if ((b << 1) == 0) return 0;
  return (b < 0) ? -1 : 1;
}

// Number of eigenvalues of the symmetric tridiagonal (d, e^2) below x: sign
// changes of the Sturm sequence p_0 = 1, p_i = (d_{i-1} - x) p_{i-1}
// - e_{i-2}^2 p_{i-2}. No divisions; the two live terms are rescaled by exact
// powers of two near the ends of the FP64 range; a zero term takes the sign
// opposite to its predecessor.
__device__ int sturm_count(const double* d, const double* e2, int p, double x) {
  double pm = 1.0, pc = d[0] - x;
  int s = dsign(pc);
  if (s == 0) s = -1;
  int cnt = (s < 0);
  for (int i = 1; i < p; ++i) {
    const double pn = fma(d[i] - x, pc, -e2[i - 1] * pm);
    pm = pc;
    pc = pn;
    const int ex = max(dexp_bits(pc), dexp_bits(pm));
    if (ex > 1023 + 600) {
      pc *= 0x1p-600;
      pm *= 0x1p-600;
    } else if (ex < 1023 - 600) {
      pc *= 0x1p+600;
      pm *= 0x1p+600;
    }
    int sn = dsign(pc);
    if (sn == 0) sn = -s;
    cnt += (sn != s);
    s = sn;
  }
  return cnt;
}

// ---------------------------------------------------------------- phase 3 --
// Orthonormalise the rw vectors Z[i*p ..] in order (classical Gram-Schmidt,
// applied twice), vectors spread over warps, rows over threads.
__device__ void orthonormalize(double* Z, int rw, int p, double* coef, double* red, double* sc) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = 0; i < rw; ++i) {
    double* zi = Z + (int64_t)i * p;
    for (int pass = 0; pass < 2 && i > 0; ++pass) {
      for (int j = warp; j < i; j += kWarps) {
        const double* zj = Z + (int64_t)j * p;
        double s = 0.0;
        for (int q = lane; q < p; q += 32) s = fma(zj[q], zi[q], s);
        s = warp_sum(s);
        if (lane == 0) coef[j] = s;
      }
      __syncthreads();
      for (int q = tid; q < p; q += kThreads) {
        double s = zi[q];
        for (int j = 0; j < i; ++j) s = fma(-coef[j], Z[(int64_t)j * p + q], s);
        zi[q] = s;
      }
      __syncthreads();
    }
    double nn = 0.0;
    for (int q = tid; q < p; q += kThreads) nn = fma(zi[q], zi[q], nn);
    nn = warp_sum(nn);
    if (lane == 0) red[warp] = nn;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < kWarps; ++w) t += red[w];
      sc[3] = (t > 0.0) ? 1.0 / sqrt(t) : 0.0;
    }
    __syncthreads();
    const double inv = sc[3];
    for (int q = tid; q < p; q += kThreads) zi[q] *= inv;
    __syncthreads();
  }
}

// Shared-memory plan (dynamic): vectors first, then one big region that
// holds G_X (phases 0-4) and later the complex r x r eigen-workspace.
struct SmemPlan {
  int a_in_smem, eig_in_smem;
  int64_t vec_doubles, big_doubles;
};

__host__ __device__ inline SmemPlan smem_plan(int p, int r) {
  SmemPlan s;
  const int64_t P = (p + 3) & ~3;
  s.vec_doubles = 8 * P + 64;
  s.a_in_smem = (p <= kSmemMaxP);
  s.eig_in_smem = (r <= kSmemMaxR);
  const int64_t a = s.a_in_smem ? (int64_t)p * p : 0;
  const int64_t g = s.eig_in_smem ? (int64_t)8 * r * r : 0;   // H, Q, W, y: 4 x r^2 complex
  s.big_doubles = a > g ? a : g;
  return s;
}

__global__ void __launch_bounds__(kThreads, 1) modes_small_kernel(ModesArgs a, ModesLayout L) {
  extern __shared__ double smem[];
  __shared__ double red[kWarps + 1];
  __shared__ double sc[8];
  __shared__ int sh_reff;
  __shared__ double cs[SDMD_MAX_M];
  __shared__ C2 sn[SDMD_MAX_M];
  __shared__ int order[SDMD_MAX_M];
  __shared__ double coef[SDMD_MAX_M];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  WS w = carve(a.ws, L);
  long long* clk = reinterpret_cast<long long*>(w.clk);
  const int m = a.m, p = a.c - 1;
  const int rw = min(a.r_req, p);
  const SmemPlan plan = smem_plan(p, a.r_req);
  const int64_t P = (p + 3) & ~3;
  double* d = smem;
  double* e = d + P;
  double* e2 = e + P;
  double* vs = e2 + P;
  double* pv = vs + P;
  double* wv = pv + P;
  double* lam = wv + P;
  double* big = smem + plan.vec_doubles;
  double* A = plan.a_in_smem ? big : w.A;
  if (tid == 0) clk[0] = clock64();

  // ---- 0. gather time-ordered blocks
  for (int idx = tid; idx < p * p; idx += kThreads) {
    const int i = idx / p, j = idx - i * p;
    const int si = (a.start + i) % m, sj = (a.start + j) % m, sj1 = (a.start + j + 1) % m;
    double gx, gxy;
    if (a.g_is_int) {
      const long long* G = static_cast<const long long*>(a.G);
      gx = (double)G[(int64_t)si * m + sj];
      gxy = (double)G[(int64_t)si * m + sj1];
    } else {
      const double* G = static_cast<const double*>(a.G);
      gx = G[(int64_t)si * m + sj];
      gxy = G[(int64_t)si * m + sj1];
    }
    A[idx] = gx;
    w.GXY[idx] = gxy;
  }
  __syncthreads();
  if (tid == 0) clk[1] = clock64();

  // ---- 1. tridiagonalise G_X
  tridiagonalize(A, p, d, e, vs, pv, wv, sc);
  if (tid == 0) clk[2] = clock64();

  // ---- 2. bisection for the rw largest eigenvalues
  for (int i = tid; i < p; i += kThreads) e2[i] = (i + 1 < p) ? e[i] * e[i] : 0.0;
  if (tid == 0) {
    double gl = 0.0, gu = 0.0;
    for (int i = 0; i < p; ++i) {
      const double rad = ((i > 0) ? fabs(e[i - 1]) : 0.0) + ((i + 1 < p) ? fabs(e[i]) : 0.0);
      gl = (i == 0) ? d[0] - rad : fmin(gl, d[i] - rad);
      gu = (i == 0) ? d[0] + rad : fmax(gu, d[i] + rad);
    }
    const double tn = fmax(fabs(gl), fabs(gu));
    sc[4] = gl - 4.0 * kEps * tn * p - DBL_MIN;
    sc[5] = gu + 4.0 * kEps * tn * p + DBL_MIN;
    sc[6] = tn;
  }
  __syncthreads();
  const double gl = sc[4], gu = sc[5], tnorm = sc[6];
  // thread owner(i) bisects for eigenvalue i; owners are spread one per warp
  // first so that the sub-partitions' FP64 units work in parallel
  for (int i = 0; i < rw; ++i) {
    const int owner = (i % kWarps) * 32 + (i / kWarps) % 32;
    if (tid != owner) continue;
    const int target = p - 1 - i;
    double lo = gl, hi = gu;
    const double atol = kEps * tnorm;
    for (int it = 0; it < kBisectMax; ++it) {
      if (hi - lo <= fmax(1e-11 * fmax(fabs(lo), fabs(hi)), atol)) break;
      const double mid = 0.5 * (lo + hi);
      if (sturm_count(d, e2, p, mid) > target)
        hi = mid;
      else
        lo = mid;
    }
    lam[i] = 0.5 * (lo + hi);
  }
  __syncthreads();
  if (tid == 0) clk[3] = clock64();

  // ---- 3. inverse iteration (thread per vector), Gram-Schmidt between solves
  const double tiny = fmax(kEps * tnorm, DBL_MIN);
  for (int i = 0; i < rw; ++i) {
    const int owner = (i % kWarps) * 32 + (i / kWarps) % 32;
    if (tid != owner) continue;
    double* u0 = w.lu + (int64_t)i * 5 * p;
    double *u1 = u0 + p, *u2 = u1 + p, *mu = u2 + p, *pvt = mu + p;
    double shift = lam[i];
    for (int q = 0; q < i; ++q)      // numerically equal eigenvalues: distinct shifts
      if (fabs(lam[q] - shift) < 4.0 * kEps * tnorm) shift -= 4.0 * kEps * tnorm;
    tri_lu(d, e, p, shift, tiny, u0, u1, u2, mu, pvt);
    double* z = w.Z + (int64_t)i * p;
    for (int j = 0; j < p; ++j) z[j] = 1.0 + 0.1 * (double)(((j + 1) * 7919 + (i + 1) * 104729) % 97) / 97.0;
  }
  __syncthreads();
  for (int it = 0; it < kInvIters; ++it) {
    for (int i = 0; i < rw; ++i) {
      const int owner = (i % kWarps) * 32 + (i / kWarps) % 32;
      if (tid != owner) continue;
      double* u0 = w.lu + (int64_t)i * 5 * p;
      tri_solve(p, u0, u0 + p, u0 + 2 * p, u0 + 3 * p, u0 + 4 * p, w.Z + (int64_t)i * p);
    }
    __syncthreads();
    orthonormalize(w.Z, rw, p, coef, red, sc);
  }
  // Rayleigh quotients z^T T z refine the eigenvalues (warp per vector)
  for (int i = warp; i < rw; i += kWarps) {
    const double* z = w.Z + (int64_t)i * p;
    double s = 0.0;
    for (int q = lane; q < p; q += 32) {
      double tz = d[q] * z[q];
      if (q > 0) tz = fma(e[q - 1], z[q - 1], tz);
      if (q + 1 < p) tz = fma(e[q], z[q + 1], tz);
      s = fma(z[q], tz, s);
    }
    s = warp_sum(s);
    if (lane == 0) lam[i] = s;
  }
  __syncthreads();
  if (tid == 0) clk[4] = clock64();

  // ---- 4. back-transform: v = H_0 H_1 ... H_{p-3} z  (warp per vector)
  for (int i = warp; i < rw; i += kWarps) {
    double* z = w.Z + (int64_t)i * p;
    for (int k = p - 3; k >= 0; --k) {
      const int Lk = p - k - 1;
      const double* v = A + (int64_t)k * p + (k + 1);
      double s = 0.0;
      for (int j = lane; j < Lk; j += 32) s = fma(v[j], z[k + 1 + j], s);
      s = warp_sum(s);
      for (int j = lane; j < Lk; j += 32) z[k + 1 + j] = fma(-2.0 * s, v[j], z[k + 1 + j]);
      __syncwarp();
    }
  }
  __syncthreads();
  if (tid == 0) clk[5] = clock64();

  // ---- 5. rank, sigma, V, vsi = V Sigma^-1 (in place in Z)
  if (tid == 0) {
    int k = 0;
    const double lam0 = (rw > 0) ? lam[0] : 0.0;
    if (lam0 > 0.0) {
      const double thr = lam0 * kRankRtol * (double)p * kEps;
      while (k < rw && lam[k] > thr) ++k;
    }
    sh_reff = k;
    for (int i = 0; i < a.r_req; ++i) {
      w.sig[i] = (i < k) ? sqrt(lam[i]) : 0.0;
      cs[i] = (i < k) ? 1.0 / w.sig[i] : 0.0;
    }
  }
  __syncthreads();
  const int re = sh_reff;
  for (int idx = tid; idx < a.r_req * p; idx += kThreads) {
    const int i = idx / p;
    const double z = (i < re) ? w.Z[idx] : 0.0;
    w.V[idx] = z;
    if (i < re) w.Z[idx] = z * cs[i];
  }
  __syncthreads();

  // ---- 6. A~ = vsi^T G_XY vsi  (Y = G_XY vsi first)
  for (int idx = tid; idx < re * p; idx += kThreads) {
    const int k = idx / p, row = idx - k * p;
    const double* g = w.GXY + (int64_t)row * p;
    const double* v = w.Z + (int64_t)k * p;
    double s0 = 0.0, s1 = 0.0;
    int b = 0;
    for (; b + 1 < p; b += 2) {
      s0 = fma(g[b], v[b], s0);
      s1 = fma(g[b + 1], v[b + 1], s1);
    }
    if (b < p) s0 = fma(g[b], v[b], s0);
    w.Y[idx] = s0 + s1;
  }
  __syncthreads();
  C2* Hc = plan.eig_in_smem ? reinterpret_cast<C2*>(big) : reinterpret_cast<C2*>(w.Hc);
  C2* Qc = plan.eig_in_smem ? Hc + re * re : reinterpret_cast<C2*>(w.Qc);
  C2* Wc = plan.eig_in_smem ? Qc + re * re : reinterpret_cast<C2*>(w.Wc);
  C2* ycol = plan.eig_in_smem ? Wc + re * re : reinterpret_cast<C2*>(w.lu);
  for (int idx = tid; idx < re * re; idx += kThreads) {
    const int k = idx / re, l = idx - k * re;
    const double* v = w.Z + (int64_t)k * p;
    const double* y = w.Y + (int64_t)l * p;
    double s = 0.0;
    for (int b = 0; b < p; ++b) s = fma(v[b], y[b], s);
    w.At[idx] = s;
    Hc[idx] = {s, 0.0};
  }
  __syncthreads();
  if (tid == 0) clk[6] = clock64();

  // ---- 7. eig(A~) on warp 0
  if (warp == 0 && re > 0) {
    const bool ok = warp_eig(Hc, Qc, Wc, ycol, re, cs, sn);
    if (!ok && lane == 0) atomicOr(a.status, kDevRank);
    if (lane == 0) {
      for (int k = 0; k < re; ++k) order[k] = k;
      for (int k = 0; k < re; ++k) {
        int best = k;
        for (int q = k + 1; q < re; ++q) {
          const C2 lb = Hc[order[best] * re + order[best]], lq = Hc[order[q] * re + order[q]];
          const double mb = cabs(lb), mq = cabs(lq);
          if (mq > mb || (mq == mb && atan2(lq.im, lq.re) < atan2(lb.im, lb.re))) best = q;
        }
        const int t = order[k];
        order[k] = order[best];
        order[best] = t;
      }
    }
  }
  __syncthreads();
  if (tid == 0) clk[7] = clock64();

  // ---- 8. outputs: lambda, M = vsi W (FP64 and FP32 copies)
  C2* lamout = reinterpret_cast<C2*>(w.lamout);
  for (int k = tid; k < a.r_req; k += kThreads)
    lamout[k] = (k < re) ? Hc[order[k] * re + order[k]] : C2{0.0, 0.0};
  C2* Mc = reinterpret_cast<C2*>(w.M);
  const int R = a.r_req;
  for (int idx = tid; idx < p * R; idx += kThreads) {
    const int row = idx / R, k = idx - row * R;
    C2 s = {0.0, 0.0};
    if (k < re) {
      const int kk = order[k];
      for (int l = 0; l < re; ++l) {
        const double z = w.Z[(int64_t)l * p + row];
        const C2 wv2 = Wc[l * re + kk];
        s.re = fma(wv2.re, z, s.re);
        s.im = fma(wv2.im, z, s.im);
      }
    }
    Mc[idx] = s;
    w.Mf[2 * idx] = (float)s.re;
    w.Mf[2 * idx + 1] = (float)s.im;
  }
  __syncthreads();
  if (tid == 0) {
    *a.r_dev = re;
    clk[8] = clock64();
  }
}

}  // namespace

ModesLayout modes_layout(int m) {
  const int64_t p = m - 1 > 1 ? m - 1 : 1;
  const int64_t p2 = p * p;
  ModesLayout L;
  int64_t o = 0;
  auto take = [&](int64_t n) {
    const int64_t at = o;
    o += (n + 31) & ~int64_t(31);   // 256-byte aligned sub-arrays
    return at;
  };
  L.A = take(p2);
  L.GXY = take(p2);
  L.HV = 0;
  L.d = take(p);
  L.e = take(p);
  L.lam = take(p);
  L.Z = take(p2);
  L.V = take(p2);
  L.Y = take(p2);
  L.At = take(p2);
  L.Hc = take(2 * p2);
  L.Qc = take(2 * p2);
  L.Wc = take(2 * p2);
  L.M = take(2 * p2);
  L.Mf = take(p2);          // p x 2r floats
  L.sig = take(p);
  L.lamout = take(2 * p);
  L.tmp = take(4 * p);
  L.lu = take(5 * p2 + 2 * p2);
  L.clk = take(16);
  L.total = o;
  return L;
}

int64_t modes_ws_doubles(int m) { return modes_layout(m).total; }

cudaError_t launch_modes_small(const ModesArgs& a, cudaStream_t st) {
  static size_t attr_bytes = 0;   // dynamic shared memory opted in so far
  const SmemPlan plan = smem_plan(a.c - 1, a.r_req);
  const size_t bytes = (size_t)(plan.vec_doubles + plan.big_doubles) * sizeof(double);
  if (bytes > attr_bytes) {
    cudaError_t e = cudaFuncSetAttribute(modes_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
    if (e != cudaSuccess) return e;
    attr_bytes = bytes;
  }
  modes_small_kernel<<<1, kThreads, bytes, st>>>(a, modes_layout(a.m));
  return cudaGetLastError();
}

}  // namespace sdmd
