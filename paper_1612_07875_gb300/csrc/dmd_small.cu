// Small dense FP64 algebra of the exact DMD step (Sec. 2.1 Eqs. 3-4, Sec. 2.2
// Eqs. 7-9; Algorithm 1's eig/sort and Algorithm 2's vsi, A~, eig, vsi*W).
// Everything here is O(m^3) on m <= 256 and runs in one CTA of 256 threads,
// in FP64, on data that stays in L1/L2.
//
// Steps (one kernel, phases separated by __syncthreads):
//  0. gather  G_X = G[0:p, 0:p], G_XY = G[0:p, 1:p+1] in time order from the
//     ring-indexed physical G (p = c-1).
//  1. Householder tridiagonalisation of G_X: Q^T G_X Q = T (d, e).
//  2. the r largest eigenvalues of T by Sturm-count bisection (one thread
//     per eigenvalue).
//  3. their eigenvectors by inverse iteration on T (LU with partial
//     pivoting), re-orthogonalised inside clusters of close eigenvalues.
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
constexpr int kInvIters = 4;                     // inverse-iteration solves per vector
constexpr int kBisectMax = 160;                  // bisection iteration cap

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

// Fixed-order block sum (256 threads); every thread gets the result.
__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kWarps; ++w) t += red[w];
    red[kWarps] = t;
  }
  __syncthreads();
  const double t = red[kWarps];
  __syncthreads();
  return t;
}

// Number of eigenvalues of the symmetric tridiagonal (d, e) below x.
__device__ int sturm_count(const double* d, const double* e2, int p, double x, double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0.0) ++cnt;
  for (int i = 1; i < p; ++i) {
    q = (d[i] - x) - e2[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

struct WS {
  double *A, *GXY, *HV, *d, *e, *lam, *Z, *V, *Y, *At, *Hc, *Qc, *Wc, *M, *sig, *lamout, *tmp, *lu;
  float* Mf;
};

__device__ WS carve(double* base, const ModesLayout& L) {
  WS w;
  w.A = base + L.A;
  w.GXY = base + L.GXY;
  w.HV = base + L.HV;
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
  w.Mf = reinterpret_cast<float*>(base + L.Mf);
  return w;
}

// ---------------------------------------------------------------- phase 1 --
// Householder reduction of the symmetric p x p matrix A (row-major, full
// storage) to tridiagonal form. Reflector k is H_k = I - 2 v v^T acting on
// indices k+1..p-1, v unit (zero when column k is already reduced), stored in
// HV[k*p + 0..p-k-2].
__device__ void tridiagonalize(double* A, int p, double* d, double* e, double* HV, double* pv,
                               double* wv, double* red) {
  const int tid = threadIdx.x;
  for (int k = 0; k + 2 < p; ++k) {
    const int L = p - k - 1;
    const double* col = A + (int64_t)k * p + (k + 1);   // A[k][k+1..] == A[k+1..][k]
    double* v = HV + (int64_t)k * p;
    double tail = 0.0;
    for (int i = 1 + tid; i < L; i += kThreads) tail += col[i] * col[i];
    tail = block_sum(tail, red);
    const double x0 = col[0];
    if (tail == 0.0) {
      for (int i = tid; i < L; i += kThreads) v[i] = 0.0;
      if (tid == 0) {
        d[k] = A[(int64_t)k * p + k];
        e[k] = x0;
      }
      __syncthreads();
      continue;
    }
    const double nrm = sqrt(x0 * x0 + tail);
    const double alpha = (x0 >= 0.0) ? -nrm : nrm;
    const double v0 = x0 - alpha;                      // same sign as x0: no cancellation
    const double vn = sqrt(v0 * v0 + tail);
    for (int i = tid; i < L; i += kThreads) v[i] = (i == 0 ? v0 : col[i]) / vn;
    if (tid == 0) {
      d[k] = A[(int64_t)k * p + k];
      e[k] = alpha;
    }
    __syncthreads();
    // pv = A_sub v  (A_sub = A[k+1.., k+1..]); thread i reads column i = row i
    double* Asub = A + (int64_t)(k + 1) * p + (k + 1);
    for (int i = tid; i < L; i += kThreads) {
      double s = 0.0;
      for (int j = 0; j < L; ++j) s += Asub[(int64_t)j * p + i] * v[j];
      pv[i] = s;
    }
    __syncthreads();
    double kv = 0.0;
    for (int i = tid; i < L; i += kThreads) kv += v[i] * pv[i];
    kv = block_sum(kv, red);
    for (int i = tid; i < L; i += kThreads) wv[i] = 2.0 * pv[i] - 2.0 * kv * v[i];
    __syncthreads();
    // A_sub -= v w^T + w v^T  (H A_sub H)
    for (int idx = tid; idx < L * L; idx += kThreads) {
      const int i = idx / L, j = idx - i * L;
      Asub[(int64_t)i * p + j] -= v[i] * wv[j] + wv[i] * v[j];
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
    const double ax0 = cabs(x0);
    const double nrm = sqrt(ax0 * ax0 + tail);
    const C2 ph = (ax0 > 0.0) ? cscale(x0, 1.0 / ax0) : C2{1.0, 0.0};
    const C2 alpha = cscale(ph, -nrm);                 // -e^{i arg x0} |x|
    const C2 v0 = csub(x0, alpha);
    const double vn = sqrt(cabs2(v0) + tail);
    // v stored in ycol[0..L-1]
    for (int i = lane; i < L; i += 32) ycol[i] = cscale(i == 0 ? v0 : H[(j + 1 + i) * r + j], 1.0 / vn);
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
    // deflation scan
    int l = hi;
    while (l > 0) {
      const double sub = cabs(H[l * r + l - 1]);
      double scale = cabs(H[l * r + l]) + cabs(H[(l - 1) * r + l - 1]);
      if (scale == 0.0) scale = hnorm;
      if (sub <= kEps * scale) break;
      --l;
    }
    __syncwarp();
    if (l > 0 && lane == 0) H[l * r + l - 1] = {0.0, 0.0};
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
    // Wilkinson shift from the trailing 2 x 2 of the active block
    C2 mu;
    {
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
    for (int q = l + lane; q <= hi; q += 32) H[q * r + q] = csub(H[q * r + q], mu);
    __syncwarp();
    // H - mu I = Q R by Givens rotations on rows j, j+1
    for (int j = l; j < hi; ++j) {
      const C2 a = H[j * r + j], b = H[(j + 1) * r + j];
      const double aa = cabs(a), rho = hypot(aa, cabs(b));
      double c;
      C2 s;
      if (rho == 0.0) {
        c = 1.0;
        s = {0.0, 0.0};
      } else if (aa == 0.0) {
        c = 0.0;
        s = {1.0, 0.0};
      } else {
        c = aa / rho;
        s = cscale(cmul(cscale(a, 1.0 / aa), cconj(b)), 1.0 / rho);
      }
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

__global__ void __launch_bounds__(kThreads, 1) modes_small_kernel(ModesArgs a, ModesLayout L) {
  __shared__ double red[kWarps + 1];
  __shared__ int sh_reff;
  __shared__ double cs[SDMD_MAX_M];
  __shared__ C2 sn[SDMD_MAX_M];
  __shared__ int order[SDMD_MAX_M];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  WS w = carve(a.ws, L);
  const int m = a.m, p = a.c - 1;
  const int rw = min(a.r_req, p);   // eigenpairs of G_X to compute

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
    w.A[idx] = gx;
    w.GXY[idx] = gxy;
  }
  __syncthreads();

  // ---- 1. tridiagonalise G_X
  tridiagonalize(w.A, p, w.d, w.e, w.HV, w.tmp, w.tmp + p, red);

  // ---- 2. bisection for the rw largest eigenvalues
  double* e2 = w.tmp + 2 * p;
  for (int i = tid; i < p; i += kThreads) e2[i] = (i + 1 < p) ? w.e[i] * w.e[i] : 0.0;
  __syncthreads();
  double gl = 0.0, gu = 0.0, emax2 = 0.0;
  // Gershgorin interval and pivmin, computed redundantly by every thread
  for (int i = 0; i < p; ++i) {
    const double rad = ((i > 0) ? fabs(w.e[i - 1]) : 0.0) + ((i + 1 < p) ? fabs(w.e[i]) : 0.0);
    if (i == 0) {
      gl = w.d[0] - rad;
      gu = w.d[0] + rad;
    } else {
      gl = fmin(gl, w.d[i] - rad);
      gu = fmax(gu, w.d[i] + rad);
    }
    if (i + 1 < p) emax2 = fmax(emax2, w.e[i] * w.e[i]);
  }
  const double tnorm = fmax(fabs(gl), fabs(gu));
  const double pivmin = DBL_MIN * fmax(1.0, emax2);
  gl -= 2.0 * kEps * tnorm * p + 2.0 * pivmin;
  gu += 2.0 * kEps * tnorm * p + 2.0 * pivmin;
  for (int i = tid; i < rw; i += kThreads) {
    const int target = p - 1 - i;     // 0-based ascending index
    double lo = gl, hi = gu;
    for (int it = 0; it < kBisectMax; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (!(hi - lo > 2.0 * kEps * fmax(fabs(lo), fabs(hi)) + 4.0 * pivmin)) break;
      if (mid <= lo || mid >= hi) break;
      if (sturm_count(w.d, e2, p, mid, pivmin) > target)
        hi = mid;
      else
        lo = mid;
    }
    w.lam[i] = 0.5 * (lo + hi);
  }
  __syncthreads();

  // ---- 3. inverse iteration; clusters of close eigenvalues share a thread
  const double ortol = 1e-3 * tnorm;
  const double tiny = fmax(kEps * tnorm, DBL_MIN);
  for (int i0 = tid; i0 < rw; i0 += kThreads) {
    if (i0 > 0 && w.lam[i0 - 1] - w.lam[i0] <= ortol) continue;   // not a cluster start
    int i1 = i0;
    while (i1 + 1 < rw && w.lam[i1] - w.lam[i1 + 1] <= ortol) ++i1;
    double* u0 = w.lu + (int64_t)i0 * 5 * p;
    double *u1 = u0 + p, *u2 = u1 + p, *mu = u2 + p, *pv = mu + p;
    for (int i = i0; i <= i1; ++i) {
      double lam = w.lam[i];
      // separate (numerically) equal eigenvalues of a cluster, as inverse
      // iteration needs distinct shifts
      if (i > i0 && w.lam[i - 1] - lam < 10.0 * kEps * tnorm) lam = w.lam[i - 1] - 10.0 * kEps * tnorm;
      tri_lu(w.d, w.e, p, lam, tiny, u0, u1, u2, mu, pv);
      double* z = w.Z + (int64_t)i * p;
      for (int j = 0; j < p; ++j) z[j] = 1.0 + 0.1 * (double)(((j + 1) * 7919 + (i + 1) * 104729) % 97) / 97.0;
      for (int it = 0; it < kInvIters; ++it) {
        tri_solve(p, u0, u1, u2, mu, pv, z);
        for (int q = i0; q < i; ++q) {       // re-orthogonalise inside the cluster
          const double* zq = w.Z + (int64_t)q * p;
          double s = 0.0;
          for (int j = 0; j < p; ++j) s += zq[j] * z[j];
          for (int j = 0; j < p; ++j) z[j] -= s * zq[j];
        }
        double nn = 0.0;
        for (int j = 0; j < p; ++j) nn += z[j] * z[j];
        const double inv = (nn > 0.0) ? 1.0 / sqrt(nn) : 0.0;
        for (int j = 0; j < p; ++j) z[j] *= inv;
      }
    }
  }
  __syncthreads();

  // ---- 4. back-transform: v = H_0 H_1 ... H_{p-3} z  (warp per vector)
  for (int i = warp; i < rw; i += kWarps) {
    double* z = w.Z + (int64_t)i * p;
    for (int k = p - 3; k >= 0; --k) {
      const int Lk = p - k - 1;
      const double* v = w.HV + (int64_t)k * p;
      double s = 0.0;
      for (int j = lane; j < Lk; j += 32) s += v[j] * z[k + 1 + j];
      s = warp_sum(s);
      for (int j = lane; j < Lk; j += 32) z[k + 1 + j] -= 2.0 * s * v[j];
      __syncwarp();
    }
  }
  __syncthreads();

  // ---- 5. rank, sigma, vsi = V Sigma^-1 (in place in Z)
  if (tid == 0) {
    int k = 0;
    const double lam0 = (rw > 0) ? w.lam[0] : 0.0;
    if (lam0 > 0.0) {
      const double thr = lam0 * kRankRtol * (double)p * kEps;
      while (k < rw && w.lam[k] > thr) ++k;
    }
    sh_reff = k;
  }
  __syncthreads();
  const int re = sh_reff;
  for (int i = tid; i < a.r_req; i += kThreads) w.sig[i] = (i < re) ? sqrt(w.lam[i]) : 0.0;
  for (int idx = tid; idx < a.r_req * p; idx += kThreads) w.V[idx] = (idx / p < re) ? w.Z[idx] : 0.0;
  __syncthreads();
  for (int idx = tid; idx < re * p; idx += kThreads) {
    const int i = idx / p;
    w.Z[idx] /= w.sig[i];
  }
  __syncthreads();

  // ---- 6. A~ = vsi^T G_XY vsi  (Y = G_XY vsi first)
  for (int idx = tid; idx < re * p; idx += kThreads) {
    const int k = idx / p, row = idx - k * p;
    const double* g = w.GXY + (int64_t)row * p;
    const double* v = w.Z + (int64_t)k * p;
    double s = 0.0;
    for (int b = 0; b < p; ++b) s += g[b] * v[b];
    w.Y[idx] = s;
  }
  __syncthreads();
  C2* Hc = reinterpret_cast<C2*>(w.Hc);
  for (int idx = tid; idx < re * re; idx += kThreads) {
    const int k = idx / re, l = idx - k * re;
    const double* v = w.Z + (int64_t)k * p;
    const double* y = w.Y + (int64_t)l * p;
    double s = 0.0;
    for (int b = 0; b < p; ++b) s += v[b] * y[b];
    w.At[idx] = s;
    Hc[idx] = {s, 0.0};
  }
  __syncthreads();

  // ---- 7. eig(A~) on warp 0
  C2* Qc = reinterpret_cast<C2*>(w.Qc);
  C2* Wc = reinterpret_cast<C2*>(w.Wc);
  C2* ycol = reinterpret_cast<C2*>(w.lu);   // LU scratch is free again
  if (warp == 0 && re > 0) {
    const bool ok = warp_eig(Hc, Qc, Wc, ycol, re, cs, sn);
    if (!ok && lane == 0) atomicOr(a.status, kDevRank);
    if (lane == 0) {
      // order eigenpairs by descending |lambda|, then by angle
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
      for (int l = 0; l < re; ++l) s = cadd(s, cscale(Wc[l * re + kk], w.Z[(int64_t)l * p + row]));
    }
    Mc[idx] = s;
    w.Mf[2 * idx] = (float)s.re;
    w.Mf[2 * idx + 1] = (float)s.im;
  }
  if (tid == 0) *a.r_dev = re;
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
  L.HV = take(p2);
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
  L.total = o;
  return L;
}

int64_t modes_ws_doubles(int m) { return modes_layout(m).total; }

cudaError_t launch_modes_small(const ModesArgs& a, cudaStream_t st) {
  modes_small_kernel<<<1, kThreads, 0, st>>>(a, modes_layout(a.m));
  return cudaGetLastError();
}

}  // namespace sdmd
