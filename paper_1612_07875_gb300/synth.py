"""Seeded synthetic snapshot streams shaped like the paper's workloads.

This module holds no arithmetic of the method itself (no Gram, no SVD, no
DMD): it only draws inputs. Both the CUDA path's tests/bench and the CPU
oracle take their inputs from here. Every stream is a pure function of
(seed, t), so any snapshot can be regenerated on its own.

Streams:

* PlantedStream   -- dense FP32 field, side x side (n = side^2), a sum of
  planted spatial modes (periodic Gaussian-smoothed random fields, unit RMS)
  evolving with planted eigenvalues (conjugate pairs plus real modes, so the
  data are real), plus i.i.d. Gaussian noise. Noise-free it is exactly a
  linear system x_{k+1} = A x_k on the span of the modes.
* VideoStream     -- uint8 H x W x 3 frames: static smoothed-noise textured
  background in 0..200, moving solid rectangles (constant velocity, wrapping
  at the edges), integer-uniform pixel noise, clamped to 0..255.
* FourierSparseStream -- complex64 orthonormal 2-D Fourier coefficients of a
  periodic field, ~1% nonzero, support drawn with P(k) ~ |k|^-5/3, each
  coefficient rotating at a planted frequency with slow decay, with a small
  per-snapshot churn of the support.
* ConditionedStream -- dense FP32 snapshots whose windows have planted
  geometric singular values, for precision sweeps over cond(G).
"""
import numpy as np

SEED_BASE = 161207875


def config_seed(cfg_index):
    """Seed of synthetic configuration 1..5."""
    return SEED_BASE + int(cfg_index)


def smooth_periodic_field(shape, sigma_px, rng):
    """White noise smoothed by a periodic Gaussian (FFT), unit RMS."""
    white = rng.standard_normal(shape)
    freqs = [np.fft.fftfreq(s) for s in shape]
    k2 = np.zeros(shape)
    for ax, f in enumerate(freqs):
        sh = [1] * len(shape)
        sh[ax] = shape[ax]
        k2 = k2 + (f.reshape(sh)) ** 2
    kern = np.exp(-2.0 * np.pi ** 2 * sigma_px ** 2 * k2)
    field = np.fft.ifftn(np.fft.fftn(white) * kern).real
    field /= np.sqrt(np.mean(field ** 2))
    return field


class PlantedStream:
    """Dense FP32 stream of planted DMD modes (synthetic configuration 1)."""

    def __init__(self, side=64, n_pairs=2, n_real=1, noise_var=1e-3, sigma_px=3.0,
                 seed=config_seed(1)):
        rng = np.random.default_rng(seed)
        self.side = side
        self.n = side * side
        self.seed = seed
        self.noise_std = float(np.sqrt(noise_var))
        nf = 2 * n_pairs + n_real
        self.fields = np.stack([smooth_periodic_field((side, side), sigma_px, rng).reshape(-1)
                                for _ in range(nf)], axis=1)          # n x nf
        mod = rng.uniform(0.95, 1.0, n_pairs)
        ang = rng.uniform(0.15, np.pi - 0.15, n_pairs) * rng.choice([-1.0, 1.0], n_pairs)
        self.lam_pairs = mod * np.exp(1j * ang)
        self.lam_real = rng.uniform(0.95, 1.0, n_real)
        self.c_pairs = rng.uniform(0.5, 1.5, n_pairs) * np.exp(1j * rng.uniform(-np.pi, np.pi, n_pairs))
        self.c_real = rng.uniform(0.5, 1.5, n_real) * rng.choice([-1.0, 1.0], n_real)
        self.n_pairs = n_pairs
        self.n_real = n_real

    def planted_lambdas(self):
        return np.concatenate([self.lam_pairs, np.conj(self.lam_pairs),
                               self.lam_real.astype(np.complex128)])

    def planted_modes(self):
        """Complex spatial modes matching planted_lambdas() (up to scale)."""
        F = self.fields
        cols = []
        for p in range(self.n_pairs):
            cols.append(F[:, 2 * p] - 1j * F[:, 2 * p + 1])
        for p in range(self.n_pairs):
            cols.append(F[:, 2 * p] + 1j * F[:, 2 * p + 1])
        for q in range(self.n_real):
            cols.append(F[:, 2 * self.n_pairs + q].astype(np.complex128))
        return np.stack(cols, axis=1)

    def snapshot(self, t):
        F = self.fields
        x = np.zeros(self.n)
        for p in range(self.n_pairs):
            z = self.c_pairs[p] * self.lam_pairs[p] ** t
            x += z.real * F[:, 2 * p] + z.imag * F[:, 2 * p + 1]
        for q in range(self.n_real):
            x += self.c_real[q] * self.lam_real[q] ** t * F[:, 2 * self.n_pairs + q]
        if self.noise_std > 0:
            x += self.noise_std * np.random.default_rng([self.seed, 1, t]).standard_normal(self.n)
        return x.astype(np.float32)


class VideoStream:
    """uint8 HD-video-shaped frames (synthetic configuration 2), HWC order."""

    def __init__(self, H=1080, W=1920, C=3, n_rect=3, noise=4, seed=config_seed(2)):
        rng = np.random.default_rng(seed)
        self.H, self.W, self.C = H, W, C
        self.n = H * W * C
        self.seed = seed
        self.noise = int(noise)
        bg = np.empty((H, W, C))
        for ch in range(C):
            f = smooth_periodic_field((H, W), max(2.0, min(H, W) / 60.0), rng)
            f = (f - f.min()) / max(f.max() - f.min(), 1e-12)
            bg[:, :, ch] = 200.0 * f
        self.bg = np.rint(bg).astype(np.int16)
        lo = max(1, min(40, H // 4, W // 4))
        hi = max(lo + 1, min(200, H // 2, W // 2))
        self.rects = []
        for _ in range(n_rect):
            rh, rw = (int(v) for v in rng.integers(lo, hi + 1, 2))
            y0, x0 = int(rng.integers(0, H)), int(rng.integers(0, W))
            vy, vx = (int(v) for v in rng.integers(-8, 9, 2))
            if vx == 0 and vy == 0:
                vx = 3
            col = rng.integers(0, 256, C).astype(np.int16)
            self.rects.append((rh, rw, y0, x0, vy, vx, col))

    def frame(self, t):
        f = self.bg.copy()
        for (rh, rw, y0, x0, vy, vx, col) in self.rects:
            ys = (y0 + vy * t + np.arange(rh)) % self.H
            xs = (x0 + vx * t + np.arange(rw)) % self.W
            f[np.ix_(ys, xs)] = col
        if self.noise > 0:
            nz = np.random.default_rng([self.seed, 1, t]).integers(
                -self.noise, self.noise + 1, size=f.shape, dtype=np.int16)
            f += nz
        np.clip(f, 0, 255, out=f)
        return f.astype(np.uint8).reshape(-1)


class FourierSparseStream:
    """Sparse orthonormal 2-D Fourier coefficients (synthetic configuration 3).

    snapshot(t) -> (idx int32 sorted, val complex64). Linear index = iy*side+ix
    with ix, iy the numpy FFT bin numbers (0..side-1). The physical field is
    numpy.fft.ifft2(coeffs.reshape(side, side), norm="ortho").
    """

    def __init__(self, side=1024, nnz=10486, churn=0.10, seed=config_seed(3)):
        rng = np.random.default_rng(seed)
        self.side = side
        self.N = side * side
        self.seed = seed
        self.nnz = int(nnz)
        self.n_churn = int(round(churn * (self.nnz - 1)))
        kf = np.fft.fftfreq(side, 1.0 / side)
        kmag = np.sqrt(kf[None, :] ** 2 + kf[:, None] ** 2).reshape(-1)
        w = np.zeros(self.N)
        w[1:] = kmag[1:] ** (-5.0 / 3.0)
        w /= w.sum()
        # base support plus a reserve pool that churned-in entries come from
        npool = min(self.N - 1, (self.nnz - 1) + 4 * self.n_churn + 16)
        drawn = rng.choice(self.N, size=npool, replace=False, p=w)
        self.base = np.concatenate([[0], drawn[:self.nnz - 1]]).astype(np.int64)
        self.pool = drawn[self.nnz - 1:].astype(np.int64)
        allk = np.concatenate([self.base, self.pool])
        amp_scale = np.ones(allk.size)
        amp_scale[1:] = kmag[allk[1:]] ** (-5.0 / 6.0)
        amp = amp_scale * (rng.standard_normal(allk.size) + 1j * rng.standard_normal(allk.size))
        amp[0] = 4.0  # mean field
        omega = rng.uniform(-np.pi, np.pi, allk.size)
        omega[0] = 0.0
        rho = rng.uniform(0.995, 1.0, allk.size)
        rho[0] = 1.0
        self._coef = {int(k): (amp[i], omega[i], rho[i]) for i, k in enumerate(allk)}

    def support(self, t):
        if self.n_churn == 0:
            return np.sort(self.base)
        rng = np.random.default_rng([self.seed, 2, t])
        keep = np.ones(self.base.size, dtype=bool)
        drop = rng.choice(self.base.size - 1, size=self.n_churn, replace=False) + 1
        keep[drop] = False
        add = rng.choice(self.pool.size, size=self.n_churn, replace=False)
        return np.sort(np.concatenate([self.base[keep], self.pool[add]]))

    def snapshot(self, t):
        idx = self.support(t)
        val = np.empty(idx.size, dtype=np.complex128)
        for i, k in enumerate(idx):
            a, om, rh = self._coef[int(k)]
            val[i] = a * (rh ** t) * np.exp(1j * om * t)
        return idx.astype(np.int32), val.astype(np.complex64)

    def dense_coeffs(self, t):
        idx, val = self.snapshot(t)
        out = np.zeros(self.N, dtype=np.complex128)
        out[idx] = val.astype(np.complex128)
        return out

    def physical(self, t):
        c = self.dense_coeffs(t).reshape(self.side, self.side)
        return np.fft.ifft2(c, norm="ortho").reshape(-1)


class ConditionedStream:
    """Dense FP32 snapshots with planted geometric spectrum (configuration 4).

    x_t = sum_k s_k a_k(t) u_k with u_k orthonormal cosine/sine fields of
    distinct integer frequencies (exactly orthogonal for distinct k < n/2),
    a_k(t) i.i.d. N(0,1) temporal coefficients, and s_k geometric from 1 down
    to 1/sqrt(kappa). A window of m such snapshots has Gram condition number
    close to kappa (the ratio is measured, not assumed).
    """

    def __init__(self, n=1 << 22, K=256, kappa=1e4, seed=config_seed(4)):
        rng = np.random.default_rng(seed)
        self.n = int(n)
        self.K = int(K)
        self.seed = seed
        self.s = np.geomspace(1.0, 1.0 / np.sqrt(kappa), self.K)
        self.freq = 1 + rng.permutation(max(self.K, self.n // 2 - 2))[:self.K]
        self.phase_kind = rng.integers(0, 2, self.K)  # 0 = cos, 1 = sin

    def _basis(self, k, lo, hi):
        i = np.arange(lo, hi, dtype=np.float64)
        arg = 2.0 * np.pi * float(self.freq[k]) * i / self.n
        v = np.cos(arg) if self.phase_kind[k] == 0 else np.sin(arg)
        return v * np.sqrt(2.0 / self.n)

    def coeffs(self, t):
        return np.random.default_rng([self.seed, 1, t]).standard_normal(self.K)

    def snapshot(self, t, lo=0, hi=None):
        hi = self.n if hi is None else hi
        a = self.coeffs(t) * self.s
        x = np.zeros(hi - lo)
        for k in range(self.K):
            x += a[k] * self._basis(k, lo, hi)
        return (x * np.sqrt(self.n)).astype(np.float32)

    def snapshots(self, ts, lo=0, hi=None):
        """Positions lo .. hi - 1 of the snapshots for the times `ts` as a
        len(ts) x (hi - lo) float32 array: the same construction as
        `snapshot`, with the K basis fields built once and combined by one
        matrix product (faster for many snapshots). A full-length window can
        be drawn in position blocks; each block equals the same columns of
        the whole array."""
        hi = self.n if hi is None else hi
        B = np.stack([self._basis(k, lo, hi) for k in range(self.K)])        # K x (hi - lo)
        A = np.stack([self.coeffs(t) * self.s for t in ts])                  # T x K
        return ((A @ B) * np.sqrt(self.n)).astype(np.float32)


def random_dense(n, seed, dtype=np.float32):
    """i.i.d. test vector: N(0,1) floats or uniform 0..255 bytes."""
    rng = np.random.default_rng(seed)
    if dtype == np.uint8:
        return rng.integers(0, 256, n, dtype=np.uint8)
    return rng.standard_normal(n).astype(dtype)


class ServingMix:
    """Many concurrent streams for serving: per stream an element type (FP32
    or uint8, equally likely), n log-uniform in [2^lo, 2^hi], a window m drawn
    from `windows`, and Poisson frame arrivals at a rate uniform in
    [hz_lo, hz_hi]. Frame contents are windows of one seeded random pool per
    element type (the Gram row's cost does not depend on them)."""

    def __init__(self, streams=64, lo=16, hi=22, windows=(16, 32, 64, 128, 256), hz_lo=10.0, hz_hi=120.0,
                 seed=config_seed(5)):
        rng = np.random.default_rng(seed)
        self.seed = seed
        self.specs = []
        for _ in range(streams):
            kind = "u8" if rng.random() < 0.5 else "f32"
            n = int(round(2.0 ** rng.uniform(lo, hi)))
            m = int(rng.choice(windows))
            hz = float(rng.uniform(hz_lo, hz_hi))
            self.specs.append((kind, n, m, hz))
        self.pool_len = (1 << hi) + (1 << 16)

    def arrivals(self, seconds):
        """Per stream, sorted arrival times in seconds within [0, seconds)."""
        rng = np.random.default_rng(self.seed + 1)
        out = []
        for _, _, _, hz in self.specs:
            k = int(hz * seconds * 1.5) + 16
            t = np.cumsum(rng.exponential(1.0 / hz, k))
            out.append(t[t < seconds])
        return out

    def pools(self):
        """(uint8 pool, float32 pool), each pool_len long."""
        rng = np.random.default_rng(self.seed + 2)
        return (rng.integers(0, 256, self.pool_len, dtype=np.uint8),
                rng.standard_normal(self.pool_len, dtype=np.float32))

    def offset(self, i, j):
        """Start of stream i's j-th frame inside its pool."""
        n = self.specs[i][1]
        return (j * 4099 + i * 131) % (self.pool_len - n + 1)
