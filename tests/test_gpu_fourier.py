"""GPU parity of DMD entirely in Fourier coefficient space (Sec. 3.5): complex
small-matrix DMD on the sparse (Parseval) Gram and the compressed modes
Phi-hat = X'-hat M on the union of the X' supports (sdmd_modes +
sdmd_fourier_modes), and complex DMD of dense complex windows, against the
CPU oracle.

Tolerances: eigenvalues within 1e-6 (matched as multisets); the support
indices bit-exact; each mode's contribution b_k phi_k (independent of how W
is normalised) within 1e-4 of its 2-norm (FP32 M and products, FP64 small
algebra); sigma^2 within 1e-6 sigma_1^2 and complex V columns (sigma_k^2 >=
1e-2 sigma_1^2) within 1e-5 after fixing their phase.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1612_07875_gb300 import sdmd as S
from paper_1612_07875_gb300 import synth

from helpers import match_eigs, normalize_cols, rel_fro

pytestmark = pytest.mark.gpu


def _fill_sparse(fs, m, T):
    h = S.sdmd_create_sparse(fs.N, m, fs.nnz + 16)
    snaps = [fs.snapshot(t) for t in range(T)]
    for idx, val in snaps:
        S.sdmd_push_sparse(h, idx.size, idx, val.view(np.float32))
    return h, snaps[-min(T, m):]


def _modes(h, r):
    lam = np.zeros(2 * r)
    rout = np.zeros(1, dtype=np.int32)
    S.sdmd_modes(h, r, None, lam, rout)
    b = np.zeros(2 * r)
    S.sdmd_amplitudes(h, b, want_index=False)
    torch.cuda.synchronize()
    k = int(rout[0])
    return k, (lam[0::2] + 1j * lam[1::2])[:k], (b[0::2] + 1j * b[1::2])[:k]


def _fourier(h, r, dev):
    cnt = S.sdmd_fourier_modes(h, r)
    idx = torch.empty(max(cnt, 1), dtype=torch.int32, device=dev)
    phi = torch.empty(r, max(cnt, 1), 2, dtype=torch.float32, device=dev)
    assert S.sdmd_fourier_modes(h, r, idx, phi, cnt) == cnt
    torch.cuda.synchronize()
    ph = phi.cpu().numpy()
    return idx.cpu().numpy()[:cnt].astype(np.int64), (ph[..., 0] + 1j * ph[..., 1])[:, :cnt].T


def _check_modes_against_oracle(h, window, r, dev, rows=None):
    k, lam, b = _modes(h, r)
    ref = oracle.fourier_dmd(window, r)
    assert k == ref.r
    err, perm = match_eigs(lam, ref.lam)
    assert err <= 1e-6
    assert list(perm) == list(range(k))          # the same order (|lambda| desc, angle)
    sup, Phi = _fourier(h, r, dev)
    ref_sup = oracle.fourier_support(window)
    assert np.array_equal(sup, ref_sup)
    b_ref = oracle.pod_amplitudes(ref)
    sel = np.arange(sup.size) if rows is None else rows(sup.size)
    ref_rows = oracle.fourier_phi_rows(window, ref.M, sup[sel])
    for q in range(k):
        got = b[q] * Phi[sel, q]
        exp = b_ref[q] * ref_rows[:, q]
        assert np.linalg.norm(got - exp) <= 1e-4 * np.linalg.norm(exp), q
    assert S.sdmd_status(h) == S.SDMD_OK
    return ref


@pytest.mark.parametrize("side,nnz,m,r,T", [(64, 400, 16, 6, 20), (32, 100, 9, 8, 9), (128, 1500, 24, 10, 30)])
def test_fourier_modes_match_oracle(cuda_device, side, nnz, m, r, T):
    fs = synth.FourierSparseStream(side=side, nnz=nnz, churn=0.1, seed=synth.config_seed(3) + side)
    h, window = _fill_sparse(fs, m, T)
    try:
        _check_modes_against_oracle(h, window, r, cuda_device)
    finally:
        S.sdmd_destroy(h)


def test_fourier_modes_full_configuration(cuda_device):
    # 1024 x 1024 field, ~1 % nonzero coefficients, window 64, r = 10: the
    # eigenvalues, the support and 400 sampled rows of Phi-hat
    fs = synth.FourierSparseStream(seed=synth.config_seed(3))
    rng = np.random.default_rng(0)
    h, window = _fill_sparse(fs, 64, 66)
    try:
        _check_modes_against_oracle(h, window, 10, cuda_device,
                                    rows=lambda u: np.unique(np.concatenate([np.arange(200),
                                                                             rng.integers(0, u, 200)])))
    finally:
        S.sdmd_destroy(h)


def test_dense_complex_window_equals_its_coefficients(cuda_device):
    # Parseval: the physical complex fields and their Fourier coefficients
    # have the same Gram, so the same eigenvalues and the same sigma; V
    # (complex) against the oracle's up to each column's phase
    fs = synth.FourierSparseStream(side=32, nnz=120, churn=0.1, seed=17)
    m, r, T = 12, 6, 14
    hd = S.sdmd_create(fs.N, m, S.SDMD_C64)
    hs, window = _fill_sparse(fs, m, T)
    try:
        for t in range(T):
            x = fs.physical(t).astype(np.complex64)
            S.sdmd_push(hd, torch.from_numpy(x.view(np.float32)).to(cuda_device))
        kd, lam_d, _ = _modes(hd, r)
        ks, lam_s, _ = _modes(hs, r)
        W = np.stack([fs.physical(t) for t in range(T - m, T)], axis=1).astype(np.complex64)
        ref = oracle.exact_dmd(W, r)
        assert kd == ks == ref.r
        assert match_eigs(lam_d, ref.lam)[0] <= 1e-6
        assert match_eigs(lam_s, lam_d)[0] <= 1e-6
        sig = np.zeros(r)
        V = np.zeros(2 * r * (m - 1))
        S.sdmd_svd(hd, r, sig, V)
        torch.cuda.synchronize()
        assert np.abs(sig[:kd] ** 2 - ref.sigma ** 2).max() <= 1e-6 * ref.sigma[0] ** 2   # normwise
        Vc = (V[0::2] + 1j * V[1::2]).reshape(r, m - 1)
        for q in range(kd):
            if ref.sigma[q] ** 2 < 1e-2 * ref.sigma[0] ** 2:
                continue
            v, w = Vc[q], ref.V[:, q]
            ph = np.vdot(v, w) / abs(np.vdot(v, w))
            assert np.linalg.norm(v * ph - w) <= 1e-5, q
        # dense complex Phi = X' M of the physical window against the oracle's
        phi = torch.zeros(r, fs.N, 2, dtype=torch.float32, device=cuda_device)
        lam = np.zeros(2 * r)
        S.sdmd_modes(hd, r, phi, lam)
        torch.cuda.synchronize()
        P = phi.cpu().numpy()
        got = (P[..., 0] + 1j * P[..., 1]).T[:, :kd]
        err, perm = match_eigs((lam[0::2] + 1j * lam[1::2])[:kd], ref.lam)
        assert rel_fro(normalize_cols(got), normalize_cols(ref.Phi[:, perm])) <= 1e-4
        with pytest.raises(S.SdmdError) as ei:                    # Fourier-sparse: no dense Phi
            S.sdmd_modes(hs, r, torch.empty(r, fs.N, 2, device=cuda_device), None)
        assert ei.value.code == S.SDMD_ERR_UNSUPPORTED
        assert S.sdmd_status(hd) == S.SDMD_OK and S.sdmd_status(hs) == S.SDMD_OK
    finally:
        S.sdmd_destroy(hd)
        S.sdmd_destroy(hs)


def test_fourier_modes_error_paths(cuda_device):
    fs = synth.FourierSparseStream(side=32, nnz=60, churn=0.1, seed=3)
    h, _ = _fill_sparse(fs, 8, 10)
    hd = S.sdmd_create(100, 8, S.SDMD_F32)
    try:
        with pytest.raises(S.SdmdError) as ei:
            S.sdmd_fourier_modes(h, 4)
        assert ei.value.code == S.SDMD_ERR_NOT_READY
        S.sdmd_modes(h, 4, None, None)
        with pytest.raises(S.SdmdError) as ei:
            S.sdmd_fourier_modes(h, 3)
        assert ei.value.code == S.SDMD_ERR_ARG
        cnt = S.sdmd_fourier_modes(h, 4)
        assert cnt > 1
        idx = torch.empty(cnt, dtype=torch.int32, device=cuda_device)
        phi = torch.empty(4, cnt, 2, dtype=torch.float32, device=cuda_device)
        with pytest.raises(S.SdmdError) as ei:                    # cap too small
            S.sdmd_fourier_modes(h, 4, idx, phi, cnt - 1)
        assert ei.value.code == S.SDMD_ERR_ARG
        with pytest.raises(S.SdmdError) as ei:
            S.sdmd_fourier_modes(hd, 4)
        assert ei.value.code == S.SDMD_ERR_UNSUPPORTED
        assert S.sdmd_status(h) == S.SDMD_OK
    finally:
        S.sdmd_destroy(h)
        S.sdmd_destroy(hd)


@pytest.mark.parametrize("n,m,r", [(40000 + 37, 20, 7), (3 * 65536 + 5, 40, 18)])
def test_dense_complex_phi_matches_oracle(cuda_device, n, m, r):
    # complex64 windows of planted rotating modes plus noise: Phi = X' M on
    # the CUDA cores (several position tiles, a ragged tail, one or two mode
    # passes) against the oracle's DMD from the same Gram and its product
    # X' M; columns compared after normalisation (unit norm, phase of the
    # largest entry)
    rng = np.random.default_rng(n + m)
    k = 5
    F = rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))
    lam_p = 0.98 * np.exp(1j * rng.uniform(-np.pi, np.pi, k))
    c0 = rng.standard_normal(k) + 1j * rng.standard_normal(k)
    T = m + 3
    frames = [(F @ (c0 * lam_p ** t) + 1e-3 * (rng.standard_normal(n) + 1j * rng.standard_normal(n)))
              .astype(np.complex64) for t in range(T)]
    h = S.sdmd_create(n, m, S.SDMD_C64)
    try:
        for x in frames:
            S.sdmd_push(h, torch.from_numpy(x.view(np.float32)).to(cuda_device))
        phi = torch.zeros(r, n, 2, dtype=torch.float32, device=cuda_device)
        lam = np.zeros(2 * r)
        rk = np.zeros(1, dtype=np.int32)
        S.sdmd_modes(h, r, phi, lam, rk)
        torch.cuda.synchronize()
        # the oracle's algebra on the device's own Gram (same-input parity: the
        # FP32-product Gram's rounding is not Phi's), Phi = X' M by the oracle
        G = np.zeros((m, m, 2))
        S.sdmd_gram(h, G)
        Gc = G[..., 0] + 1j * G[..., 1]
        ref = oracle.dmd_from_gram(Gc[:-1, :-1], Gc[:-1, 1:], r)
        kept = int(rk[0])
        assert kept == ref.r
        lg = (lam[0::2] + 1j * lam[1::2])[:kept]
        err, perm = match_eigs(lg, ref.lam)
        assert err <= 1e-6                       # the eigenvalue tolerance (FP32 Schur + FP64 refinement)
        Xp = np.stack(frames[-(m - 1):], axis=1).astype(np.complex128)
        Pref = Xp @ ref.M[:, perm]
        P = phi.cpu().numpy()
        got = (P[..., 0] + 1j * P[..., 1]).T
        # the planted modes are well separated from the noise ones: their columns
        big = [q for q in range(kept) if abs(lg[q]) > 0.9]
        assert len(big) >= k - 1
        assert rel_fro(normalize_cols(got[:, big]), normalize_cols(Pref[:, big])) <= 1e-4
        assert np.all(got[:, kept:] == 0)
        assert S.sdmd_status(h) == S.SDMD_OK
    finally:
        S.sdmd_destroy(h)


@pytest.mark.parametrize("n,m,r,noise", [(5000, 64, 5, 0.01), (4096, 64, 10, 0.01), (3000, 33, 10, 0.01),
                                         (6000, 50, 8, 0.3)])
def test_complex_eigensolver_paths_on_same_gram(cuda_device, n, m, r, noise):
    # Complex windows of up to 72 snapshots take the real df64 eigensolver on
    # the 2p x 2p real embedding of G_X; when its df64 Sturm count finds an
    # eigenvalue above the smallest kept one that it did not return (the r
    # requested include a noise floor below the FP32 multisection's
    # resolution: the r = 10 cases with 6 planted modes and noise 0.01), the
    # FP64 Jacobi runs instead. Either way: rank, sigma (1e-10 relative) and
    # lambda (1e-9) against the oracle's LAPACK DMD of the device's own G.
    rng = np.random.default_rng(n + m + r)
    modes = rng.standard_normal((n, 6)) + 1j * rng.standard_normal((n, 6))
    lamt = np.exp(1j * rng.uniform(0, 1, 6)) * rng.uniform(0.95, 1.0, 6)
    X = np.stack([(modes * lamt ** t).sum(1) + noise * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
                  for t in range(m)]).astype(np.complex64)
    h = S.sdmd_create(n, m, S.SDMD_C64)
    try:
        for t in range(m):
            S.sdmd_push(h, torch.from_numpy(X[t].view(np.float32).reshape(n, 2)).to(cuda_device))
        G = torch.empty(m, m, dtype=torch.complex128, device=cuda_device)
        S.sdmd_gram(h, G)
        lam = np.zeros(2 * r)
        rout = np.zeros(1, dtype=np.int32)
        S.sdmd_modes(h, r, None, lam, rout)
        sig = np.zeros(r)
        S.sdmd_svd(h, r, sig, None)
        torch.cuda.synchronize()
        assert S.sdmd_status(h) == S.SDMD_OK
        Gn = G.cpu().numpy()
        ref = oracle.dmd_from_gram(Gn[:-1, :-1], Gn[:-1, 1:], r)
        rk = int(rout[0])
        assert rk == ref.r
        assert np.allclose(sig[:rk], ref.sigma, rtol=1e-10, atol=0)
        err, _ = match_eigs((lam[0::2] + 1j * lam[1::2])[:rk], ref.lam)
        assert err <= 1e-9, err
    finally:
        S.sdmd_destroy(h)
