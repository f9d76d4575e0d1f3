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

from helpers import match_eigs

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
        with pytest.raises(S.SdmdError) as ei:                    # no dense complex Phi
            S.sdmd_modes(hd, r, torch.empty(r, fs.N, 2, device=cuda_device), None)
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
