"""GPU parity of the SVD-only output and of the several-mode background
(sdmd_pod_modes: U = X V Sigma^-1, Sec. 2.1 Eq. 4; sdmd_reconstruct_ex with
SDMD_RECON_BACKGROUND_SLOW / _FOREGROUND_SLOW: Eq. 11 over every mode with
|log lambda| <= tol) against the CPU oracle on the same windows.

Tolerances: POD columns (unit norm, sign fixed) within 1e-3 for modes with
sigma_k >= 1e-2 sigma_1 and U^T U within 1e-3 of the identity there (FP32
products over the window, V and sigma from the FP64-class eigensolver);
slow-mode background / foreground columns within 1e-4 of the window's largest
snapshot norm, as the other reconstructions. The tolerance tol is put in the
middle of the widest gap between the oracle's |log lambda| values, so both
sides select the same modes.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1612_07875_gb300 import sdmd as S
from paper_1612_07875_gb300 import synth

pytestmark = pytest.mark.gpu


def _stream(kind, seed):
    if kind == "f32":
        ps = synth.PlantedStream(side=32, noise_var=1e-6, seed=seed)
        return ps.n, S.SDMD_F32, "f32", lambda t: ps.snapshot(t)
    vs = synth.VideoStream(H=24, W=40, C=3, seed=seed)
    return vs.n, S.SDMD_U8, "u8", lambda t: vs.frame(t)


def _fill(kind, seed, m, extra, dev):
    n, dt, ok, gen = _stream(kind, seed)
    h = S.sdmd_create(n, m, dt)
    so = oracle.StreamOracle(n, m, ok)
    for t in range(m + extra):
        x = gen(t)
        S.sdmd_push(h, torch.from_numpy(x).to(dev))
        so.push(x)
    return h, so, n


@pytest.mark.parametrize("kind,m,r", [("f32", 16, 5), ("u8", 12, 4), ("f32", 9, 8)])
def test_pod_modes_match_oracle(cuda_device, kind, m, r):
    h, so, n = _fill(kind, synth.config_seed(1) + m, m, 3, cuda_device)
    try:
        rout = np.zeros(1, dtype=np.int32)
        S.sdmd_modes(h, r, None, None, rout)
        U = torch.full((r, n), float("nan"), dtype=torch.float32, device=cuda_device)
        S.sdmd_pod_modes(h, r, U)
        torch.cuda.synchronize()
        U = U.cpu().numpy().astype(np.float64).T                    # n x r
        Uref, sref = oracle.pod_modes(so.window(), r)
        kept = int(rout[0])
        assert kept == Uref.shape[1]
        good = [k for k in range(kept) if sref[k] >= 1e-2 * sref[0]]
        assert good
        for k in good:
            sgn = np.sign(U[:, k] @ Uref[:, k])
            assert np.linalg.norm(U[:, k] - sgn * Uref[:, k]) <= 1e-3, k
        Ug = U[:, good]
        assert np.abs(Ug.T @ Ug - np.eye(len(good))).max() <= 1e-3
        assert not U[:, kept:].any()                                 # beyond the kept rank: zero
        sig = np.zeros(r)
        S.sdmd_svd(h, r, sig, None)
        torch.cuda.synchronize()
        assert np.abs(sig[:kept] ** 2 - sref ** 2).max() <= 1e-6 * sref[0] ** 2   # normwise
        assert S.sdmd_status(h) == S.SDMD_OK
    finally:
        S.sdmd_destroy(h)


@pytest.mark.parametrize("kind,m,r", [("f32", 16, 5), ("u8", 12, 6)])
def test_slow_mode_background_matches_oracle(cuda_device, kind, m, r):
    h, so, n = _fill(kind, synth.config_seed(2) + m, m, 4, cuda_device)
    try:
        S.sdmd_modes(h, r, None, None)
        S.sdmd_amplitudes(h, None, want_index=False)
        ref = so.modes(r)
        b = oracle.pod_amplitudes(ref)
        g = np.sort(np.abs(np.log(ref.lam)))
        gaps = np.diff(g)
        i = int(np.argmax(gaps))
        assert gaps[i] > 1e-3
        tol = 0.5 * (g[i] + g[i + 1])
        W = so.window()
        c = W.shape[1]
        scale = np.linalg.norm(W.astype(np.float64), axis=0).max()
        out = torch.empty(n, dtype=torch.float32, device=cuda_device)
        for t in (0, c // 2, c - 1):
            S.sdmd_reconstruct_ex(h, t, S.SDMD_RECON_BACKGROUND_SLOW, tol, out)
            torch.cuda.synchronize()
            exp = oracle.slow_background_column(ref, b, t, tol).real
            assert np.linalg.norm(out.cpu().numpy() - exp) <= 1e-4 * scale, ("background", t)
            S.sdmd_reconstruct_ex(h, t, S.SDMD_RECON_FOREGROUND_SLOW, tol, out)
            torch.cuda.synchronize()
            exp = oracle.slow_foreground_column(W, ref, b, t, tol)
            assert np.linalg.norm(out.cpu().numpy() - exp) <= 1e-4 * scale, ("foreground", t)
        # a tolerance above every |log lambda| gives the full reconstruction
        S.sdmd_reconstruct_ex(h, 1, S.SDMD_RECON_BACKGROUND_SLOW, 10.0, out)
        full = torch.empty_like(out)
        S.sdmd_reconstruct(h, 1, S.SDMD_RECON_MODES, full)
        torch.cuda.synchronize()
        assert torch.allclose(out, full, rtol=0, atol=1e-5 * float(scale))
        assert S.sdmd_status(h) == S.SDMD_OK
    finally:
        S.sdmd_destroy(h)


def test_pod_and_slow_error_paths(cuda_device):
    n, m = 300, 6
    rng = np.random.default_rng(4)
    h = S.sdmd_create(n, m, S.SDMD_F32)
    U = torch.zeros(3, n, dtype=torch.float32, device=cuda_device)
    out = torch.zeros(n, dtype=torch.float32, device=cuda_device)
    try:
        for _ in range(m):
            S.sdmd_push(h, torch.from_numpy(rng.standard_normal(n).astype(np.float32)).to(cuda_device))
        with pytest.raises(S.SdmdError) as ei:
            S.sdmd_pod_modes(h, 3, U)
        assert ei.value.code == S.SDMD_ERR_NOT_READY
        S.sdmd_modes(h, 3, None, None)
        for r, buf in ((2, U), (3, np.zeros((3, n), np.float32))):
            with pytest.raises(S.SdmdError) as ei:
                S.sdmd_pod_modes(h, r, buf)
            assert ei.value.code == S.SDMD_ERR_ARG
        with pytest.raises(S.SdmdError) as ei:                 # the slow variants need a tolerance
            S.sdmd_reconstruct(h, 0, S.SDMD_RECON_BACKGROUND_SLOW, out)
        assert ei.value.code == S.SDMD_ERR_ARG
        with pytest.raises(S.SdmdError) as ei:
            S.sdmd_reconstruct_ex(h, 0, S.SDMD_RECON_BACKGROUND_SLOW, -1.0, out)
        assert ei.value.code == S.SDMD_ERR_ARG
        S.sdmd_pod_modes(h, 3, U)
        assert S.sdmd_status(h) == S.SDMD_OK
    finally:
        S.sdmd_destroy(h)
    h = S.sdmd_create(n, m, S.SDMD_C64)
    try:
        with pytest.raises(S.SdmdError) as ei:
            S.sdmd_pod_modes(h, 3, U)
        assert ei.value.code == S.SDMD_ERR_UNSUPPORTED
    finally:
        S.sdmd_destroy(h)
