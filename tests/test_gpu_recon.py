"""GPU parity of the reconstruction, the mode amplitudes and the background /
foreground split (Sec. 2.2 Eq. 11, Sec. 3.3 Eq. 14a-e, Algorithm 3) against
the CPU oracle on the same windows.

Tolerance: every reconstructed column within 1e-4 of the window snapshot's
2-norm (the GPU keeps eigenvalues to FP64 accuracy but W and M = V Sigma^-1 W
in FP32); background eigenvalue within 1e-6 of the oracle's.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1612_07875_gb300 import sdmd as S
from paper_1612_07875_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _recon(h, t, what, n, dev):
    out = torch.full((n,), float("nan"), dtype=torch.float32, device=dev)
    S.sdmd_reconstruct(h, t, what, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def _lam(buf):
    return buf[0::2] + 1j * buf[1::2]


def _check_window(h, so, r, dev, ts):
    W = so.window()
    n, c = W.shape
    ref = so.modes(r)
    b_ref = oracle.pod_amplitudes(ref)
    lam = np.zeros(2 * r)
    rout = np.zeros(1, dtype=np.int32)
    S.sdmd_modes(h, r, None, lam, rout)
    torch.cuda.synchronize()
    assert int(rout[0]) == ref.r
    got_lam = _lam(lam)[:ref.r]
    bbuf = np.zeros(2 * r)
    bi = S.sdmd_amplitudes(h, bbuf)
    assert 0 <= bi < ref.r
    assert abs(got_lam[bi] - ref.lam[oracle.background_index(ref.lam)]) <= 1e-6
    assert np.isfinite(bbuf).all()
    scale = np.linalg.norm(W.astype(np.float64), axis=0).max()
    for t in ts:
        got = _recon(h, t, S.SDMD_RECON_MODES, n, dev)
        exp = oracle.reconstruct(ref, b_ref, t).real
        assert np.linalg.norm(got - exp) <= TOL * scale, ("modes", t)
    for t in (0, c // 2, c - 1):
        got = _recon(h, t, S.SDMD_RECON_BACKGROUND, n, dev)
        exp = oracle.background_column(ref, b_ref, t).real
        assert np.linalg.norm(got - exp) <= TOL * scale, ("background", t)
        got = _recon(h, t, S.SDMD_RECON_FOREGROUND, n, dev)
        exp = oracle.foreground_column(W, ref, b_ref, t)
        assert np.linalg.norm(got - exp) <= TOL * scale, ("foreground", t)
    assert S.sdmd_status(h) == S.SDMD_OK
    return ref


def test_reconstruct_planted_f32_matches_oracle(cuda_device):
    ps = synth.PlantedStream(side=32, noise_var=1e-6, seed=synth.config_seed(1))
    n, m, r = ps.n, 16, 5
    h = S.sdmd_create(n, m, S.SDMD_F32)
    so = oracle.StreamOracle(n, m, "f32")
    try:
        for t in range(m + 4):
            x = ps.snapshot(t)
            S.sdmd_push(h, torch.from_numpy(x).to(cuda_device))
            so.push(x)
        ref = _check_window(h, so, r, cuda_device, ts=(0, 3, m - 1, m + 3))
        # the planted data are nearly linear: the modes reproduce the window
        W = so.window()
        got = _recon(h, m - 1, S.SDMD_RECON_MODES, n, cuda_device)
        assert np.linalg.norm(got - W[:, -1]) <= 1e-2 * np.linalg.norm(W[:, -1])
        assert ref.r == r
    finally:
        S.sdmd_destroy(h)


@pytest.mark.parametrize("shape", [(36, 64, 3), (7, 11, 13)])   # n = 6912 and a ragged 1001
def test_background_foreground_u8_video_matches_oracle(cuda_device, shape):
    H, Wd, C = shape
    vs = synth.VideoStream(H=H, W=Wd, C=C, seed=synth.config_seed(2))
    m, r = 12, 6
    h = S.sdmd_create(vs.n, m, S.SDMD_U8)
    so = oracle.StreamOracle(vs.n, m, "u8")
    try:
        for t in range(m + 3):
            f = vs.frame(t)
            S.sdmd_push(h, torch.from_numpy(f).to(cuda_device))
            so.push(f)
        _check_window(h, so, r, cuda_device, ts=(0, m - 1))
    finally:
        S.sdmd_destroy(h)


def test_reconstruct_ramp_up_window(cuda_device):
    # fewer snapshots than the window: c = 6 of m = 16
    ps = synth.PlantedStream(side=16, noise_var=1e-6, seed=synth.config_seed(1) + 5)
    n, m, r = ps.n, 16, 3
    h = S.sdmd_create(n, m, S.SDMD_F32)
    so = oracle.StreamOracle(n, m, "f32")
    try:
        for t in range(6):
            x = ps.snapshot(t)
            S.sdmd_push(h, torch.from_numpy(x).to(cuda_device))
            so.push(x)
        _check_window(h, so, r, cuda_device, ts=(0, 5))
    finally:
        S.sdmd_destroy(h)


def test_reconstruct_error_paths(cuda_device):
    n, m = 256, 6
    rng = np.random.default_rng(9)
    h = S.sdmd_create(n, m, S.SDMD_F32)
    out = torch.zeros(n + 4, dtype=torch.float32, device=cuda_device)
    try:
        for _ in range(m):
            S.sdmd_push(h, torch.from_numpy(rng.standard_normal(n).astype(np.float32)).to(cuda_device))
        with pytest.raises(S.SdmdError) as ei:                      # no modes yet
            S.sdmd_reconstruct(h, 0, S.SDMD_RECON_MODES, out)
        assert ei.value.code == S.SDMD_ERR_NOT_READY
        with pytest.raises(S.SdmdError) as ei:
            S.sdmd_amplitudes(h, None)
        assert ei.value.code == S.SDMD_ERR_NOT_READY
        S.sdmd_modes(h, 3, None, None)
        S.sdmd_reconstruct(h, 0, S.SDMD_RECON_MODES, out)
        for t, what in ((m, S.SDMD_RECON_FOREGROUND), (-1, S.SDMD_RECON_MODES), (0, 7)):
            with pytest.raises(S.SdmdError) as ei:
                S.sdmd_reconstruct(h, t, what, out)
            assert ei.value.code == S.SDMD_ERR_ARG
        with pytest.raises(S.SdmdError) as ei:                      # 4-byte offset: misaligned
            S.sdmd_reconstruct(h, 0, S.SDMD_RECON_MODES, out[1:])
        assert ei.value.code == S.SDMD_ERR_ARG
        with pytest.raises(S.SdmdError) as ei:                      # host output
            S.sdmd_reconstruct(h, 0, S.SDMD_RECON_MODES, np.zeros(n, np.float32))
        assert ei.value.code == S.SDMD_ERR_ARG
        S.sdmd_push(h, torch.from_numpy(rng.standard_normal(n).astype(np.float32)).to(cuda_device))
        with pytest.raises(S.SdmdError) as ei:                      # window moved since modes
            S.sdmd_reconstruct(h, 0, S.SDMD_RECON_MODES, out)
        assert ei.value.code == S.SDMD_ERR_NOT_READY
        assert S.sdmd_status(h) == S.SDMD_OK
    finally:
        S.sdmd_destroy(h)
    h = S.sdmd_create(n, m, S.SDMD_C64)
    try:
        with pytest.raises(S.SdmdError) as ei:
            S.sdmd_reconstruct(h, 0, S.SDMD_RECON_MODES, out)
        assert ei.value.code == S.SDMD_ERR_UNSUPPORTED
    finally:
        S.sdmd_destroy(h)


def test_reconstruct_on_pipelined_handle_follows_serial_modes(cuda_device):
    # sdmd_step frames keep their results per frame; a serial sdmd_modes call
    # on the same handle is what sdmd_reconstruct reads
    ps = synth.PlantedStream(side=16, noise_var=1e-6, seed=synth.config_seed(1) + 7)
    n, m, r = ps.n, 10, 3
    h = S.sdmd_create_ex(n, m, S.SDMD_F32, 3)
    so = oracle.StreamOracle(n, m, "f32")
    out = torch.zeros(n, dtype=torch.float32, device=cuda_device)
    try:
        for t in range(m + 2):
            x = ps.snapshot(t)
            S.sdmd_step(h, torch.from_numpy(x).to(cuda_device), r, None, None, None)
            so.push(x)
        with pytest.raises(S.SdmdError) as ei:      # only steps so far
            S.sdmd_reconstruct(h, 0, S.SDMD_RECON_MODES, out)
        assert ei.value.code == S.SDMD_ERR_NOT_READY
        S.sdmd_sync(h, None)
        _check_window(h, so, r, cuda_device, ts=(0, m - 1))
    finally:
        S.sdmd_destroy(h)
