"""GPU parity of the exact-DMD step (sdmd_modes / sdmd_svd) against the oracle.

Two kinds of check:
* same-input parity: the oracle's FP64 dense DMD (numpy/LAPACK) run on the
  GPU's own G, so only the eigensolvers and small products are compared;
* end-to-end parity: the oracle recomputes G from the window (exact for
  uint8) and everything after; eigenvalues within 1e-6 absolute.
Phi is compared column by column after fixing each column's scale and phase.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1612_07875_gb300 import sdmd as S
from paper_1612_07875_gb300 import synth

from helpers import col_cos, match_eigs, normalize_cols, rel_fro

pytestmark = pytest.mark.gpu

EIG_TOL = 1e-6


def _stream(h, so, frames, dev):
    for x in frames:
        S.sdmd_push(h, torch.from_numpy(x).to(dev))
        so.push(x)


def _modes(h, n, r, dev, c):
    phi = torch.zeros(r, n, 2, dtype=torch.float32, device=dev)
    lam = np.zeros(2 * r)
    rout = np.zeros(1, np.int32)
    S.sdmd_modes(h, r, phi, lam, rout)
    sig = np.zeros(r)
    V = np.zeros(r * (c - 1))
    S.sdmd_svd(h, r, sig, V)
    torch.cuda.synchronize()
    assert S.sdmd_status(h) == S.SDMD_OK
    P = phi.cpu().numpy()
    P = (P[..., 0] + 1j * P[..., 1]).T          # n x r
    return int(rout[0]), lam[0::2] + 1j * lam[1::2], sig, V.reshape(r, c - 1).T, P


def _gram(h, c, dev, is_u8):
    G = torch.empty(c, c, dtype=torch.int64 if is_u8 else torch.float64, device=dev)
    S.sdmd_gram(h, G)
    torch.cuda.synchronize()
    return G.cpu().numpy().astype(np.float64)


def _compare_same_input(G, rk, lam, sig, V, r):
    ref = oracle.dmd_from_gram(G[:-1, :-1], G[:-1, 1:], r)
    assert rk == ref.r
    assert np.allclose(sig[:rk], ref.sigma, rtol=1e-10, atol=0)
    err, _ = match_eigs(lam[:rk], ref.lam)
    assert err <= 1e-9, err
    assert (col_cos(V[:, :rk], ref.V) > 1 - 1e-9).all()
    assert np.all(lam[rk:] == 0)
    return ref


def test_planted_fp32_config1_shape(cuda_device):
    # Synthetic configuration 1: 64x64 field, window 32, r = 10, noise var 1e-3.
    ps = synth.PlantedStream(seed=synth.config_seed(1))
    n, m, r, T = ps.n, 32, 10, 60
    h = S.sdmd_create(n, m, S.SDMD_F32)
    so = oracle.StreamOracle(n, m, "f32")
    try:
        _stream(h, so, [ps.snapshot(t) for t in range(T)], cuda_device)
        rk, lam, sig, V, P = _modes(h, n, r, cuda_device, m)
        G = _gram(h, m, cuda_device, False)
        ref = _compare_same_input(G, rk, lam, sig, V, r)
        # Phi = X' M: oracle product with the oracle's M on the same window
        W = so.window()
        Pref = W[:, 1:].astype(np.float64) @ ref.M
        _, perm = match_eigs(lam[:rk], ref.lam)
        Pn = normalize_cols(P[:, :rk])
        Rn = normalize_cols(Pref[:, perm])
        assert rel_fro(Pn, Rn) <= 1e-4
        assert np.all(P[:, rk:] == 0)
        # end-to-end: the 5 planted (signal) eigenvalues agree with the oracle
        # that recomputes G from the window
        full = so.modes(5)
        rk5, lam5, *_ = _modes(h, n, 5, cuda_device, m)
        err, _ = match_eigs(lam5[:rk5], full.lam)
        assert rk5 == 5 and err <= EIG_TOL, err
    finally:
        S.sdmd_destroy(h)


def test_u8_video_end_to_end_exact_gram(cuda_device):
    vs = synth.VideoStream(H=72, W=128, C=3, seed=synth.config_seed(2))
    n, m, r, T = vs.n, 20, 8, 27
    h = S.sdmd_create(n, m, S.SDMD_U8)
    so = oracle.StreamOracle(n, m, "u8")
    try:
        _stream(h, so, [vs.frame(t) for t in range(T)], cuda_device)
        rk, lam, sig, V, P = _modes(h, n, r, cuda_device, m)
        ref = so.modes(r)
        assert rk == ref.r
        err, perm = match_eigs(lam[:rk], ref.lam)
        assert err <= EIG_TOL, err
        assert np.allclose(sig[:rk], ref.sigma, rtol=1e-10)
        Pn = normalize_cols(P[:, :rk])
        Rn = normalize_cols(ref.Phi[:, perm])
        assert rel_fro(Pn, Rn) <= 1e-4
    finally:
        S.sdmd_destroy(h)


@pytest.mark.parametrize("seed_off,T", [(0, 32), (0, 45), (3, 32), (5, 40), (11, 33)])
def test_planted_fp32_noise_floor_cluster(cuda_device, seed_off, T):
    # r = 10 on a window with 5 planted modes: the other 5 requested
    # eigenvalues sit in the noise floor's cluster, where inverse iteration
    # needs its Gram-Schmidt / Rayleigh-Ritz rounds to resolve the subspace.
    ps = synth.PlantedStream(seed=synth.config_seed(1) + seed_off)
    n, m, r = ps.n, 32, 10
    h = S.sdmd_create(n, m, S.SDMD_F32)
    so = oracle.StreamOracle(n, m, "f32")
    try:
        _stream(h, so, [ps.snapshot(t) for t in range(T)], cuda_device)
        rk, lam, sig, V, _ = _modes(h, n, r, cuda_device, m)
        G = _gram(h, m, cuda_device, False)
        _compare_same_input(G, rk, lam, sig, V, r)
    finally:
        S.sdmd_destroy(h)


@pytest.mark.parametrize("noise_var,seed_off", [(1e-8, 0), (1e-10, 2), (1e-9, 4)])
def test_noise_floor_below_fp32_resolution(cuda_device, noise_var, seed_off):
    # r = 10 with 5 planted modes reaches into a noise floor 1e-8 .. 1e-10 of
    # lambda_1: above the rank threshold, below what the FP32 multisection
    # resolves. The kept eigenvalues must still be the r largest of G_X: sigma^2
    # within 1e-12 lambda_1 of the oracle's (the noise eigenvalues are about
    # 1e-11 lambda_1 apart, and the df64 and LAPACK backward errors are
    # relative to lambda_1, so sigma of a noise mode is not compared relatively).
    ps = synth.PlantedStream(noise_var=noise_var, seed=synth.config_seed(1) + 20 + seed_off)
    n, m, r = ps.n, 32, 10
    h = S.sdmd_create(n, m, S.SDMD_F32)
    so = oracle.StreamOracle(n, m, "f32")
    try:
        _stream(h, so, [ps.snapshot(t) for t in range(40)], cuda_device)
        rk, lam, sig, V, _ = _modes(h, n, r, cuda_device, m)
        G = _gram(h, m, cuda_device, False)
        ref = oracle.dmd_from_gram(G[:-1, :-1], G[:-1, 1:], r)
        assert rk == ref.r
        l1 = ref.sigma[0] ** 2
        assert np.max(np.abs(sig[:rk] ** 2 - ref.sigma ** 2)) <= 1e-12 * l1
    finally:
        S.sdmd_destroy(h)


def test_ramp_up_window_not_full(cuda_device):
    ps = synth.PlantedStream(side=24, noise_var=1e-4, seed=77)
    n, m = ps.n, 32
    h = S.sdmd_create(n, m, S.SDMD_F32)
    so = oracle.StreamOracle(n, m, "f32")
    try:
        _stream(h, so, [ps.snapshot(t) for t in range(9)], cuda_device)
        rk, lam, sig, V, P = _modes(h, n, 5, cuda_device, 9)
        G = _gram(h, 9, cuda_device, False)
        _compare_same_input(G, rk, lam, sig, V, 5)
        ref = so.modes(5)
        err, _ = match_eigs(lam[:rk], ref.lam)
        assert err <= EIG_TOL
    finally:
        S.sdmd_destroy(h)


def test_rank_clamped_to_numerical_rank(cuda_device):
    # uint8 frames that are integer combinations of 3 patterns: X has rank 3
    # exactly and G is exact, so exactly 3 modes survive the FP64 floor.
    rng = np.random.default_rng(3)
    n, m = 2000, 12
    P = rng.integers(0, 41, (3, n))
    frames = [(rng.integers(0, 3, 3) @ P).astype(np.uint8) for _ in range(m)]
    h = S.sdmd_create(n, m, S.SDMD_U8)
    so = oracle.StreamOracle(n, m, "u8")
    try:
        _stream(h, so, frames, cuda_device)
        rk, lam, sig, V, P_ = _modes(h, n, 8, cuda_device, m)
        ref = so.modes(8)
        assert ref.r == 3 and rk == 3
        assert np.all(lam[3:] == 0) and np.all(sig[3:] == 0) and np.all(P_[:, 3:] == 0)
        err, _ = match_eigs(lam[:3], ref.lam)
        assert err <= EIG_TOL
    finally:
        S.sdmd_destroy(h)


def test_cluster_at_the_requested_boundary(cuda_device):
    # Five planted modes plus noise: the three noise eigenvalues of G_X lie
    # closer together than FP32 resolves, so requesting 6, 7 or all 8 of them
    # cuts a cluster; every requested eigenvalue and the kept rank must still
    # match the FP64 eigenvalues of the same G (same-input parity).
    ps = synth.PlantedStream(side=32, noise_var=1e-6, seed=synth.config_seed(1) + 9)
    n, m = ps.n, 9
    h = S.sdmd_create(n, m, S.SDMD_F32)
    try:
        for t in range(m + 3):
            S.sdmd_push(h, torch.from_numpy(ps.snapshot(t)).to(cuda_device))
        G = _gram(h, m, cuda_device, False)
        ev = np.sort(np.linalg.eigvalsh(G[:-1, :-1]))[::-1]
        for r in range(4, m):
            rout = np.zeros(1, dtype=np.int32)
            S.sdmd_modes(h, r, None, None, rout)
            sig = np.zeros(r)
            S.sdmd_svd(h, r, sig, None)
            torch.cuda.synchronize()
            assert int(rout[0]) == r
            assert np.abs(sig ** 2 - ev[:r]).max() <= 1e-9 * ev[0], r
            assert S.sdmd_status(h) == S.SDMD_OK
    finally:
        S.sdmd_destroy(h)


def test_rank_fp32_matches_oracle_on_same_gram(cuda_device):
    # FP32 data from a 3-dimensional subspace: G carries FP32 accumulation
    # rounding, which the rank rule (FP64 floor) does not remove; the kept
    # rank and spectrum equal the oracle's on the same G.
    rng = np.random.default_rng(3)
    n, m = 2000, 12
    B = rng.standard_normal((n, 3))
    frames = [(B @ rng.standard_normal(3)).astype(np.float32) for _ in range(m)]
    h = S.sdmd_create(n, m, S.SDMD_F32)
    so = oracle.StreamOracle(n, m, "f32")
    try:
        _stream(h, so, frames, cuda_device)
        rk, lam, sig, V, P = _modes(h, n, 3, cuda_device, m)
        G = _gram(h, m, cuda_device, False)
        _compare_same_input(G, rk, lam, sig, V, 3)
        assert rk == 3
    finally:
        S.sdmd_destroy(h)


def test_max_window_256(cuda_device):
    rng = np.random.default_rng(4)
    n, m, r = 3000, 256, 12
    h = S.sdmd_create(n, m, S.SDMD_U8)
    so = oracle.StreamOracle(n, m, "u8")
    try:
        base = rng.integers(0, 200, n)
        frames = [np.clip(base + rng.integers(-30, 31, n), 0, 255).astype(np.uint8) for _ in range(m + 3)]
        _stream(h, so, frames, cuda_device)
        rk, lam, sig, V, P = _modes(h, n, r, cuda_device, m)
        ref = so.modes(r)
        assert rk == ref.r
        err, _ = match_eigs(lam[:rk], ref.lam)
        assert err <= EIG_TOL, err
    finally:
        S.sdmd_destroy(h)


def test_full_size_hd_video_modes(cuda_device):
    # Benchmark launch configuration: n = 1920*1080*3 uint8, m = 100, r = 10.
    vs = synth.VideoStream(seed=synth.config_seed(2))
    n, m, r, T = vs.n, 100, 10, 103
    h = S.sdmd_create(n, m, S.SDMD_U8)
    frames = []
    try:
        for t in range(T):
            f = vs.frame(t)
            frames.append(f)
            S.sdmd_push(h, torch.from_numpy(f).to(cuda_device))
        frames = frames[-m:]
        rk, lam, sig, V, P = _modes(h, n, r, cuda_device, m)
        Gref = oracle.gram_u8_cols(frames).astype(np.float64)     # exact
        G = _gram(h, m, cuda_device, True)
        assert np.array_equal(G, Gref)
        ref = oracle.dmd_from_gram(Gref[:-1, :-1], Gref[:-1, 1:], r)
        assert rk == ref.r
        err, perm = match_eigs(lam[:rk], ref.lam)
        assert err <= EIG_TOL, err
        # sampled rows of Phi, computed one by one by the oracle
        rows = np.random.default_rng(1).integers(0, n, 64)
        Xp_rows = np.stack([f[rows] for f in frames[1:]], axis=1).astype(np.float64)
        Pref = Xp_rows @ ref.M[:, perm]
        got = P[rows, :rk]
        scale = np.abs(Pref).max(axis=0)
        # fix each column's phase on the sampled rows (columns match up to a unit factor)
        for k in range(rk):
            i = int(np.argmax(np.abs(Pref[:, k])))
            got[:, k] *= (Pref[i, k] / got[i, k]) / abs(Pref[i, k] / got[i, k])
        assert (np.abs(got - Pref).max(axis=0) <= 1e-4 * scale).all()
    finally:
        S.sdmd_destroy(h)


@pytest.mark.parametrize("n,m,r", [(72 * 128 * 3, 20, 8), (1000, 12, 5), (4096 + 77, 40, 17), (128 * 40 + 3, 120, 3),
                                   (5000, 150, 9), (3000, 256, 12)])
def test_phi_tensor_core_matches_cuda_core_and_oracle(cuda_device, n, m, r):
    # uint8 windows: Phi on tcgen05 (fp16 pixels exact, M in three fp16
    # terms, FP32 accumulation) against the FP32 CUDA-core kernel and the
    # FP64 oracle product X' M with the same M; the shapes cover every
    # K padding / chunking configuration of the kernel.
    rng = np.random.default_rng(n + m)
    base = rng.integers(0, 200, n)
    frames = [np.clip(base + rng.integers(-40, 41, n), 0, 255).astype(np.uint8) for _ in range(m + 2)]
    h = S.sdmd_create(n, m, S.SDMD_U8)
    try:
        for f in frames:
            S.sdmd_push(h, torch.from_numpy(f).to(cuda_device))
        outs = {}
        for tensor in (1, 2, 0):                # tensor cores (modes per pass fitted to r, 16 per pass), CUDA cores
            S.sdmd_set_option(h, S.SDMD_OPT_PHI_TENSOR, tensor)
            phi = torch.zeros(r, n, 2, dtype=torch.float32, device=cuda_device)
            lam = np.zeros(2 * r)
            S.sdmd_modes(h, r, phi, lam)
            torch.cuda.synchronize()
            P = phi.cpu().numpy()
            outs[tensor] = P[..., 0] + 1j * P[..., 1]
        assert S.sdmd_status(h) == S.SDMD_OK
        assert np.array_equal(outs[1], outs[2])     # both tensor-core pass shapes: same arithmetic, same bits
        scale = np.abs(outs[0]).max(axis=1, keepdims=True) + 1e-30
        assert (np.abs(outs[1] - outs[0]) <= 2e-5 * scale).all()
        # against the oracle product with the oracle's M on the same window
        W = np.stack(frames[-m:], axis=1)
        ref = oracle.exact_dmd(W, r)
        lam_c = lam[0::2] + 1j * lam[1::2]
        err, perm = match_eigs(lam_c[:ref.r], ref.lam)
        Pn = normalize_cols(outs[1][:ref.r].T)
        Rn = normalize_cols(ref.Phi[:, perm])
        assert rel_fro(Pn, Rn) <= 1e-4
    finally:
        S.sdmd_destroy(h)
