"""GPU parity of the Fourier-sparse streaming Gram (Sec. 3.5) and of the dense
complex64 path against the CPU oracle.

Tolerance for these complex64 paths: every entry within 1e-5 of the
Cauchy-Schwarz scale sqrt(G_ii G_jj) and relative Frobenius error <= 1e-5
(FP32 products, FP64 sums).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1612_07875_gb300 import sdmd as S
from paper_1612_07875_gb300 import synth

from helpers import rel_fro

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _read(h, c, dev):
    G = torch.empty(c, c, 2, dtype=torch.float64, device=dev)
    S.sdmd_gram(h, G)
    torch.cuda.synchronize()
    g = G.cpu().numpy()
    return g[..., 0] + 1j * g[..., 1]


def _check(G, ref):
    assert rel_fro(G, ref) <= TOL
    d = np.sqrt(np.abs(np.outer(np.diag(ref).real, np.diag(ref).real)))
    assert (np.abs(G - ref) <= TOL * d + 1e-300).all()
    assert np.allclose(G, G.conj().T, rtol=0, atol=0)


@pytest.mark.parametrize("device_input", [True, False])
def test_sparse_gram_every_step_matches_oracle(cuda_device, device_input):
    fs = synth.FourierSparseStream(side=128, nnz=164, churn=0.1, seed=31)
    m, T = 12, 20
    h = S.sdmd_create_sparse(fs.N, m, 200)
    so = oracle.StreamOracle(fs.N, m, "sparse")
    try:
        for t in range(T):
            idx, val = fs.snapshot(t)
            if device_input:
                S.sdmd_push_sparse(h, idx.size, torch.from_numpy(idx).to(cuda_device),
                                   torch.from_numpy(val.view(np.float32)).to(cuda_device))
            else:
                S.sdmd_push_sparse(h, idx.size, idx, val)
            so.push((idx, val))
            c = min(t + 1, m)
            _check(_read(h, c, cuda_device), so.gram())
        assert S.sdmd_status(h) == S.SDMD_OK
    finally:
        S.sdmd_destroy(h)


def test_parseval_sparse_equals_dense_physical_on_gpu(cuda_device):
    # Same stream twice: sparse orthonormal-FFT coefficients, and the dense
    # physical fields (ifft2, norm="ortho") through the dense complex64 path.
    fs = synth.FourierSparseStream(side=64, nnz=41, churn=0.1, seed=32)
    m, T = 8, 11
    hs = S.sdmd_create_sparse(fs.N, m, 64)
    hd = S.sdmd_create(fs.N, m, S.SDMD_C64)
    try:
        for t in range(T):
            idx, val = fs.snapshot(t)
            S.sdmd_push_sparse(hs, idx.size, idx, val)
            phys = fs.physical(t).astype(np.complex64)
            S.sdmd_push(hd, torch.from_numpy(phys.view(np.float32)).to(cuda_device))
        Gs = _read(hs, m, cuda_device)
        Gd = _read(hd, m, cuda_device)
        assert rel_fro(Gs, Gd) <= 1e-5
        # and the dense path matches its own oracle (physical fields, FP64)
        phys = np.stack([fs.physical(t).astype(np.complex64) for t in range(T - m, T)], axis=1)
        _check(Gd, oracle.gram_dense(phys))
    finally:
        S.sdmd_destroy(hs)
        S.sdmd_destroy(hd)


def test_dense_complex_gram_ragged_sizes(cuda_device):
    rng = np.random.default_rng(5)
    for n in (1, 7, 1023, 70001):
        m = 4
        h = S.sdmd_create(n, m, S.SDMD_C64)
        so = oracle.StreamOracle(n, m, "f32")
        try:
            for t in range(6):
                x = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
                S.sdmd_push(h, torch.from_numpy(x.view(np.float32)).to(cuda_device))
                so.push(x)
            _check(_read(h, m, cuda_device), so.gram())
        finally:
            S.sdmd_destroy(h)


def test_sparse_edge_cases(cuda_device):
    n, m = 1000, 3
    h = S.sdmd_create_sparse(n, m, 16)
    try:
        e_idx = np.zeros(0, np.int32)
        e_val = np.zeros(0, np.complex64)
        S.sdmd_push_sparse(h, 0, e_idx, e_val)                       # empty snapshot
        idx = np.array([0, 5, 999], np.int32)
        val = np.array([1 + 2j, -3j, 4], np.complex64)
        S.sdmd_push_sparse(h, 3, idx, val)
        S.sdmd_push_sparse(h, 2, np.array([5, 6], np.int32), np.array([2, 1j], np.complex64))
        G = _read(h, 3, cuda_device)
        assert G[0, 0] == 0 and G[0, 1] == 0
        assert abs(G[1, 1] - (5 + 9 + 16)) < 1e-12
        assert abs(G[1, 2] - np.conj(-3j) * 2) < 1e-12               # only index 5 is shared
        # host index checks
        for bad in (np.array([3, 3], np.int32), np.array([4, 2], np.int32), np.array([1, 1000], np.int32)):
            with pytest.raises(S.SdmdError) as ei:
                S.sdmd_push_sparse(h, 2, bad, np.ones(2, np.complex64))
            assert ei.value.code == S.SDMD_ERR_ARG
        with pytest.raises(S.SdmdError) as ei:
            S.sdmd_push_sparse(h, 17, np.arange(17, dtype=np.int32), np.ones(17, np.complex64))
        assert ei.value.code == S.SDMD_ERR_ARG
        # device index out of range: skipped by the kernel, reported by sdmd_status
        bad_dev = torch.tensor([7, 5000], dtype=torch.int32, device=cuda_device)
        S.sdmd_push_sparse(h, 2, bad_dev, torch.ones(4, dtype=torch.float32, device=cuda_device))
        assert S.sdmd_status(h) == S.SDMD_ERR_ARG
        assert S.sdmd_status(h) == S.SDMD_OK
        # modes of a sparse window stay in coefficient space (sdmd_fourier_modes):
        # a dense Phi is refused, the small-matrix part runs
        with pytest.raises(S.SdmdError) as ei:
            S.sdmd_modes(h, 1, torch.zeros(1, n, 2, device=cuda_device), None)
        assert ei.value.code == S.SDMD_ERR_UNSUPPORTED
        S.sdmd_modes(h, 1, None, None)
        assert S.sdmd_status(h) == S.SDMD_OK
    finally:
        S.sdmd_destroy(h)


def test_full_size_fourier_sparse_config(cuda_device):
    # 1024 x 1024 periodic field, ~1% (10,486) coefficients, window 64.
    fs = synth.FourierSparseStream(seed=synth.config_seed(3))
    m, T = 64, 68
    h = S.sdmd_create_sparse(fs.N, m, fs.nnz + 16)
    snaps = {}
    try:
        for t in range(T):
            idx, val = fs.snapshot(t)
            if t >= T - m:
                snaps[t] = (idx, val)
            S.sdmd_push_sparse(h, idx.size, torch.from_numpy(idx).to(cuda_device),
                               torch.from_numpy(val.view(np.float32)).to(cuda_device))
        G = _read(h, m, cuda_device)
        ts = sorted(snaps)
        rng = np.random.default_rng(2)
        pairs = [(m - 1, j) for j in range(0, m, 5)] + [tuple(rng.integers(0, m, 2)) for _ in range(8)]
        for i, j in pairs:
            ref = oracle.sparse_inner(*snaps[ts[i]], *snaps[ts[j]])
            scale = np.sqrt(abs(G[i, i] * G[j, j]))
            assert abs(G[i, j] - ref) <= TOL * scale, (i, j)
        assert S.sdmd_status(h) == S.SDMD_OK
    finally:
        S.sdmd_destroy(h)
