"""BF16x3 split-precision Gram of FP32 windows on the tensor cores
(SDMD_OPT_F32_BF16X3): sdmd_rebuild and the multi-column catch-up
sdmd_push_batch, against the FP64 oracle Gram of the same FP32 snapshots.
Catch-ups of at most 16 snapshots (and rebuilds of windows of at most 16)
take the CUDA-core pass with FP32 products under the same option and bound.

Bound (from the arithmetic: dropped split products and remainders below
2^-22 |x y|, about four full-magnitude FP32 roundings of the accumulator per
64 positions, compensated sums after that):
    |G_ij - <x_i, x_j>| <= 1e-6 * sum_p |x_ip| |x_jp|      for every entry,
and the relative Frobenius error of G <= 1e-6. Shapes cover ragged tails
(n not a multiple of 64 or 1024), several chunks per CTA, windows of 1..256
snapshots (so one to seven launches of up to 64 targets x 128 rows), and the
window ramp-up. Repeated runs are bitwise identical (static chunk order).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1612_07875_gb300 import sdmd as S

from helpers import rel_fro

pytestmark = pytest.mark.gpu

TOL = 1e-6


def _frames(n, count, seed, kind="normal"):
    rng = np.random.default_rng(seed)
    if kind == "normal":
        return rng.standard_normal((count, n)).astype(np.float32)
    # positive data with a common offset: every product has the same sign,
    # so no cancellation hides a systematic error
    return (3.0 + rng.random((count, n))).astype(np.float32)


def _check(G, W):
    """G (c x c) against the window W (c x n, float32), oldest first."""
    Wd = W.astype(np.float64)
    ref = Wd @ Wd.T
    bound = np.abs(Wd) @ np.abs(Wd).T
    err = np.abs(G - ref)
    worst = float((err / bound).max())
    assert worst <= TOL, worst
    assert rel_fro(G, ref) <= TOL
    assert np.array_equal(G, G.T)
    return worst


def _gram(h, c, dev):
    G = torch.empty(c, c, dtype=torch.float64, device=dev)
    S.sdmd_gram(h, G)
    torch.cuda.synchronize()
    return G.cpu().numpy()


@pytest.mark.parametrize("n,m,data", [(5, 3, "normal"), (1000, 8, "normal"), (64 * 1024 * 3 + 17, 33, "normal"),
                                      ((1 << 20) + 63, 100, "normal"), ((1 << 18) + 1, 100, "offset"),
                                      (4099, 256, "normal"), (2 * 152 * 1024 + 1000, 130, "offset")])
def test_rebuild_bf16x3_within_bound(cuda_device, n, m, data):
    T = m + 3
    X = _frames(n, T, seed=n + m, kind=data)
    h = S.sdmd_create(n, m, S.SDMD_F32)
    try:
        for t in range(T):
            S.sdmd_push(h, torch.from_numpy(X[t]).to(cuda_device))
        S.sdmd_set_option(h, S.SDMD_OPT_F32_BF16X3, 1)
        S.sdmd_rebuild(h)
        G1 = _gram(h, m, cuda_device)
        worst = _check(G1, X[T - m:])
        S.sdmd_rebuild(h)
        G2 = _gram(h, m, cuda_device)
        assert np.array_equal(G1, G2)              # same chunk order every run
        assert S.sdmd_status(h) == S.SDMD_OK
        print("n=%d m=%d %s: worst |dG|/sum|x y| = %.2e" % (n, m, data, worst))
    finally:
        S.sdmd_destroy(h)


@pytest.mark.parametrize("n,m,pre,k", [(70001, 16, 0, 5), (70001, 16, 20, 2), ((1 << 19) + 5, 100, 100, 8),
                                       ((1 << 19) + 5, 100, 37, 64), ((1 << 18) + 3, 256, 256, 65),
                                       ((1 << 18) + 3, 256, 10, 200), (3000, 128, 128, 128),
                                       # k <= 16: one CUDA-core pass with FP32 products
                                       (70001, 256, 256, 16), ((1 << 18) + 3, 200, 150, 9), (100, 40, 3, 16),
                                       # one row per thread up to c = 128, two above (and the k <= 4 instance)
                                       (70001, 128, 128, 4), (70001, 129, 129, 7), ((1 << 18) + 3, 180, 177, 3)])
def test_push_batch_bf16x3_within_bound(cuda_device, n, m, pre, k):
    X = _frames(n, pre + k, seed=3 * n + k)
    h = S.sdmd_create(n, m, S.SDMD_F32)
    so = oracle.StreamOracle(n, m, "f32")
    try:
        S.sdmd_set_option(h, S.SDMD_OPT_F32_BF16X3, 1)
        for t in range(pre):
            S.sdmd_push(h, torch.from_numpy(X[t]).to(cuda_device))
            so.push(X[t])
        S.sdmd_push_batch(h, k, torch.from_numpy(X[pre:]).to(cuda_device), n)
        for t in range(pre, pre + k):
            so.push(X[t])
        c = min(pre + k, m)
        G = _gram(h, c, cuda_device)
        _check(G, X[pre + k - c:pre + k])
        ref = so.gram()
        assert rel_fro(G, ref) <= TOL
        assert S.sdmd_status(h) == S.SDMD_OK
        # streaming continues from the caught-up window with FP32 rows
        x = _frames(n, 1, seed=7)[0]
        S.sdmd_push(h, torch.from_numpy(x).to(cuda_device))
        so.push(x)
        assert rel_fro(_gram(h, min(c + 1, m), cuda_device), so.gram()) <= TOL
    finally:
        S.sdmd_destroy(h)


@pytest.mark.parametrize("n,m,data", [(70001, 40, "normal"), ((1 << 18) + 1, 100, "offset"), (70001, 16, "normal")])
def test_rebuild_two_term_split_within_its_bound(cuda_device, n, m, data):
    # two bf16 terms, three products: dropped b1 c1 and remainders about
    # 2^-16 |x y| per product; bound used: 3e-5 sum_p |x_ip x_jp|
    X = _frames(n, m, seed=11 * n + m, kind=data)
    h = S.sdmd_create(n, m, S.SDMD_F32)
    try:
        for t in range(m):
            S.sdmd_push(h, torch.from_numpy(X[t]).to(cuda_device))
        S.sdmd_set_option(h, S.SDMD_OPT_F32_BF16X3, 2)
        S.sdmd_rebuild(h)
        G = _gram(h, m, cuda_device)
        Wd = X.astype(np.float64)
        ref = Wd @ Wd.T
        worst = float((np.abs(G - ref) / (np.abs(Wd) @ np.abs(Wd).T)).max())
        print("two-term n=%d m=%d %s: worst %.2e, rel Frobenius %.2e" % (n, m, data, worst, rel_fro(G, ref)))
        assert worst <= 3e-5
        assert np.array_equal(G, G.T)
        with pytest.raises(S.SdmdError):
            S.sdmd_set_option(h, S.SDMD_OPT_F32_BF16X3, 3)
    finally:
        S.sdmd_destroy(h)


def test_fp64_reference_rows(cuda_device):
    # FP64 products (exact for FP32 inputs) and FP64 sums: the oracle's Gram
    # up to FP64 summation order; batched rows equal single pushes bit for bit
    n, m = (1 << 17) + 9, 12
    X = _frames(n, m + 4, seed=2)
    ha = S.sdmd_create(n, m, S.SDMD_F32)
    hb = S.sdmd_create(n, m, S.SDMD_F32)
    hc = S.sdmd_create(777, 5, S.SDMD_U8)
    so = oracle.StreamOracle(n, m, "f32")
    try:
        for h in (ha, hb):
            S.sdmd_set_option(h, S.SDMD_OPT_F32_FP64, 1)
        u8 = np.random.default_rng(3).integers(0, 256, (m + 4, 777), dtype=np.uint8)
        for t in range(m + 4):
            x = torch.from_numpy(X[t]).to(cuda_device)
            S.sdmd_push(ha, x)
            S.sdmd_push_many([hb, hc], [x, torch.from_numpy(u8[t]).to(cuda_device)])
            so.push(X[t])
        Ga, Gb = _gram(ha, m, cuda_device), _gram(hb, m, cuda_device)
        assert np.array_equal(Ga, Gb)
        ref = so.gram()
        assert rel_fro(Ga, ref) <= 1e-14
        assert np.abs(Ga - ref).max() <= 1e-13 * np.abs(ref).max()
    finally:
        for h in (ha, hb, hc):
            S.sdmd_destroy(h)


def test_bf16x3_option_off_keeps_fp32_rows(cuda_device):
    n, m, k = 20000, 12, 6
    X = _frames(n, m + k, seed=5)
    ha = S.sdmd_create(n, m, S.SDMD_F32)
    hb = S.sdmd_create(n, m, S.SDMD_F32)
    try:
        for t in range(m):
            for h in (ha, hb):
                S.sdmd_push(h, torch.from_numpy(X[t]).to(cuda_device))
        S.sdmd_set_option(ha, S.SDMD_OPT_F32_BF16X3, 0)
        S.sdmd_push_batch(ha, k, X[m:], n)                 # host source, option off: k FP32 pushes
        for t in range(m, m + k):
            S.sdmd_push(hb, torch.from_numpy(X[t]).to(cuda_device))
        assert np.array_equal(_gram(ha, m, cuda_device), _gram(hb, m, cuda_device))
    finally:
        S.sdmd_destroy(ha)
        S.sdmd_destroy(hb)
