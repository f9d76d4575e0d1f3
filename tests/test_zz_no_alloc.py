"""sdmd_gram_row_static, the Gram-row entry point that allocates no device
memory, checked through the C ABI against the regular handle path
(sdmd_push + sdmd_gram) on the same snapshots.

It serves callers that cannot call cudaMalloc (device memory owned by another
allocator or runtime, loops that must not take cudaMalloc's synchronisation,
plugins whose host forbids allocation); its output must be the same Gram row.
Kept in a file that pytest collects last.
"""
import numpy as np
import pytest
import torch

from paper_1612_07875_gb300 import sdmd as S

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5


def _snapshots(kind, c, n, ld, dev, seed):
    g = torch.Generator(device="cpu").manual_seed(seed)
    if kind == "u8":
        X = torch.randint(0, 256, (c, ld), dtype=torch.uint8, generator=g)
    else:
        X = torch.randn(c, ld, dtype=torch.float32, generator=g)
    return X.to(dev)      # columns n..ld-1 hold data the kernel must not read


def _reference_gram(kind, X, n, dev):
    c = X.shape[0]
    h = S.sdmd_create(n, c, S.SDMD_U8 if kind == "u8" else S.SDMD_F32)
    try:
        for j in range(c):
            S.sdmd_push(h, X[j, :n].contiguous())
        G = torch.empty(c, c, dtype=torch.int64 if kind == "u8" else torch.float64, device=dev)
        S.sdmd_gram(h, G)
        torch.cuda.synchronize()
        return G.cpu().numpy()
    finally:
        S.sdmd_destroy(h)


def _check(kind, got, ref, diag_i, diag_j):
    if kind == "u8":
        assert np.array_equal(got, ref)
    else:
        scale = np.sqrt(np.abs(diag_i * diag_j))
        assert (np.abs(got - ref) <= F32_TOL * scale).all()


@pytest.mark.parametrize("kind", ["u8", "f32"])
def test_static_row_matches_push_row_on_two_calls_in_a_row(cuda_device, kind):
    n, c = 1_000_003, 37               # ragged: n * sizeof(elem) is not a multiple of 16
    ld = (n + 15) // 16 * 16
    X = _snapshots(kind, c, n, ld, cuda_device, seed=11)
    G = _reference_gram(kind, X, n, cuda_device)
    d = np.diag(G).astype(np.float64)
    out_t = torch.int64 if kind == "u8" else torch.float64
    dt = S.SDMD_U8 if kind == "u8" else S.SDMD_F32

    # call 1: every snapshot against the newest one
    g1 = torch.full((c,), -7, dtype=out_t, device=cuda_device)
    S.sdmd_gram_row_static(dt, X, ld, c, X[c - 1], n, g1)
    # call 2, straight after: fewer snapshots against another y
    c2 = 5
    g2 = torch.full((c2,), -7, dtype=out_t, device=cuda_device)
    S.sdmd_gram_row_static(dt, X, ld, c2, X[2], n, g2)
    torch.cuda.synchronize()

    _check(kind, g1.cpu().numpy(), G[c - 1, :], d, d[c - 1])
    _check(kind, g2.cpu().numpy(), G[:c2, 2], d[:c2], d[2])


@pytest.mark.parametrize("kind", ["u8", "f32"])
@pytest.mark.parametrize("n", [1, 3, 17])
def test_static_row_tail_only(cuda_device, kind, n):
    # fewer than 16 bytes past the last whole vector: one CTA whose lane 0
    # adds the scalar tail (for n = 1 and 3 with uint8, all of the row)
    c, ld = 9, (n + 15) // 16 * 16
    X = _snapshots(kind, c, n, ld, cuda_device, seed=21 + n)
    G = _reference_gram(kind, X, n, cuda_device)
    d = np.diag(G).astype(np.float64)
    out_t = torch.int64 if kind == "u8" else torch.float64
    dt = S.SDMD_U8 if kind == "u8" else S.SDMD_F32
    for rep in range(2):
        g = torch.full((c,), -7, dtype=out_t, device=cuda_device)
        S.sdmd_gram_row_static(dt, X, ld, c, X[rep], n, g)
        torch.cuda.synchronize()
        _check(kind, g.cpu().numpy(), G[rep, :], d, d[rep])


@pytest.mark.parametrize("kind", ["u8", "f32"])
def test_static_row_max_window_large_n(cuda_device, kind):
    # c = SDMD_GRAM_ROW_STATIC_MAX_C fills every row of the partials array;
    # n = 2^22 splits into as many CTAs as the launch allows (two per SM)
    c, n = S.SDMD_GRAM_ROW_STATIC_MAX_C, 1 << 22
    g = torch.Generator(device=cuda_device).manual_seed(31)
    if kind == "u8":
        X = torch.randint(0, 256, (c, n), dtype=torch.uint8, device=cuda_device, generator=g)
    else:
        X = torch.randn(c, n, dtype=torch.float32, device=cuda_device, generator=g)
    G = _reference_gram(kind, X, n, cuda_device)
    d = np.diag(G).astype(np.float64)
    out_t = torch.int64 if kind == "u8" else torch.float64
    dt = S.SDMD_U8 if kind == "u8" else S.SDMD_F32
    for y in (c - 1, 0):
        out = torch.full((c,), -7, dtype=out_t, device=cuda_device)
        S.sdmd_gram_row_static(dt, X, n, c, X[y], n, out)
        torch.cuda.synchronize()
        _check(kind, out.cpu().numpy(), G[y, :], d, d[y])


def test_static_row_rejects_oversized_window(cuda_device):
    n = 1024
    X = torch.zeros(2, n, dtype=torch.float32, device=cuda_device)
    g = torch.zeros(S.SDMD_GRAM_ROW_STATIC_MAX_C + 1, dtype=torch.float64, device=cuda_device)
    with pytest.raises(S.SdmdError) as ei:
        S.sdmd_gram_row_static(S.SDMD_F32, X, n, S.SDMD_GRAM_ROW_STATIC_MAX_C + 1, X[0], n, g)
    assert ei.value.code == S.SDMD_ERR_ARG
    assert "not in [1, %d]" % S.SDMD_GRAM_ROW_STATIC_MAX_C in S.sdmd_last_error()
