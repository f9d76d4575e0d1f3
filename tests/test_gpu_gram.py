"""GPU parity of the streaming Gram update (sdmd_push + sdmd_gram) against the
CPU oracle, which recomputes G = W^H W from the window at every step.

uint8: bit-exact every step. float32: relative Frobenius error <= 1e-5 and
every entry within 1e-5 * sqrt(G_ii G_jj) (the Cauchy-Schwarz scale of that
entry), against the FP64 oracle on the same float32 inputs.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1612_07875_gb300 import sdmd as S
from paper_1612_07875_gb300 import synth

from helpers import rel_fro

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5


def _gen(kind, n, seed):
    rng = np.random.default_rng(seed)
    if kind == "u8":
        return lambda t: rng.integers(0, 256, n, dtype=np.uint8)
    return lambda t: rng.standard_normal(n).astype(np.float32)


def _check_gram(G, ref, kind):
    if kind == "u8":
        assert G.dtype == np.int64
        assert np.array_equal(G, ref)
    else:
        assert rel_fro(G, ref) <= F32_TOL
        d = np.sqrt(np.abs(np.outer(np.diag(ref), np.diag(ref))))
        assert (np.abs(G - ref) <= F32_TOL * d + 1e-30).all()


def _read_gram(h, c, kind, dev):
    G = torch.empty(c, c, dtype=torch.int64 if kind == "u8" else torch.float64, device=dev)
    S.sdmd_gram(h, G)
    torch.cuda.synchronize()
    return G.cpu().numpy()


@pytest.mark.parametrize("kind", ["u8", "f32"])
@pytest.mark.parametrize("n,m", [(1, 2), (3, 5), (127, 3), (4097, 16), (65549, 7),
                                 ((1 << 20) + 7, 5), (513, 256)])
def test_gram_every_step_matches_oracle(cuda_device, kind, n, m):
    T = m + 6 if m < 64 else m + 2
    gen = _gen(kind, n, seed=n * 31 + m)
    dt = S.SDMD_U8 if kind == "u8" else S.SDMD_F32
    h = S.sdmd_create(n, m, dt)
    so = oracle.StreamOracle(n, m, kind)
    try:
        for t in range(T):
            x = gen(t)
            S.sdmd_push(h, torch.from_numpy(x).to(cuda_device))
            so.push(x)
            c = min(t + 1, m)
            if m <= 16 or t >= T - 2:
                _check_gram(_read_gram(h, c, kind, cuda_device), so.gram(), kind)
        assert S.sdmd_count(h) == T
    finally:
        S.sdmd_destroy(h)


@pytest.mark.parametrize("kind", ["u8", "f32"])
def test_streaming_equals_recomputed_bitwise(cuda_device, kind):
    # Eq. 12: the streamed G equals a G built from scratch on the final window;
    # the Gram-row schedule depends only on n, so even FP32 is bit-identical.
    n, m, T = 50021, 9, 31
    gen = _gen(kind, n, seed=5)
    xs = [gen(t) for t in range(T)]
    dt = S.SDMD_U8 if kind == "u8" else S.SDMD_F32
    a = S.sdmd_create(n, m, dt)
    b = S.sdmd_create(n, m, dt)
    try:
        for x in xs:
            S.sdmd_push(a, torch.from_numpy(x).to(cuda_device))
        for x in xs[-m:]:
            S.sdmd_push(b, torch.from_numpy(x).to(cuda_device))
        Ga = _read_gram(a, m, kind, cuda_device)
        Gb = _read_gram(b, m, kind, cuda_device)
        assert np.array_equal(Ga.view(np.int64), Gb.view(np.int64))
    finally:
        S.sdmd_destroy(a)
        S.sdmd_destroy(b)


@pytest.mark.parametrize("kind", ["f32", "u8"])
def test_host_pageable_pinned_and_device_inputs_agree(cuda_device, kind):
    # device rows with 16-byte aligned addresses go through the library's copy
    # kernel (n = 30011: the last 12 (f32) or 11 (u8) bytes by its tail path),
    # a device view one element off and host sources through cudaMemcpyAsync:
    # the same G bit for bit
    n, m = 30011, 4
    gen = _gen(kind, n, seed=9)
    xs = [gen(t) for t in range(6)]
    dt = S.SDMD_U8 if kind == "u8" else S.SDMD_F32
    Gs = []
    for mode in ("device", "device_offset", "pageable", "pinned"):
        h = S.sdmd_create(n, m, dt)
        keep = []      # sources must outlive their asynchronous copies
        try:
            for x in xs:
                xt = torch.from_numpy(x)
                if mode == "device":
                    S.sdmd_push(h, xt.to(cuda_device))
                elif mode == "device_offset":
                    buf = torch.empty(n + 1, dtype=xt.dtype, device=cuda_device)
                    buf[1:].copy_(xt)
                    keep.append(buf)
                    S.sdmd_push(h, buf[1:])
                elif mode == "pageable":
                    S.sdmd_push(h, x)
                else:
                    keep.append(xt.pin_memory())
                    S.sdmd_push(h, keep[-1])
            torch.cuda.synchronize()
            out = np.zeros((m, m), dtype=np.int64 if kind == "u8" else np.float64)
            S.sdmd_gram(h, out)           # pageable host output: call waits
            Gs.append(out)
        finally:
            S.sdmd_destroy(h)
    for G in Gs[1:]:
        assert np.array_equal(Gs[0], G)


def test_u8_extreme_values_exact_beyond_int32(cuda_device):
    n, m = 3 * 1920 * 1080, 3
    frames = [np.full(n, 255, np.uint8), np.full(n, 254, np.uint8), np.zeros(n, np.uint8)]
    frames[2][::2] = 255
    h = S.sdmd_create(n, m, S.SDMD_U8)
    try:
        for f in frames:
            S.sdmd_push(h, torch.from_numpy(f).to(cuda_device))
        G = _read_gram(h, m, "u8", cuda_device)
        assert G[0, 0] == 255 * 255 * n and G[0, 0] > 2 ** 31
        assert G[0, 1] == 255 * 254 * n
        assert G[2, 2] == 255 * 255 * (n // 2)
        assert np.array_equal(G, oracle.gram_u8(np.stack(frames, axis=1)))
    finally:
        S.sdmd_destroy(h)


def test_full_size_hd_video_sampled_entries(cuda_device):
    # The benchmark's launch configuration: n = 1920*1080*3 uint8, m = 100,
    # window full and wrapped. Sampled entries checked one by one (exact).
    vs = synth.VideoStream(seed=synth.config_seed(2))
    m, T = 100, 104
    h = S.sdmd_create(vs.n, m, S.SDMD_U8)
    frames = {}
    try:
        for t in range(T):
            f = vs.frame(t)
            if t >= T - m:
                frames[t] = f
            S.sdmd_push(h, torch.from_numpy(f).to(cuda_device))
        G = _read_gram(h, m, "u8", cuda_device)
        ts = sorted(frames)
        rng = np.random.default_rng(0)
        pairs = [(m - 1, j) for j in range(0, m, 7)] + [tuple(rng.integers(0, m, 2)) for _ in range(12)]
        for i, j in pairs:
            assert G[i, j] == oracle.dot_u8(frames[ts[i]], frames[ts[j]]), (i, j)
        assert np.array_equal(G, G.T)
        # the tensor-core rebuild of the same full-size window: equal to the streamed G
        S.sdmd_rebuild(h)
        assert np.array_equal(_read_gram(h, m, "u8", cuda_device), G)
        assert S.sdmd_status(h) == S.SDMD_OK
    finally:
        S.sdmd_destroy(h)


def test_error_paths(cuda_device):
    h = S.sdmd_create(1000, 4, S.SDMD_F32)
    try:
        x = torch.zeros(1000, device=cuda_device)
        S.sdmd_push(h, x)
        S.sdmd_push(h, x)
        with pytest.raises(S.SdmdError) as ei:
            S.sdmd_modes(h, 1, None, None)
        assert ei.value.code == S.SDMD_ERR_NOT_READY
        S.sdmd_push(h, x + 1)
        with pytest.raises(S.SdmdError) as ei:
            S.sdmd_modes(h, 4, None, None)           # r > m-1
        assert ei.value.code == S.SDMD_ERR_ARG
        host_phi = np.zeros(2 * 1000 * 2, np.float32)
        with pytest.raises(S.SdmdError) as ei:
            S.sdmd_modes(h, 2, host_phi, None)       # phi must be device memory
        assert ei.value.code == S.SDMD_ERR_ARG
        with pytest.raises(S.SdmdError) as ei:
            S.sdmd_svd(h, 2, None, None)             # no modes call yet
        assert ei.value.code == S.SDMD_ERR_NOT_READY
        with pytest.raises(S.SdmdError) as ei:
            S.sdmd_push(h, None)
        assert ei.value.code == S.SDMD_ERR_ARG
    finally:
        S.sdmd_destroy(h)


@pytest.mark.parametrize("kind", ["u8", "f32", "c64", "sparse"])
def test_full_window_rebuild_equals_streamed_gram_bitwise(cuda_device, kind):
    # Algorithm 1's first-step branch (G = X^T X from scratch) against the
    # streamed G: same per-entry reduction, so equal bit for bit.
    rng = np.random.default_rng(12)
    m, T = 9, 23
    if kind == "sparse":
        fs = synth.FourierSparseStream(side=64, nnz=41, churn=0.2, seed=33)
        h = S.sdmd_create_sparse(fs.N, m, 64)
    else:
        n = 40009
        dt = {"u8": S.SDMD_U8, "f32": S.SDMD_F32, "c64": S.SDMD_C64}[kind]
        h = S.sdmd_create(n, m, dt)
    try:
        for t in range(T):
            if kind == "sparse":
                idx, val = fs.snapshot(t)
                S.sdmd_push_sparse(h, idx.size, idx, val)
            elif kind == "u8":
                S.sdmd_push(h, torch.from_numpy(rng.integers(0, 256, n, dtype=np.uint8)).to(cuda_device))
            elif kind == "f32":
                S.sdmd_push(h, torch.from_numpy(rng.standard_normal(n).astype(np.float32)).to(cuda_device))
            else:
                x = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
                S.sdmd_push(h, torch.from_numpy(x.view(np.float32)).to(cuda_device))
        words = 2 if kind in ("c64", "sparse") else 1
        G1 = torch.empty(m, m, words, dtype=torch.int64, device=cuda_device)
        S.sdmd_gram(h, G1)
        S.sdmd_rebuild(h)
        G2 = torch.empty(m, m, words, dtype=torch.int64, device=cuda_device)
        S.sdmd_gram(h, G2)
        torch.cuda.synchronize()
        assert torch.equal(G1, G2)
        assert S.sdmd_status(h) == S.SDMD_OK
    finally:
        S.sdmd_destroy(h)


@pytest.mark.parametrize("n,m,pushes,pattern", [
    (40009, 9, 23, "random"),         # window full, ragged n
    (4096 * 3 + 17, 127, 130, "random"),   # the largest window on the tensor path
    (100003, 100, 40, "extreme"),     # ramp-up (40 of 100), pixels 0 / 255 only
    (1, 3, 5, "random"),              # a single position
    (5000, 128, 128, "random"),       # past one tile: groups of 64 targets with older blocks
    (70001, 256, 260, "random"),      # the largest window: 4 groups, 10 launches
    (9000, 200, 230, "extreme"),      # uneven groups (64, 64, 64, 8), pixels 0 / 255 only
])
def test_tensor_core_rebuild_exact(cuda_device, n, m, pushes, pattern):
    # Algorithm 1's first step on the tensor cores (centred fp16 pixels,
    # FP32 accumulators drained into int64): equal to the oracle's exact
    # int64 Gram and to the streamed G, and to the row-kernel rebuild.
    rng = np.random.default_rng(n + m)
    h = S.sdmd_create(n, m, S.SDMD_U8)
    so = oracle.StreamOracle(n, m, "u8")
    try:
        for _ in range(pushes):
            if pattern == "extreme":
                x = (rng.integers(0, 2, n, dtype=np.uint8) * 255).astype(np.uint8)
            else:
                x = rng.integers(0, 256, n, dtype=np.uint8)
            S.sdmd_push(h, torch.from_numpy(x).to(cuda_device))
            so.push(x)
        c = min(pushes, m)
        G0 = torch.empty(c, c, dtype=torch.int64, device=cuda_device)
        S.sdmd_gram(h, G0)
        out = {}
        for opt in (1, 0):
            S.sdmd_set_option(h, S.SDMD_OPT_REBUILD_TENSOR, opt)
            S.sdmd_rebuild(h)
            G = torch.empty(c, c, dtype=torch.int64, device=cuda_device)
            S.sdmd_gram(h, G)
            out[opt] = G
        torch.cuda.synchronize()
        ref = so.gram()
        assert np.array_equal(out[1].cpu().numpy(), ref)
        assert torch.equal(out[1], out[0]) and torch.equal(out[1], G0)
        assert S.sdmd_status(h) == S.SDMD_OK
    finally:
        S.sdmd_destroy(h)


@pytest.mark.parametrize("n,m,pre,k,dtype,device_src", [
    (40009, 9, 23, 4, "u8", True),          # wrapped window
    (4096 * 3 + 17, 100, 120, 8, "u8", False),   # host source
    (100003, 20, 5, 10, "u8", True),        # ramp-up: 5 resident, 10 new
    (5000, 16, 3, 16, "u8", True),          # k = m: every resident snapshot is new
    (6000, 127, 130, 127, "u8", True),      # the largest window in one tile
    (5000, 128, 130, 3, "u8", True),        # past one tile: 3 targets, older in blocks of 124
    (70001, 256, 256, 8, "u8", True),       # the largest window, the bench's catch-up size
    (9000, 200, 150, 100, "u8", False),     # ramp-up into a wrapped window: groups of 64 and 36
    (3001, 12, 15, 5, "f32", True),         # float: k ordinary pushes
])
def test_push_batch_equals_sequential_pushes(cuda_device, n, m, pre, k, dtype, device_src):
    # multi-column catch-up: k new rows/columns of G in one pass
    # over the window; the Gram must equal that of k single pushes (exactly
    # for uint8, bit for bit for the float fallback) and the oracle's.
    rng = np.random.default_rng(n + k)
    dt = S.SDMD_U8 if dtype == "u8" else S.SDMD_F32
    make = (lambda: rng.integers(0, 256, n, dtype=np.uint8)) if dtype == "u8" else \
        (lambda: rng.standard_normal(n).astype(np.float32))
    first = [make() for _ in range(pre)]
    batch = np.stack([make() for _ in range(k)])          # k x n, snapshot j in row j
    h1 = S.sdmd_create(n, m, dt)
    h2 = S.sdmd_create(n, m, dt)
    so = oracle.StreamOracle(n, m, dtype)
    try:
        for x in first:
            S.sdmd_push(h1, torch.from_numpy(x).to(cuda_device))
            S.sdmd_push(h2, torch.from_numpy(x).to(cuda_device))
            so.push(x)
        src = torch.from_numpy(batch).to(cuda_device) if device_src else batch
        S.sdmd_push_batch(h1, k, src, n)
        for j in range(k):
            S.sdmd_push(h2, torch.from_numpy(batch[j]).to(cuda_device))
            so.push(batch[j])
        c = min(pre + k, m)
        words = torch.int64 if dtype == "u8" else torch.float64
        G1 = torch.empty(c, c, dtype=words, device=cuda_device)
        G2 = torch.empty(c, c, dtype=words, device=cuda_device)
        S.sdmd_gram(h1, G1)
        S.sdmd_gram(h2, G2)
        torch.cuda.synchronize()
        assert torch.equal(G1, G2)
        if dtype == "u8":
            assert np.array_equal(G1.cpu().numpy(), so.gram())
        assert S.sdmd_status(h1) == S.SDMD_OK
    finally:
        S.sdmd_destroy(h1)
        S.sdmd_destroy(h2)


def test_push_batch_argument_errors(cuda_device):
    h = S.sdmd_create(100, 4, S.SDMD_U8)
    x = torch.zeros(5, 100, dtype=torch.uint8, device=cuda_device)
    try:
        for k, ld in ((0, 100), (5, 100), (2, 99)):
            with pytest.raises(S.SdmdError) as ei:
                S.sdmd_push_batch(h, k, x, ld)
            assert ei.value.code == S.SDMD_ERR_ARG
    finally:
        S.sdmd_destroy(h)
