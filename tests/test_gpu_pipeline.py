"""Pipelined streaming DMD (sdmd_step with frames in flight) against the
unpipelined path (sdmd_push + sdmd_modes) on the same frames: the pipeline
only reorders independent work across streams, so every frame's eigenvalues,
rank and modes must be identical bit for bit, including after the ring has
wrapped several times (which exercises the ring-slot hazard tracking)."""
import numpy as np
import pytest
import torch

from paper_1612_07875_gb300 import sdmd as S
from paper_1612_07875_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,depth,m,r", [("u8", 4, 12, 5), ("f32", 3, 12, 5), ("u8", 1, 12, 5), ("u8", 2, 12, 5),
                                            ("u8", 6, 12, 5), ("u8", 3, 130, 5), ("u8", 4, 40, 20),
                                            ("u8", 7, 250, 10), ("u8", 8, 250, 10)])
def test_pipelined_step_equals_serial(cuda_device, kind, depth, m, r):
    # uint8 with depth >= 2: each frame's Phi runs fused with the Gram row
    # depth - 1 frames later (depth 2: the new window starts at the first
    # staged row; m = 130: K padded to 160, eight units per converter lane;
    # r = 20: two mode passes, the Gram dots in the first; m = 250 at depth 7:
    # a union of 255 slots, K = 256 with four converter warps; at depth 8 the
    # union would pass 255 slots and Phi and the Gram row run apart)
    if kind == "u8":
        vs = synth.VideoStream(H=60 if m < 100 else 24, W=80 if m < 100 else 40, C=3, seed=synth.config_seed(2))
        n = vs.n
        frames = [vs.frame(t) for t in range(3 * (m + depth) + 5)]
        dt = S.SDMD_U8
    else:
        ps = synth.PlantedStream(side=40, noise_var=1e-4, seed=5)
        n = ps.n
        frames = [ps.snapshot(t) for t in range(3 * (m + depth) + 5)]
        dt = S.SDMD_F32
    dev_frames = [torch.from_numpy(f).to(cuda_device) for f in frames]
    T = len(frames)
    # frames compared (every frame for short windows; for long ones every
    # seventh, the eigensolver being O(m^3) per frame)
    check = set(range(2, T)) if m < 200 else set(range(6, T, 7)) | {T - 1}
    hp = S.sdmd_create_ex(n, m, dt, depth)
    hs = S.sdmd_create(n, m, dt)
    # the serial handle's Phi in tensor-core passes of 16 modes: the
    # pipelined one (one pass of 10 modes where r <= 10) must give the same bits
    S.sdmd_set_option(hs, S.SDMD_OPT_PHI_TENSOR, 2)
    nb = max(depth, 1)
    phis = [torch.zeros(r, n, 2, dtype=torch.float32, device=cuda_device) for _ in range(nb)]
    lam_p = torch.zeros(T, 2 * r, dtype=torch.float64, device=cuda_device)
    rk_p = torch.zeros(T, dtype=torch.int32, device=cuda_device)
    phi_p = {}
    stream = torch.cuda.Stream(device=cuda_device)
    try:
        with torch.cuda.stream(stream):
            for t in range(T):
                S.sdmd_step(hp, dev_frames[t], r, phis[t % nb], lam_p[t], rk_p[t:t + 1], stream)
                if t % 7 == 6 and t >= 2:
                    # keep a copy of this frame's modes once its outputs are complete
                    S.sdmd_sync(hp, stream)
                    phi_p[t] = phis[t % nb].clone()
            S.sdmd_sync(hp, stream)
        stream.synchronize()
        assert S.sdmd_status(hp) == S.SDMD_OK
        phi_s = torch.zeros(r, n, 2, dtype=torch.float32, device=cuda_device)
        for t in range(T):
            S.sdmd_push(hs, dev_frames[t])
            if t not in check:
                continue
            lam_s = torch.zeros(2 * r, dtype=torch.float64, device=cuda_device)
            rk_s = torch.zeros(1, dtype=torch.int32, device=cuda_device)
            S.sdmd_modes(hs, r, phi_s, lam_s, rk_s)
            torch.cuda.synchronize()
            assert torch.equal(lam_s, lam_p[t]), t
            assert torch.equal(rk_s, rk_p[t:t + 1]), t
            if t in phi_p:
                assert torch.equal(phi_s, phi_p[t]), t
    finally:
        S.sdmd_destroy(hp)
        S.sdmd_destroy(hs)


def test_rebuild_waits_for_frames_in_flight(cuda_device):
    # the eigensolvers of frames in flight read the window's G in place; a
    # rebuild rewrites every entry (BF16x3 on an FP32 window: within 1e-6 of
    # the FP32 row passes, not equal to them), so it must wait for them: every
    # frame stepped before the rebuild matches the serial handle bit for bit
    ps = synth.PlantedStream(side=40, noise_var=1e-4, seed=9)
    n, m, depth, r = ps.n, 24, 4, 5
    T = m + 12
    t_rb = T - 5
    frames = [torch.from_numpy(ps.snapshot(t)).to(cuda_device) for t in range(T)]
    hp = S.sdmd_create_ex(n, m, S.SDMD_F32, depth)
    hs = S.sdmd_create(n, m, S.SDMD_F32)
    lam_p = torch.zeros(T, 2 * r, dtype=torch.float64, device=cuda_device)
    rk_p = torch.zeros(T, dtype=torch.int32, device=cuda_device)
    phis = [torch.zeros(r, n, 2, dtype=torch.float32, device=cuda_device) for _ in range(depth)]
    stream = torch.cuda.Stream(device=cuda_device)
    try:
        S.sdmd_set_option(hp, S.SDMD_OPT_F32_BF16X3, 1)   # single pushes stay FP32 row passes
        with torch.cuda.stream(stream):
            for t in range(T):
                S.sdmd_step(hp, frames[t], r, phis[t % depth], lam_p[t], rk_p[t:t + 1], stream)
                if t == t_rb:
                    S.sdmd_rebuild(hp, stream)
            S.sdmd_sync(hp, stream)
        stream.synchronize()
        assert S.sdmd_status(hp) == S.SDMD_OK
        for t in range(T):
            S.sdmd_push(hs, frames[t])
            if t < 2 or t > t_rb:
                continue
            lam_s = torch.zeros(2 * r, dtype=torch.float64, device=cuda_device)
            rk_s = torch.zeros(1, dtype=torch.int32, device=cuda_device)
            S.sdmd_modes(hs, r, None, lam_s, rk_s)
            torch.cuda.synchronize()
            assert torch.equal(lam_s, lam_p[t]), t
            assert torch.equal(rk_s, rk_p[t:t + 1]), t
    finally:
        S.sdmd_destroy(hp)
        S.sdmd_destroy(hs)


def _phi_reference_full(frames, t, m, M):
    """The oracle's modes X' M of the window ending at frame t, every row:
    X' = frames t - m + 2 .. t (exact uint8 values in FP64), M from the
    oracle's Algorithm 2 (complex, p x k); row blocks keep the FP64 copy of
    X' small."""
    slots = list(range(t - m + 2, t + 1))
    n = frames[slots[0]].size
    out = np.empty((n, M.shape[1]), dtype=np.complex128)
    blk = 1 << 18
    for lo in range(0, n, blk):
        hi = min(n, lo + blk)
        Xb = np.stack([frames[s][lo:hi] for s in slots], axis=1).astype(np.float64)
        out[lo:hi] = Xb @ M.real + 1j * (Xb @ M.imag)
    return out


@pytest.mark.parametrize("D", [8, 10])
def test_full_size_hd_video_pipelined(cuda_device, D):
    # The benchmark's launch configuration: n = 1920*1080*3 uint8, m = 100,
    # r = 10, sdmd_step with D frames in flight (each frame's Phi fused with
    # the Gram row of the frame D - 1 steps later: 106 or 108 union slots,
    # K = 112; the bench default is 8).
    # Against the oracle: the final G exactly, and for two of the last frames
    # the rank, the eigenvalues (1e-6) and every one of the n x r entries of
    # Phi (1e-4 of each column's largest entry, after fixing the column's
    # phase at that entry), so a wrong tile anywhere (the ragged last tile,
    # the last CTA's chunk, a tile after a chunk grab) fails.
    import oracle
    from helpers import match_eigs
    vs = synth.VideoStream(seed=synth.config_seed(2))
    n, m, r = vs.n, 100, 10
    T = m + D + 6
    frames = [vs.frame(t) for t in range(T)]
    dev_frames = [torch.from_numpy(f).to(cuda_device) for f in frames]
    h = S.sdmd_create_ex(n, m, S.SDMD_U8, D)
    phis = [torch.zeros(r, n, 2, dtype=torch.float32, device=cuda_device) for _ in range(D)]
    lam = torch.zeros(T, 2 * r, dtype=torch.float64, device=cuda_device)
    rk = torch.zeros(T, dtype=torch.int32, device=cuda_device)
    stream = torch.cuda.Stream(device=cuda_device)
    try:
        with torch.cuda.stream(stream):
            for t in range(T):
                S.sdmd_step(h, dev_frames[t], r, phis[t % D], lam[t], rk[t:t + 1], stream)
            S.sdmd_sync(h, stream)
        stream.synchronize()
        assert S.sdmd_status(h) == S.SDMD_OK
        G = torch.empty(m, m, dtype=torch.int64, device=cuda_device)
        S.sdmd_gram(h, G)
        torch.cuda.synchronize()
        Gall = oracle.gram_u8_cols(frames)                      # exact, all T frames
        assert np.array_equal(G.cpu().numpy(), Gall[T - m:, T - m:])
        lam_h = lam.cpu().numpy()
        rk_h = rk.cpu().numpy()
        for t in (T - 1, T - D):
            Gw = Gall[t - m + 1:t + 1, t - m + 1:t + 1].astype(np.float64)
            ref = oracle.dmd_from_gram(Gw[:-1, :-1], Gw[:-1, 1:], r)
            k = int(rk_h[t])
            assert k == ref.r, t
            got_lam = lam_h[t, 0::2] + 1j * lam_h[t, 1::2]
            err, perm = match_eigs(got_lam[:k], ref.lam)
            assert err <= 1e-6, (t, err)
            Pref = _phi_reference_full(frames, t, m, ref.M[:, perm])
            P = phis[t % D].cpu().numpy()                     # r x n x (re, im)
            for q in range(k):
                got = P[q, :, 0].astype(np.float64) + 1j * P[q, :, 1].astype(np.float64)
                col = Pref[:, q]
                i = int(np.argmax(np.abs(col)))
                scale = abs(col[i])
                ph = (col[i] / got[i]) / abs(col[i] / got[i])
                dev_max = np.abs(got * ph - col).max()
                assert dev_max <= 1e-4 * scale, (t, q, dev_max / scale)
    finally:
        S.sdmd_destroy(h)


def test_host_early_read_equals_device_frames(cuda_device):
    # SDMD_OPT_HOST_EARLY_READ: pinned host frames copied on the handle's copy
    # stream as soon as each call is made (two staging slots, then a device
    # copy into the ring on the push stream). Every frame's eigenvalues, rank
    # and modes, and the final G, equal those of the same frames given on the
    # device; sdmd_push of host frames with the option gives the same G too.
    vs = synth.VideoStream(H=60, W=80, C=3, seed=synth.config_seed(2) + 7)
    n, m, depth, r = vs.n, 16, 4, 5
    T = 3 * (m + depth) + 3
    host = torch.from_numpy(np.stack([vs.frame(t) for t in range(T)])).pin_memory()
    dev = host.to(cuda_device)
    out = []
    for early in (False, True):
        h = S.sdmd_create_ex(n, m, S.SDMD_U8, depth)
        if early:
            S.sdmd_set_option(h, S.SDMD_OPT_HOST_EARLY_READ, 1)
        phis = [torch.zeros(r, n, 2, dtype=torch.float32, device=cuda_device) for _ in range(depth)]
        lam = torch.zeros(T, 2 * r, dtype=torch.float64, device=cuda_device)
        rk = torch.zeros(T, dtype=torch.int32, device=cuda_device)
        stream = torch.cuda.Stream(device=cuda_device)
        try:
            with torch.cuda.stream(stream):
                for t in range(T):
                    S.sdmd_step(h, host[t] if early else dev[t], r, phis[t % depth], lam[t], rk[t:t + 1], stream)
                S.sdmd_sync(h, stream)
            stream.synchronize()
            assert S.sdmd_status(h) == S.SDMD_OK
            G = torch.empty(m, m, dtype=torch.int64, device=cuda_device)
            S.sdmd_gram(h, G)
            torch.cuda.synchronize()
            out.append((lam.cpu(), rk.cpu(), [p.cpu() for p in phis], G.cpu()))
        finally:
            S.sdmd_destroy(h)
    (l0, r0, p0, g0), (l1, r1, p1, g1) = out
    assert torch.equal(l0, l1) and torch.equal(r0, r1) and torch.equal(g0, g1)
    assert all(torch.equal(a, b) for a, b in zip(p0, p1))
    hs = S.sdmd_create(n, m, S.SDMD_U8)
    try:
        S.sdmd_set_option(hs, S.SDMD_OPT_HOST_EARLY_READ, 1)
        for t in range(T):
            S.sdmd_push(hs, host[t])
        G = torch.empty(m, m, dtype=torch.int64, device=cuda_device)
        S.sdmd_gram(hs, G)
        torch.cuda.synchronize()
        assert torch.equal(G.cpu(), g0)
    finally:
        S.sdmd_destroy(hs)
