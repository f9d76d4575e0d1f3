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


@pytest.mark.parametrize("kind,depth,m", [("u8", 4, 12), ("f32", 3, 12), ("u8", 1, 12), ("u8", 2, 12), ("u8", 6, 12),
                                          ("u8", 3, 130)])
def test_pipelined_step_equals_serial(cuda_device, kind, depth, m):
    # uint8 with depth >= 2: each frame's Phi runs fused with the Gram row
    # depth - 1 frames later (depth 2: the new window starts at the first
    # staged row; m = 130: K padded to 160, eight units per converter lane)
    r = 5
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
    hp = S.sdmd_create_ex(n, m, dt, depth)
    hs = S.sdmd_create(n, m, dt)
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
            if t < 2:
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
