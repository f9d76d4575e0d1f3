"""Row-slab split on one GPU: two handles each hold one slab of the
positions of every snapshot (the split two ranks would use), their partial
Gram rows are summed after every push (what the all-reduce does between
GPUs) and written back with sdmd_set_newest_row. Against a handle that holds
whole snapshots: G bit for bit (uint8) or within the FP32 Gram tolerance,
eigenvalues and rank bit for bit on both slab handles (same G, same
eigensolver), and each slab handle's Phi equal to its rows of the whole Phi."""
import numpy as np
import pytest
import torch

from helpers import match_eigs
from paper_1612_07875_gb300 import rowslab
from paper_1612_07875_gb300 import sdmd as S
from paper_1612_07875_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ["u8", "f32"])
def test_two_slabs_equal_whole_snapshots(cuda_device, kind):
    m, r, world = 16, 5, 2
    if kind == "u8":
        vs = synth.VideoStream(H=90, W=120, C=3, seed=synth.config_seed(2) + 3)
        n, dt = vs.n, S.SDMD_U8
        frames = [vs.frame(t) for t in range(2 * m + 5)]
    else:
        ps = synth.PlantedStream(side=72, noise_var=1e-4, seed=9)
        n, dt = ps.n, S.SDMD_F32
        frames = [ps.snapshot(t) for t in range(2 * m + 5)]
    X = torch.from_numpy(np.stack(frames)).to(cuda_device)
    bounds = [rowslab.slab_bounds(n, world, k) for k in range(world)]
    engines = [rowslab.SdmdEngine(hi - lo, m, dt, cuda_device) for lo, hi in bounds]
    hw = S.sdmd_create(n, m, dt)
    try:
        for t in range(X.shape[0]):
            S.sdmd_push(hw, X[t])
            rows = []
            for e, (lo, hi) in zip(engines, bounds):
                e.push(X[t, lo:hi].contiguous())
                rows.append(e.newest_row())
            total = rows[0] + rows[1]              # the all-reduce of the partial rows
            for e in engines:
                e.set_newest_row(total)
        gt = torch.int64 if kind == "u8" else torch.float64
        Gw = torch.empty(m, m, dtype=gt, device=cuda_device)
        S.sdmd_gram(hw, Gw)
        Gs = []
        for e in engines:
            G = torch.empty(m, m, dtype=gt, device=cuda_device)
            S.sdmd_gram(e.h, G)
            Gs.append(G)
        torch.cuda.synchronize()
        for G in Gs:
            if kind == "u8":
                assert torch.equal(G, Gw)
            else:
                d = torch.sqrt(torch.diag(Gw))
                assert ((G - Gw).abs() <= 1e-5 * torch.outer(d, d)).all()
        assert torch.equal(Gs[0], Gs[1])           # every rank holds the same G
        # the replicated small algebra, Phi rows local to each slab
        phi_w = torch.zeros(r, n, 2, dtype=torch.float32, device=cuda_device)
        lam_w = torch.zeros(2 * r, dtype=torch.float64, device=cuda_device)
        rk_w = torch.zeros(1, dtype=torch.int32, device=cuda_device)
        S.sdmd_modes(hw, r, phi_w, lam_w, rk_w)
        for e, (lo, hi) in zip(engines, bounds):
            phi = torch.zeros(r, hi - lo, 2, dtype=torch.float32, device=cuda_device)
            lam = torch.zeros(2 * r, dtype=torch.float64, device=cuda_device)
            rk = torch.zeros(1, dtype=torch.int32, device=cuda_device)
            S.sdmd_modes(e.h, r, phi, lam, rk)
            torch.cuda.synchronize()
            if kind == "u8":
                assert torch.equal(lam, lam_w) and torch.equal(rk, rk_w)
                assert torch.equal(phi, phi_w[:, lo:hi])
            else:                                  # as multisets: a conjugate pair's order is rounding's
                assert torch.equal(rk, rk_w)
                k = int(rk_w.item())
                lw, ls = lam_w.cpu().numpy(), lam.cpu().numpy()
                err, _ = match_eigs((ls[0::2] + 1j * ls[1::2])[:k], (lw[0::2] + 1j * lw[1::2])[:k])
                assert err <= 1e-6
        for e in engines:
            assert S.sdmd_status(e.h) == S.SDMD_OK
    finally:
        S.sdmd_destroy(hw)
        for e in engines:
            e.close()


def test_newest_row_round_trip_host_buffers(cuda_device):
    # host (pageable) buffers for both calls; the column is the conjugate
    # (complex windows) and the row is in time order after the ring wraps
    m, n = 6, 4096
    rng = np.random.default_rng(4)
    h = S.sdmd_create(n, m, S.SDMD_C64)
    try:
        for t in range(m + 3):
            x = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
            S.sdmd_push(h, torch.from_numpy(x.view(np.float32)).to(cuda_device))
        row = np.zeros(2 * m)
        S.sdmd_newest_row(h, row)
        G = np.zeros(2 * m * m)
        S.sdmd_gram(h, G)
        Gc = G[0::2] + 1j * G[1::2]
        Gc = Gc.reshape(m, m)
        assert np.array_equal(row[0::2] + 1j * row[1::2], Gc[m - 1, :])
        new = (np.arange(m) + 1.0) + 1j * (np.arange(m) - 2.5)
        new[-1] = 7.0                              # the diagonal is real
        buf = np.zeros(2 * m)
        buf[0::2], buf[1::2] = new.real, new.imag
        S.sdmd_set_newest_row(h, buf)
        S.sdmd_gram(h, G)
        Gc = (G[0::2] + 1j * G[1::2]).reshape(m, m)
        assert np.array_equal(Gc[m - 1, :], new)
        assert np.array_equal(Gc[:, m - 1], np.conj(new))
    finally:
        S.sdmd_destroy(h)
