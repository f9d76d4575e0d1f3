"""Batching many streams (sdmd_push_many: one launch for the Gram rows of many
handles with uneven n, window and element type) and serving them
(sdmd_server_*: admission by device-memory footprint, queued streams admitted
as memory frees, ticks that batch whatever frames are waiting).

Bar: every stream's G equals, bit for bit, the G of the same frames pushed
alone on its own handle, whatever the mix it was batched with; eigenvalues
from the served handle equal those from the lone handle bit for bit.
"""
import numpy as np
import pytest
import torch

from paper_1612_07875_gb300 import sdmd as S

pytestmark = pytest.mark.gpu

DT = {"u8": S.SDMD_U8, "f32": S.SDMD_F32, "c64": S.SDMD_C64}


def _frame(kind, n, rng):
    if kind == "u8":
        return rng.integers(0, 256, n, dtype=np.uint8)
    if kind == "f32":
        return rng.standard_normal(n).astype(np.float32)
    return (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64).view(np.float32)


def _gram_bytes(h, c, kind, stream=None):
    words = 2 if kind == "c64" else 1
    G = torch.empty(c, c, words, dtype=torch.int64, device="cuda")
    S.sdmd_gram(h, G, stream)
    torch.cuda.synchronize()
    return G.cpu().numpy()


STREAMS = [("u8", 100003, 16), ("f32", (1 << 16) + 7, 32), ("c64", 5000, 8), ("u8", 6000, 127),
           ("f32", 777, 5), ("u8", 1920 * 1080 * 3, 10)]


def test_push_many_bitwise_equals_single_pushes(cuda_device):
    rng = np.random.default_rng(7)
    hb = [S.sdmd_create(n, m, DT[k]) for k, n, m in STREAMS]
    hs = [S.sdmd_create(n, m, DT[k]) for k, n, m in STREAMS]
    pushed = [0] * len(STREAMS)
    try:
        for t in range(40):
            # a different mix every tick (continuous batching)
            sub = [i for i in range(len(STREAMS)) if rng.random() < 0.7] or [0]
            xs = []
            for i in sub:
                k, n, _ = STREAMS[i]
                x = torch.from_numpy(_frame(k, n, rng)).to(cuda_device)
                xs.append(x)
                S.sdmd_push(hs[i], x)
                pushed[i] += 1
            S.sdmd_push_many([hb[i] for i in sub], xs)
        for i, (k, n, m) in enumerate(STREAMS):
            c = min(pushed[i], m)
            if c == 0:
                continue
            assert np.array_equal(_gram_bytes(hb[i], c, k), _gram_bytes(hs[i], c, k)), STREAMS[i]
            assert S.sdmd_status(hb[i]) == S.SDMD_OK
        # the eigensolvers see the same G: same eigenvalues, bit for bit
        for i in (0, 1):
            k, n, m = STREAMS[i]
            if min(pushed[i], m) < 3:
                continue
            la, lb = np.zeros(8), np.zeros(8)
            S.sdmd_modes(hb[i], 4, None, la)
            S.sdmd_modes(hs[i], 4, None, lb)
            torch.cuda.synchronize()
            assert np.array_equal(la, lb)
    finally:
        for h in hb + hs:
            S.sdmd_destroy(h)


def test_push_many_argument_errors(cuda_device):
    h = S.sdmd_create(100, 4, S.SDMD_U8)
    x = torch.zeros(100, dtype=torch.uint8, device=cuda_device)
    try:
        for hs, xs in (([h, h], [x, x]), ([], [])):
            with pytest.raises(S.SdmdError) as ei:
                S.sdmd_push_many(hs, xs)
            assert ei.value.code == S.SDMD_ERR_ARG
    finally:
        S.sdmd_destroy(h)


def test_server_admission_and_continuous_batching(cuda_device):
    rng = np.random.default_rng(11)
    specs = [("u8", 200003, 12), ("f32", 50001, 20), ("u8", 300007, 8)]
    # the first two fit; the third waits until the first closes
    probe = S.sdmd_server_create(1 << 40)
    sizes = []
    for k, n, m in specs:
        sid = S.sdmd_server_open(probe, n, m, DT[k])
        sizes.append(S.sdmd_server_used_bytes(probe) - sum(sizes))
    S.sdmd_server_destroy(probe)
    budget = sizes[0] + sizes[1] + sizes[2] // 2
    srv = S.sdmd_server_create(budget)
    alone = [S.sdmd_create(n, m, DT[k]) for k, n, m in specs]
    pushed = [0, 0, 0]
    try:
        sids = [S.sdmd_server_open(srv, n, m, DT[k]) for k, n, m in specs]
        assert [S.sdmd_server_state(srv, s) for s in sids] == [S.SDMD_STREAM_ACTIVE, S.SDMD_STREAM_ACTIVE,
                                                                S.SDMD_STREAM_WAITING]
        with pytest.raises(S.SdmdError) as ei:
            S.sdmd_server_submit(srv, sids[2], np.zeros(specs[2][1], np.uint8))
        assert ei.value.code == S.SDMD_ERR_NOT_READY
        with pytest.raises(S.SdmdError) as ei:                     # alone exceeds the budget
            S.sdmd_server_open(srv, 1 << 30, 64, S.SDMD_F32)
        assert ei.value.code == S.SDMD_ERR_ARG

        def feed(i, count):
            k, n, _ = specs[i]
            for _ in range(count):
                x = _frame(k, n, rng)
                S.sdmd_server_submit(srv, sids[i], x)           # host source
                S.sdmd_push(alone[i], torch.from_numpy(x).to(cuda_device))
                pushed[i] += 1

        for t in range(15):
            feed(0, 1)
            if t % 2 == 0:
                feed(1, 2)
            while S.sdmd_server_tick(srv) > 0:
                pass
        # backpressure: a queue holds 4 frames
        feed(1, 4)
        with pytest.raises(S.SdmdError) as ei:
            S.sdmd_server_submit(srv, sids[1], _frame("f32", specs[1][1], rng))
        assert ei.value.code == S.SDMD_ERR_NOT_READY
        while S.sdmd_server_tick(srv) > 0:
            pass
        # compare stream 0 with its lone run before it closes
        st = S.sdmd_server_stream(srv)
        c0 = min(pushed[0], specs[0][2])
        h0 = S.sdmd_server_handle(srv, sids[0])
        assert np.array_equal(_gram_bytes(h0, c0, "u8", st), _gram_bytes(alone[0], c0, "u8"))
        S.sdmd_server_close(srv, sids[0])
        assert S.sdmd_server_state(srv, sids[2]) == S.SDMD_STREAM_ACTIVE      # admitted on release
        for t in range(10):
            feed(1, 1)
            feed(2, 1)
            S.sdmd_server_tick(srv)
        for i in (1, 2):
            k, _, m = specs[i]
            c = min(pushed[i], m)
            h = S.sdmd_server_handle(srv, sids[i])
            assert np.array_equal(_gram_bytes(h, c, k, st), _gram_bytes(alone[i], c, k)), specs[i]
            assert S.sdmd_status(h, st) == S.SDMD_OK
        p50, p99, frames = S.sdmd_server_stats(srv)
        assert frames == sum(pushed)
        assert 0.0 < p50 <= p99
        # latencies against given arrival times on the server's clock
        S.sdmd_server_reset_stats(srv)
        assert S.sdmd_server_stats(srv)[2] == 0
        t_arr = S.sdmd_server_clock_ms() - 50.0
        x = _frame("f32", specs[1][1], rng)
        S.sdmd_server_submit(srv, sids[1], x, t_arr)
        assert S.sdmd_server_tick(srv) == 1
        p50, p99, frames = S.sdmd_server_stats(srv)
        assert frames == 1 and 50.0 <= p50 == p99 < S.sdmd_server_clock_ms() - t_arr
    finally:
        S.sdmd_server_destroy(srv)
        for h in alone:
            S.sdmd_destroy(h)


def test_graph_ticks_equal_direct_ticks(cuda_device):
    # the same submissions through a server with graph ticks and one without:
    # every stream's G bit for bit equal; graphs are built once per set of
    # streams and then updated in place
    rng = np.random.default_rng(21)
    specs = [("u8", 30011, 9), ("f32", 20003, 12), ("u8", 7001, 5), ("c64", 3001, 6)]
    srv = [S.sdmd_server_create(1 << 36), S.sdmd_server_create(1 << 36)]
    S.sdmd_server_set_graphs(srv[1], False)
    try:
        sids = [[S.sdmd_server_open(v, n, m, DT[k]) for k, n, m in specs] for v in srv]
        for t in range(30):
            live = [i for i in range(len(specs)) if t < 12 or rng.random() < 0.6]   # steady, then mixed
            for i in live:
                k, n, _ = specs[i]
                x = _frame(k, n, rng)
                for v in range(2):
                    S.sdmd_server_submit(srv[v], sids[v][i], x)
            for v in range(2):
                S.sdmd_server_tick(srv[v])
        builds, updates = S.sdmd_server_graph_stats(srv[0])
        assert builds >= 1 and updates >= 9           # steady ticks: one build, then in-place updates
        assert S.sdmd_server_graph_stats(srv[1]) == (0, 0)
        for i, (k, n, m) in enumerate(specs):
            hs = [S.sdmd_server_handle(srv[v], sids[v][i]) for v in range(2)]
            c = min(S.sdmd_count(hs[0]), m)
            Ga = _gram_bytes(hs[0], c, k, S.sdmd_server_stream(srv[0]))
            Gb = _gram_bytes(hs[1], c, k, S.sdmd_server_stream(srv[1]))
            assert np.array_equal(Ga, Gb), specs[i]
        builds = S.sdmd_server_graph_stats(srv[0])[0]
        S.sdmd_server_autotune(srv[0])                 # schedules re-picked; graphs rebuilt when steady again
        for _ in range(2):
            for i, (k, n, _) in enumerate(specs):
                S.sdmd_server_submit(srv[0], sids[0][i], _frame(k, n, rng))
            assert S.sdmd_server_tick(srv[0]) == len(specs)
        assert S.sdmd_server_graph_stats(srv[0])[0] == builds + 1
        for i in range(len(specs)):
            assert S.sdmd_status(S.sdmd_server_handle(srv[0], sids[0][i]), S.sdmd_server_stream(srv[0])) == S.SDMD_OK
    finally:
        for v in srv:
            S.sdmd_server_destroy(v)


def test_autotune_keeps_the_gram_exact(cuda_device):
    # sdmd_autotune picks a chunk schedule by timing; uint8 Grams stay exact
    # and float Grams within their tolerance of the oracle across the change
    import oracle
    rng = np.random.default_rng(5)
    for kind, n, m in (("u8", 1920 * 1080 * 3 // 4, 12), ("f32", (1 << 18) + 3, 10)):
        h = S.sdmd_create(n, m, DT[kind])
        so = oracle.StreamOracle(n, m, kind)
        try:
            with pytest.raises(S.SdmdError) as ei:
                S.sdmd_autotune(h)
            assert ei.value.code == S.SDMD_ERR_NOT_READY
            for t in range(m + 5):
                x = _frame(kind, n, rng)
                S.sdmd_push(h, torch.from_numpy(x).to(cuda_device))
                so.push(x)
                if t == m // 2:
                    chunk, us = S.sdmd_autotune(h)
                    assert chunk % 4096 == 0 and 4096 <= chunk <= 24576 and us > 0
            G = _gram_bytes(h, m, kind)
            ref = so.gram()
            if kind == "u8":
                assert np.array_equal(G[..., 0], ref)
            else:
                Gf = G[..., 0].view(np.float64)
                assert np.linalg.norm(Gf - ref) <= 1e-9 * np.linalg.norm(ref)
            assert S.sdmd_status(h) == S.SDMD_OK
        finally:
            S.sdmd_destroy(h)


def test_modes_many_equals_one_handle_at_a_time(cuda_device):
    # sdmd_modes_many: the eigensolvers of several windows (uneven n, window
    # length, element type, rank) in one launch give, bit for bit, the
    # eigenvalues, rank and singular values of sdmd_modes on each handle
    specs = [("u8", 100003, 16, 5), ("f32", (1 << 16) + 7, 32, 10), ("u8", 6000, 127, 20), ("f32", 777, 5, 4),
             ("u8", 4096 * 3, 64, 63), ("f32", 3000, 100, 10), ("u8", 50000, 256, 10)]
    rng = np.random.default_rng(12)
    hs = []
    try:
        for kind, n, m, _ in specs:
            h = S.sdmd_create(n, m, DT[kind])
            hs.append(h)
            base = _frame(kind, n, rng)
            for t in range(m + 3):
                # slowly drifting frames, so the windows have structure
                f = base if kind == "u8" and t % 3 else _frame(kind, n, rng)
                S.sdmd_push(h, torch.from_numpy(f).to(cuda_device))
        rs = [r for *_, r in specs]
        lams = [torch.full((2 * r,), -1.0, dtype=torch.float64, device=cuda_device) for r in rs]
        rk = torch.full((len(hs),), -1, dtype=torch.int32, device=cuda_device)
        S.sdmd_modes_many(hs, rs, lams, rk)
        sig_b = []
        for h, r in zip(hs, rs):
            sg = torch.zeros(r, dtype=torch.float64, device=cuda_device)
            S.sdmd_svd(h, r, sg, None)
            sig_b.append(sg)
        torch.cuda.synchronize()
        for i, (h, r) in enumerate(zip(hs, rs)):
            lam1 = torch.full((2 * r,), -1.0, dtype=torch.float64, device=cuda_device)
            rk1 = torch.full((1,), -1, dtype=torch.int32, device=cuda_device)
            S.sdmd_modes(h, r, None, lam1, rk1)
            sg = torch.zeros(r, dtype=torch.float64, device=cuda_device)
            S.sdmd_svd(h, r, sg, None)
            torch.cuda.synchronize()
            assert torch.equal(lam1, lams[i]), i
            assert int(rk1.item()) == int(rk[i].item()) >= 1, i
            assert torch.equal(sg, sig_b[i]), i
            assert S.sdmd_status(h) == S.SDMD_OK
        with pytest.raises(S.SdmdError) as ei:
            S.sdmd_modes_many([hs[0], hs[0]], 3)
        assert ei.value.code == S.SDMD_ERR_ARG
    finally:
        for h in hs:
            S.sdmd_destroy(h)
