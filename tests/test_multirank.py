"""The multi-rank host logic of bench.py on CPU, as two gloo ranks: each rank
reads its place from the launcher's environment, times its own region, and
the reported time is the slowest rank's (an all-reduce MAX after the closing
barrier); the whole-job rate counts every rank's steps over that time; every
rank streams its own video (distinct seeds, no data exchange); the reference
arm runs on rank 0 only, the other ranks return without work or output."""
import argparse
import contextlib
import io
import os
import socket

import pytest

mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        dist.barrier()
        own_ms = 100.0 + 50.0 * r                       # rank 1 is the slower one
        t_max = bench.max_over_ranks(own_ms, w, "cpu")
        rate = bench.job_rate(w, 10, t_max)
        printed = None
        if r != 0:                                      # the reference arm: rank 0 only
            buf = io.StringIO()
            args = argparse.Namespace(gpus=w, steps=1, warmup=3)
            with contextlib.redirect_stdout(buf):
                ret = bench.run_reference(args)
            printed = (ret, buf.getvalue())
        dist.barrier()
        q.put((r, w, local, t_max, rate, bench.rank_seed(17, r), printed))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[:3] for x in res] == [(0, 2, 0), (1, 2, 1)]
    for _, _, _, t_max, rate, _, _ in res:
        assert t_max == 150.0                           # the slowest rank's time on every rank
        assert rate == pytest.approx(2 * 10 / 0.150)     # both ranks' steps over it
    assert res[0][5] != res[1][5]                       # independent streams
    assert res[1][6] == (None, "")                      # rank 1: no reference work, no output


def test_single_rank_defaults(monkeypatch):
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (0, 1, 0)
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_rate(1, 100, 50.0) == pytest.approx(2000.0)
