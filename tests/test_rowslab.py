"""Row-slab split of one stream over ranks (positions split into slabs, one
all-reduce of the c partial Gram-row values per push), host logic on the CPU
as two and three gloo ranks.

Each rank runs the product's RowSlabStream with a stand-in engine that keeps
its slab of the window on the host and forms the partial row with the
oracle's exact dot products (the GPU's Gram-row kernel is what the real
engine calls; its own parity is tested elsewhere). After every push every
rank's G must equal the oracle's exact Gram of the whole window, so slab
bounds that miss or double-count a position, a reduction in the wrong place
or a row written in the wrong order fail.
"""
import os
import socket

import numpy as np
import pytest

mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class _HostSlabEngine:
    """CPU stand-in of SdmdEngine: ring of slab snapshots, physical G with
    the newest row/column written from time-ordered rows."""

    def __init__(self, m):
        import torch
        self.torch = torch
        self.m = m
        self.ring = [None] * m
        self.G = np.zeros((m, m), dtype=np.int64)
        self.count = 0

    def _order(self):
        c = min(self.count, self.m)
        return [(self.count - c + q) % self.m for q in range(c)]

    def push(self, xs):
        import oracle
        s = self.count % self.m
        self.ring[s] = np.ascontiguousarray(xs)
        self.count += 1
        for j in self._order():
            v = oracle.dot_u8(self.ring[j], self.ring[s])
            self.G[s, j] = self.G[j, s] = v

    def newest_row(self):
        s = (self.count - 1) % self.m
        return self.torch.tensor([self.G[s, j] for j in self._order()], dtype=self.torch.int64)

    def set_newest_row(self, row):
        s = (self.count - 1) % self.m
        for q, j in enumerate(self._order()):
            self.G[s, j] = self.G[j, s] = int(row[q])

    def gram(self):
        o = self._order()
        return self.G[np.ix_(o, o)]


def _rank(rank, world, port, n, m, T, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import oracle
    from paper_1612_07875_gb300 import rowslab
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(77)
        frames = rng.integers(0, 256, (T, n), dtype=np.uint8)
        eng = _HostSlabEngine(m)
        rs = rowslab.RowSlabStream(eng, dist.all_reduce, n, world, rank)
        ok = True
        for t in range(T):
            rs.push(frames[t])
            c = min(t + 1, m)
            ref = oracle.gram_u8(frames[t - c + 1:t + 1].T)
            ok = ok and np.array_equal(eng.gram(), ref)
        q.put((rank, rs.lo, rs.hi, ok))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_row_slab_ranks_reduce_to_the_whole_gram(world):
    n, m, T = 1000 + 7, 6, 15                 # ragged n, the ring wraps twice
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, n, m, T, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(ok for *_, ok in res)
    bounds = [(lo, hi) for _, lo, hi, _ in res]
    assert bounds[0][0] == 0 and bounds[-1][1] == n
    assert all(a[1] == b[0] for a, b in zip(bounds, bounds[1:]))


def test_slab_bounds():
    from paper_1612_07875_gb300.rowslab import slab_bounds
    for n in (16, 17, 1000, 6220800, 4096 * 3 + 5):
        for world in (1, 2, 3, 4, 8):
            if (n + 15) // 16 < world:
                with pytest.raises(ValueError):
                    slab_bounds(n, world, 0)
                continue
            b = [slab_bounds(n, world, r) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == n
            assert all(x[1] == y[0] for x, y in zip(b, b[1:]))
            assert all(lo % 16 == 0 and hi > lo for lo, hi in b)
            sizes = [hi - lo for lo, hi in b]
            assert max(sizes) - min(sizes) < 32
