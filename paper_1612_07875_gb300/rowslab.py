"""Row-slab split of one snapshot stream over several GPUs (one rank each).

Every entry of the streamed Gram row is a sum over the n positions of two
snapshots (Sec. 3.1, Eq. 12a-b), so the positions split into contiguous
slabs, one per rank. A rank keeps positions [lo, hi) of every snapshot of the
window in its own handle (n = hi - lo), and one push is:

  1. sdmd_push of the rank's part of x_new: the library's Gram-row kernel
     computes the partial row over the slab and inserts it into the rank's G;
  2. sdmd_newest_row reads that partial row (c values, time order);
  3. one all-reduce (sum) of the c values across the ranks -- the only data
     exchanged per snapshot (at most 256 x 8 bytes; exact for int64);
  4. sdmd_set_newest_row writes the sum back, so every rank's G is the whole
     window's G.

The m x m eigen-work then runs replicated (the same G gives the same
eigenvalues on every rank) and each rank's Phi holds its own rows lo .. hi-1.
Independent streams need none of this: they shard as whole streams.

This module holds the host logic only (slab bounds and the order of the four
steps). The device work is the library's (`SdmdEngine`); the reduction is
`torch.distributed.all_reduce` over whatever process group the caller set up
(NCCL between GPUs).
"""
from . import sdmd as S


def slab_bounds(n, world, rank, align=16):
    """Positions [lo, hi) of `rank`'s slab of n positions split over `world`
    ranks: contiguous, every start a multiple of `align` elements (16 keeps
    each slab's start 16-byte aligned for the bulk copies of the Gram-row
    kernel), sizes within 2 align of each other, covering 0 .. n-1 exactly
    once. Raises ValueError when some rank would get no positions."""
    if world < 1 or not 0 <= rank < world or align < 1:
        raise ValueError("bad world/rank/align: %r %r %r" % (world, rank, align))
    units = (n + align - 1) // align
    if units < world:
        raise ValueError("n = %d positions cannot give each of %d ranks a slab of whole %d-element units"
                         % (n, world, align))
    per, extra = divmod(units, world)
    u0 = rank * per + min(rank, extra)
    u1 = u0 + per + (1 if rank < extra else 0)
    return min(n, u0 * align), min(n, u1 * align)


class SdmdEngine:
    """A rank's slab handle on its GPU: the library calls of steps 1, 2, 4."""

    def __init__(self, n_slab, m, dtype, device, stream=None):
        import torch
        self.h = S.sdmd_create(n_slab, m, dtype)
        self.dtype = dtype
        self.device = device
        self.stream = stream
        self.torch = torch
        self.count = 0
        self.m = m

    def row_dtype(self):
        t = self.torch
        return {S.SDMD_U8: t.int64, S.SDMD_F32: t.float64, S.SDMD_C64: t.complex128}[self.dtype]

    def push(self, x_slab):
        S.sdmd_push(self.h, x_slab, self.stream)
        self.count += 1

    def newest_row(self):
        c = min(self.count, self.m)
        row = self.torch.empty(c, dtype=self.row_dtype(), device=self.device)
        S.sdmd_newest_row(self.h, row, self.stream)
        return row

    def set_newest_row(self, row):
        S.sdmd_set_newest_row(self.h, row, self.stream)

    def close(self):
        if self.h:
            S.sdmd_destroy(self.h)
            self.h = None


class RowSlabStream:
    """One rank's share of a row-slab-split stream.

    engine  object with push(x_slab), newest_row() -> tensor, set_newest_row(t)
    reduce  in-place sum of a tensor over all ranks (e.g.
            torch.distributed.all_reduce); called once per push
    n, world, rank, align  as slab_bounds
    """

    def __init__(self, engine, reduce, n, world, rank, align=16):
        self.engine = engine
        self.reduce = reduce
        self.lo, self.hi = slab_bounds(n, world, rank, align)

    def push(self, x):
        """Push one snapshot: `x` is the whole snapshot (n positions; this
        rank takes its slab) or already the slab (hi - lo positions)."""
        xs = x[self.lo:self.hi] if len(x) != self.hi - self.lo else x
        self.engine.push(xs)
        row = self.engine.newest_row()
        self.reduce(row)
        self.engine.set_newest_row(row)
        return row
