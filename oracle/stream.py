"""Streaming window oracle: recomputes everything from the window each step.

Test infrastructure only. It holds the last m snapshots in time order
(oldest first) and, on request, evaluates the plain definitions of
oracle.gram and oracle.dmd on that window. Before m snapshots have arrived
the window holds all of them (the ramp-up reading of Sec. 5: start with the
columns available, append without eviction until the window is full).
"""
from collections import deque

import numpy as np

from .dmd import exact_dmd
from .gram import gram_dense, gram_sparse, gram_u8_cols


class StreamOracle:
    """kind: 'f32' (dense float), 'u8' (8-bit pixels) or 'sparse' (idx, val)."""

    def __init__(self, n, m, kind):
        if kind not in ("f32", "u8", "sparse"):
            raise ValueError(kind)
        self.n = int(n)
        self.m = int(m)
        self.kind = kind
        self.win = deque(maxlen=self.m)
        self.count = 0

    def push(self, x):
        if self.kind == "sparse":
            idx, val = x
            self.win.append((np.array(idx, copy=True), np.array(val, copy=True)))
        else:
            x = np.array(x, copy=True).reshape(-1)
            if x.size != self.n:
                raise ValueError("snapshot length")
            self.win.append(x)
        self.count += 1

    def window(self):
        """n x c matrix of the resident snapshots, oldest first (dense kinds)."""
        if self.kind == "sparse":
            raise TypeError("sparse window has no dense matrix; use snapshots()")
        return np.stack(list(self.win), axis=1)

    def snapshots(self):
        return list(self.win)

    def gram(self):
        """Time-ordered Gram of the window: float64, int64 (u8) or complex128."""
        if self.kind == "u8":
            return gram_u8_cols(list(self.win))
        if self.kind == "sparse":
            return gram_sparse(list(self.win))
        return gram_dense(self.window())

    def modes(self, r):
        if self.kind == "sparse":
            raise NotImplementedError("dense window only")
        return exact_dmd(self.window(), r)
