"""Oracle inner products and Gram matrices (test infrastructure only).

Sec. 2.1 (Eq. 3) builds the method of snapshots on the inner-product matrix
X*X of the snapshot window; Sec. 3.1 (Eq. 12a-b) observes that the streaming
window's X*X shares every entry but one row/column with the previous step.
The oracle ignores that reuse on purpose: it evaluates the plain definition
from the whole window at every step, so it shares no logic with the shift.

Inner-product convention: <a, b> = a^H b (the first argument conjugated), so
G = W^H W is Hermitian; for real data this is W^T W as in Algorithm 1.
"""
import numpy as np

from . import native


def gram_dense(W):
    """G = W^H W of an n x c window, FP64 (complex128 for complex data).

    A library matmul serves as the sum; accumulation is in FP64 regardless of
    the storage type of W.
    """
    W = np.asarray(W)
    if np.iscomplexobj(W):
        Wd = W.astype(np.complex128)
        return Wd.conj().T @ Wd
    Wd = W.astype(np.float64)
    return Wd.T @ Wd


def cross_gram(A, B):
    """A^H B in FP64 / complex128 (the X^H X' block of Algorithm 2)."""
    A = np.asarray(A)
    B = np.asarray(B)
    if np.iscomplexobj(A) or np.iscomplexobj(B):
        return A.astype(np.complex128).conj().T @ B.astype(np.complex128)
    return A.astype(np.float64).T @ B.astype(np.float64)


def gram_u8(W):
    """Exact int64 Gram of an n x c uint8 window (columns are snapshots)."""
    W = np.asarray(W, dtype=np.uint8)
    cols = [np.ascontiguousarray(W[:, j]) for j in range(W.shape[1])]
    return native.gram_u8_cols(cols)


def gram_u8_cols(cols):
    """Exact int64 Gram of a list of uint8 snapshots (avoids forming W)."""
    return native.gram_u8_cols(cols)


def dot_u8(a, b):
    """Exact int64 <a, b> of two uint8 snapshots."""
    return native.dot_u8(a, b)


def sparse_inner(idx_a, val_a, idx_b, val_b):
    """<a, b> = sum over the indices present in both of conj(a_k) * b_k.

    Snapshots are stored as (sorted unique int indices, complex values), the
    coefficients of an orthonormal transform (Sec. 3.5): by Parseval's identity
    this equals the inner product of the physical fields. Indices present in
    only one snapshot multiply a zero and drop out. The shared index set comes
    from numpy's sorted intersection; the sum is complex128.
    """
    idx_a = np.asarray(idx_a)
    idx_b = np.asarray(idx_b)
    _, ia, ib = np.intersect1d(idx_a, idx_b, assume_unique=True, return_indices=True)
    a = np.asarray(val_a)[ia].astype(np.complex128)
    b = np.asarray(val_b)[ib].astype(np.complex128)
    return complex(np.sum(np.conj(a) * b))


def gram_sparse(snaps):
    """Hermitian complex128 Gram of sparse snapshots [(idx, val), ...]."""
    c = len(snaps)
    G = np.zeros((c, c), dtype=np.complex128)
    for i in range(c):
        for j in range(i, c):
            g = sparse_inner(snaps[i][0], snaps[i][1], snaps[j][0], snaps[j][1])
            G[i, j] = g
            G[j, i] = np.conj(g)
    return G


def densify_sparse(idx, val, n):
    """Dense complex128 coefficient vector of length n from (idx, val)."""
    out = np.zeros(n, dtype=np.complex128)
    out[np.asarray(idx)] = np.asarray(val).astype(np.complex128)
    return out
