"""Comparison helpers for parity tests (no method arithmetic)."""
import numpy as np


def rel_fro(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def match_eigs(got, ref):
    """Greedy nearest-neighbour matching of two eigenvalue multisets.

    Returns (max abs error, permutation p with got[i] ~ ref[p[i]])."""
    got = np.asarray(got, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    free = list(range(ref.size))
    perm = []
    err = 0.0
    for g in got:
        j = min(free, key=lambda k: abs(g - ref[k]))
        err = max(err, abs(g - ref[j]))
        perm.append(j)
        free.remove(j)
    return err, perm


def normalize_cols(P):
    """Columns scaled to unit 2-norm with the largest-modulus entry real > 0."""
    P = np.asarray(P, dtype=np.complex128).copy()
    for k in range(P.shape[1]):
        col = P[:, k]
        nrm = np.linalg.norm(col)
        if nrm == 0:
            continue
        i = int(np.argmax(np.abs(col)))
        ph = col[i] / abs(col[i])
        P[:, k] = col / (ph * nrm)
    return P


def col_cos(a, b):
    """|<a, b>| / (|a| |b|) column by column."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    num = np.abs(np.sum(np.conj(a) * b, axis=0))
    den = np.linalg.norm(a, axis=0) * np.linalg.norm(b, axis=0)
    return num / np.where(den > 0, den, 1.0)
