"""Oracle exact DMD of one window, recomputed from scratch (test infrastructure).

Follows Sec. 2.1 (method of snapshots, Eqs. 3-4), Sec. 2.2 (exact DMD,
Eqs. 5-9), Sec. 3.3 (amplitudes from POD coefficients, Eq. 14a-e) and
Algorithms 1-3, in FP64 / complex128 with LAPACK (numpy) doing the
eigendecompositions.

Readings where the paper is silent or ambiguous:

* window: the c resident snapshots W = [x_1 .. x_c]; X = W[:, :-1] and
  X' = W[:, 1:], so at most c-1 DMD eigenvalues (Algorithm 2 passes a window
  one column wider than the one its SVD sees).
* Algorithm 1 sorts sigma without saying that V follows; here V is permuted
  with sigma (descending, stable for ties).
* Algorithm 1's sqrt(abs(.)) is read as sqrt(max(lambda, 0)), and modes whose
  Gram eigenvalue is at or below the FP64 noise floor
  lambda_1 * RANK_RTOL_FACTOR * p * eps are dropped (p = c-1), so that
  Sigma^-1 exists. The requested rank r is clamped to that numerical rank.
* The POD coefficient vector alpha_1 of x_1 is U^H x_1 = Sigma V^H e_1, i.e.
  sigma_i * conj(V[0, i]) (Algorithm 3 writes it with v[:, 0]; that is the same
  vector only under a transposed storage of V).
* Algorithm 3's lstsq on the square W Lambda is a solve.
* Background mode: argmin |log lambda| with the principal complex log
  (Algorithm 3), i.e. the mode with |omega| closest to 0.
* Background column at window column t (t = 0 for x_1): b_idx phi_idx
  lambda_idx^t, the exponent of Algorithm 3's first-step branch; the
  streaming branch's exponent X.shape[1] is one larger for the last column,
  read as an off-by-one.
"""
from dataclasses import dataclass

import numpy as np

from .gram import cross_gram, gram_u8

# Modes whose Gram eigenvalue is <= lambda_1 * RANK_RTOL_FACTOR * p * eps64 are
# treated as numerically zero (eps64 = 2**-52). The GPU path uses the same rule.
RANK_RTOL_FACTOR = 64.0
EPS64 = float(np.finfo(np.float64).eps)


def numerical_rank(lam_desc, p):
    """Number of leading eigenvalues above the FP64 noise floor."""
    lam_desc = np.asarray(lam_desc, dtype=np.float64)
    if lam_desc.size == 0 or not lam_desc[0] > 0.0:
        return 0
    thr = lam_desc[0] * RANK_RTOL_FACTOR * p * EPS64
    k = 0
    while k < lam_desc.size and lam_desc[k] > thr:
        k += 1
    return k


def mos_svd(GX):
    """Method-of-snapshots SVD from the Gram matrix GX = X^H X (Eqs. 3-4).

    Returns (lam, sigma, V, rank): eigenvalues of GX sorted descending with
    the eigenvector columns of V permuted along (Algorithm 1's sort),
    sigma = sqrt(max(lam, 0)), and the numerical rank.
    U = X V Sigma^-1 (Eq. 4) is never formed, as in the paper.
    """
    GX = np.asarray(GX)
    p = GX.shape[0]
    lam, V = np.linalg.eigh(GX)
    order = np.argsort(-lam, kind="stable")
    lam = lam[order]
    V = V[:, order]
    sigma = np.sqrt(np.maximum(lam, 0.0))
    rank = numerical_rank(lam, p)
    return lam, sigma, V, rank


@dataclass
class DMDResult:
    r: int                 # modes kept (<= requested, <= numerical rank)
    rank: int              # numerical rank of X^H X
    sigma: np.ndarray      # (r,) singular values of X, descending
    V: np.ndarray          # (p, r) right singular vectors of X
    vsi: np.ndarray        # (p, r) V Sigma^-1
    Atilde: np.ndarray     # (r, r) projected operator, Eq. 7
    lam: np.ndarray        # (r,) DMD eigenvalues, Eq. 8
    W: np.ndarray          # (r, r) eigenvectors of Atilde (unit 2-norm columns)
    M: np.ndarray          # (p, r) V Sigma^-1 W
    Phi: object            # (n, r) exact DMD modes, Eq. 9 (None from dmd_from_gram)
    lam_all: np.ndarray    # (p,) all eigenvalues of X^H X, descending


def _window_blocks(W, exact_u8):
    """X^H X and X^H X' computed directly from the window (not from G)."""
    X = W[:, :-1]
    Xp = W[:, 1:]
    if exact_u8:
        G = gram_u8(W)                       # exact int64, then exact in FP64
        GX = G[:-1, :-1].astype(np.float64)
        GXY = G[:-1, 1:].astype(np.float64)
        assert np.abs(G).max(initial=0) < 2 ** 53
    else:
        GX = cross_gram(X, X)
        GXY = cross_gram(X, Xp)
    return X, Xp, GX, GXY


def dmd_from_gram(GX, GXY, r):
    """The small-matrix part of exact DMD from the two Gram blocks.

    GX = X^H X and GXY = X^H X' (both p x p). Returns a DMDResult without
    Phi (Phi = None): sigma, V, vsi, A~, lambda, W, M = vsi W.
    Steps, in the order of Algorithms 1-2:
      GX V = V Lambda_G, sort desc, sigma = sqrt      (Eq. 3, Algorithm 1)
      vsi = V_r Sigma_r^-1
      A~ = vsi^H GXY vsi  (= U^H X' V Sigma^-1)       (Eq. 7)
      A~ W = W Lambda                                (Eq. 8)
    Eigenpairs of A~ are ordered by descending |lambda|, then by angle.
    """
    GX = np.asarray(GX)
    GXY = np.asarray(GXY)
    lam_all, sigma_all, V_all, rank = mos_svd(GX)
    rr = int(min(max(r, 0), rank))
    V = V_all[:, :rr]
    s = sigma_all[:rr]
    vsi = V / s[None, :]
    At = vsi.conj().T @ GXY @ vsi
    if rr > 0:
        lam, Wd = np.linalg.eig(At)
        order = np.lexsort((np.angle(lam), -np.abs(lam)))
        lam = lam[order]
        Wd = Wd[:, order]
    else:
        lam = np.zeros(0, dtype=np.complex128)
        Wd = np.zeros((0, 0), dtype=np.complex128)
    M = vsi @ Wd
    return DMDResult(r=rr, rank=rank, sigma=s, V=V, vsi=vsi, Atilde=At,
                     lam=lam.astype(np.complex128), W=Wd.astype(np.complex128),
                     M=M.astype(np.complex128), Phi=None, lam_all=lam_all)


def exact_dmd(W, r):
    """Exact DMD of the window W (n x c, columns oldest to newest), rank <= r.

    GX = X^H X and GXY = X^H X' are computed directly from the window
    (Eqs. 3, 7), then dmd_from_gram, then Phi = X' vsi W (Eq. 9).
    """
    W = np.asarray(W)
    if W.ndim != 2 or W.shape[1] < 2:
        raise ValueError("window needs at least 2 snapshots")
    exact_u8 = W.dtype == np.uint8
    X, Xp, GX, GXY = _window_blocks(W, exact_u8)
    res = dmd_from_gram(GX, GXY, r)
    Xp_f = Xp.astype(np.complex128) if np.iscomplexobj(Xp) else Xp.astype(np.float64)
    res.Phi = (Xp_f @ res.M).astype(np.complex128)
    return res


def pod_amplitudes(res):
    """Mode amplitudes from POD coefficients (Sec. 3.3, Eq. 14a-e).

    x_1 = Phi b with x_1 = U alpha_1 gives alpha_1 = A~ W b = W Lambda b, so
    b = (W Lambda)^-1 alpha_1, with alpha_1 = Sigma V^H e_1.
    """
    alpha1 = res.sigma * np.conj(res.V[0, :])
    WL = res.W * res.lam[None, :]
    return np.linalg.solve(WL, alpha1.astype(np.complex128))


def lstsq_amplitudes(res, x1):
    """The high-dimensional least-squares amplitudes b = Phi^+ x_1 (Eq. 13)."""
    b, *_ = np.linalg.lstsq(res.Phi, np.asarray(x1).astype(np.complex128), rcond=None)
    return b


def background_index(lam):
    """argmin_i |log lambda_i| (Algorithm 3), principal complex log."""
    lam = np.asarray(lam, dtype=np.complex128)
    return int(np.argmin(np.abs(np.log(lam))))


def background_column(res, b, t):
    """l_t = b_idx phi_idx lambda_idx^t for window column t (Eq. 11, Alg. 3)."""
    idx = background_index(res.lam)
    return b[idx] * res.Phi[:, idx] * (res.lam[idx] ** t)


def reconstruct(res, b, t):
    """x_hat(t) = sum_k b_k phi_k lambda_k^t over the kept modes (Sec. 2.2,
    Eq. 11 without the background/foreground split); t = 0 is x_1."""
    return res.Phi @ (b * res.lam ** t)


def foreground_column(W, res, b, t):
    """x_t minus its background (Eq. 11's sparse part, Algorithm 3), where
    W[:, t] is the window column at time index t (t = 0 is x_1)."""
    return np.asarray(W)[:, t].astype(np.float64) - background_column(res, b, t).real


def pod_modes(W, r):
    """POD (left singular) vectors of X = W[:, :-1]: U_r = X V_r Sigma_r^-1
    (Eq. 4), with sigma and V from the method of snapshots (mos_svd of
    X^H X, Algorithm 1); r is clamped to the numerical rank. Returns
    (U, sigma) with U of shape n x r."""
    W = np.asarray(W)
    exact_u8 = W.dtype == np.uint8
    X, _, GX, _ = _window_blocks(W, exact_u8)
    _, sigma, V, rank = mos_svd(GX)
    rr = int(min(max(r, 0), rank))
    Xf = X.astype(np.complex128) if np.iscomplexobj(X) else X.astype(np.float64)
    U = Xf @ (V[:, :rr] / sigma[None, :rr])
    return U, sigma[:rr]


def slow_modes(lam, tol):
    """Indices of the slow modes: |log lambda_k| <= tol with the principal
    log (several background modes instead of the single argmin, Algorithm 3's
    criterion widened to a threshold)."""
    return np.nonzero(np.abs(np.log(np.asarray(lam, dtype=np.complex128))) <= tol)[0]


def slow_background_column(res, b, t, tol):
    """sum over the slow modes of b_k phi_k lambda_k^t (Eq. 11 with the
    low-rank part spanned by every slow mode); t = 0 is x_1."""
    idx = slow_modes(res.lam, tol)
    return res.Phi[:, idx] @ (b[idx] * res.lam[idx] ** t)


def slow_foreground_column(W, res, b, t, tol):
    """x_t minus its slow-mode background (real part)."""
    return np.asarray(W)[:, t].astype(np.float64) - slow_background_column(res, b, t, tol).real


def fourier_dmd(snaps, r):
    """Exact DMD of a window of sparse Fourier-coefficient snapshots
    [(idx, val), ...] (oldest first) without leaving coefficient space
    (Sec. 3.5): G from sparse inner products (Parseval), then the small-matrix
    part of Algorithms 1-2 (dmd_from_gram). Phi is not formed here; its rows
    come from fourier_phi_rows."""
    from .gram import gram_sparse
    G = gram_sparse(snaps)
    return dmd_from_gram(G[:-1, :-1], G[:-1, 1:], r)


def fourier_support(snaps):
    """Sorted union of the supports of X' (snapshots 1 .. c-1): the only
    coefficients where Phi-hat = X'-hat M can be nonzero."""
    return np.unique(np.concatenate([np.asarray(s[0], dtype=np.int64) for s in snaps[1:]]))


def fourier_phi_rows(snaps, M, ks):
    """Rows ks of Phi-hat = X'-hat M (Eq. 9 in coefficient space): row k is
    sum_j xhat_{j+1}[k] M[j, :] over the X' snapshots holding coefficient k."""
    ks = np.asarray(ks, dtype=np.int64)
    out = np.zeros((ks.size, M.shape[1]), dtype=np.complex128)
    for j, (idx, val) in enumerate(snaps[1:]):
        idx = np.asarray(idx, dtype=np.int64)
        pos = np.searchsorted(idx, ks)
        pos = np.minimum(pos, idx.size - 1)
        hit = idx[pos] == ks
        out[hit] += np.asarray(val)[pos[hit]].astype(np.complex128)[:, None] * M[j][None, :]
    return out
