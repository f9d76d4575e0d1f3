"""Pins for the CPU oracle: each check ties an oracle function to something
other than itself (brute-force sums, numpy.linalg.svd / pinv, closed forms,
planted linear systems, Parseval's identity, hand-computed fixtures).

Runs on CPU only (no gpu marker).
"""
import cmath
import math
import os

import numpy as np
import pytest

import oracle
from oracle import dmd as odmd
from paper_1612_07875_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _brute_gram(cols):
    """Python-loop inner products: math.fsum for reals, exact ints for ints."""
    c = len(cols)
    G = [[None] * c for _ in range(c)]
    for i in range(c):
        for j in range(c):
            a, b = cols[i], cols[j]
            if isinstance(a[0], int):
                G[i][j] = sum(x * y for x, y in zip(a, b))
            elif isinstance(a[0], complex):
                re = math.fsum((x.conjugate() * y).real for x, y in zip(a, b))
                im = math.fsum((x.conjugate() * y).imag for x, y in zip(a, b))
                G[i][j] = complex(re, im)
            else:
                G[i][j] = math.fsum(x * y for x, y in zip(a, b))
    return G


# ---------------------------------------------------------------- Gram -----

def test_gram_dense_real_brute_force():
    rng = np.random.default_rng(1)
    W = rng.standard_normal((13, 5))
    G = oracle.gram_dense(W)
    B = _brute_gram([[float(v) for v in W[:, j]] for j in range(5)])
    assert np.allclose(G, np.array(B), rtol=1e-14, atol=1e-13)


def test_gram_dense_complex_brute_force_conjugates_first_argument():
    rng = np.random.default_rng(2)
    W = rng.standard_normal((11, 4)) + 1j * rng.standard_normal((11, 4))
    G = oracle.gram_dense(W)
    B = np.array(_brute_gram([[complex(v) for v in W[:, j]] for j in range(4)]))
    assert np.allclose(G, B, rtol=1e-14, atol=1e-13)
    # <a, b> = a^H b: G[0, 1] conjugates column 0, not column 1
    assert abs(G[0, 1] - np.vdot(W[:, 0], W[:, 1])) < 1e-12
    assert np.allclose(G, G.conj().T)


def test_gram_u8_golden_hand_computed():
    rows = {}
    with open(os.path.join(GOLDEN, "gram_u8_tiny.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = (s.strip() for s in line.split("=", 1))
            rows[k] = v
    frames = [np.array([int(t) for t in rows[k].split()], dtype=np.uint8) for k in ("x1", "x2", "x3")]
    G_expect = np.array([[int(t) for t in r.split()] for r in rows["G"].split(";")], dtype=np.int64)
    W = np.stack(frames, axis=1)
    assert (oracle.gram_u8(W) == G_expect).all()


def test_gram_u8_brute_force_python_ints():
    rng = np.random.default_rng(3)
    W = rng.integers(0, 256, (37, 6), dtype=np.uint8)
    G = oracle.gram_u8(W)
    B = _brute_gram([[int(v) for v in W[:, j]] for j in range(6)])
    assert G.dtype == np.int64
    assert (G == np.array(B, dtype=np.int64)).all()


def test_gram_u8_exact_beyond_int32():
    # 255^2 * 40000 = 2.6e9 > 2^31: an int32 accumulator would wrap.
    n = 40000
    W = np.full((n, 3), 255, dtype=np.uint8)
    W[:, 1] = 254
    W[::2, 2] = 0
    G = oracle.gram_u8(W)
    assert G[0, 0] == 255 * 255 * n
    assert G[0, 1] == 255 * 254 * n
    assert G[2, 2] == 255 * 255 * (n // 2)
    assert G[0, 0] > 2 ** 31


def test_gram_u8_equals_fp64_blas_where_every_partial_sum_is_exact():
    # Every partial sum is an integer < 2^53, so an FP64 BLAS product is exact:
    # an independent route to the same integers.
    rng = np.random.default_rng(4)
    W = rng.integers(0, 256, (200001, 5), dtype=np.uint8)
    G = oracle.gram_u8(W)
    Wf = W.astype(np.float64)
    assert (G == (Wf.T @ Wf).astype(np.int64)).all()
    a, b = W[:, 1], W[:, 3]
    assert oracle.dot_u8(a, b) == int(G[1, 3])


def test_sparse_inner_brute_force_dictionary():
    a_idx = np.array([0, 3, 7, 9, 20], dtype=np.int32)
    a_val = np.array([1 + 1j, 2, -1j, 0.5, 3 - 2j], dtype=np.complex64)
    b_idx = np.array([3, 4, 9, 21], dtype=np.int32)
    b_val = np.array([1j, 5, 2 + 2j, 7], dtype=np.complex64)
    da = dict(zip(a_idx.tolist(), a_val.astype(complex).tolist()))
    db = dict(zip(b_idx.tolist(), b_val.astype(complex).tolist()))
    expect = sum(da[k].conjugate() * db[k] for k in da if k in db)
    got = oracle.sparse_inner(a_idx, a_val, b_idx, b_val)
    assert abs(got - expect) < 1e-12
    assert abs(got - (2 * 1j + 0.5 * (2 + 2j))) < 1e-12
    # disjoint supports give zero; a vector with itself gives its squared norm
    assert oracle.sparse_inner(a_idx, a_val, a_idx + 100, a_val) == 0
    assert abs(oracle.sparse_inner(a_idx, a_val, a_idx, a_val)
               - np.sum(np.abs(a_val.astype(complex)) ** 2)) < 1e-12


def test_parseval_sparse_gram_equals_physical_gram():
    # Sec. 3.5: SVD/DMD are invariant under unitary transforms such as the FFT.
    fs = synth.FourierSparseStream(side=32, nnz=41, churn=0.1, seed=7)
    snaps = [fs.snapshot(t) for t in range(6)]
    Gs = oracle.gram_sparse(snaps)
    phys = np.stack([fs.physical(t) for t in range(6)], axis=1)
    Gd = oracle.gram_dense(phys)
    scale = np.abs(Gd).max()
    assert np.abs(Gs - Gd).max() <= 1e-12 * scale
    # and the supports really differ from snapshot to snapshot (churn)
    assert not np.array_equal(snaps[0][0], snaps[1][0])


def test_gram_invariants_psd_and_cauchy_schwarz():
    rng = np.random.default_rng(5)
    for W in (rng.standard_normal((50, 7)),
              rng.standard_normal((50, 7)) + 1j * rng.standard_normal((50, 7))):
        G = oracle.gram_dense(W)
        assert np.allclose(G, G.conj().T)
        ev = np.linalg.eigvalsh(G)
        assert ev.min() > -1e-10 * ev.max()
        d = np.real(np.diag(G))
        assert (d >= 0).all()
        assert (np.abs(G) ** 2 <= np.outer(d, d) * (1 + 1e-12) + 1e-12).all()


def test_streaming_window_reuses_all_but_one_row_eq12():
    # Eq. 12a-b: the next window's Gram is the previous one shifted up-left by
    # one, plus one new row/column of inner products with the new snapshot.
    rng = np.random.default_rng(6)
    for kind in ("f32", "u8"):
        so = oracle.StreamOracle(n=64, m=5, kind=kind)
        snaps = []
        prev = None
        for t in range(9):
            x = (rng.integers(0, 256, 64, dtype=np.uint8) if kind == "u8"
                 else rng.standard_normal(64).astype(np.float32))
            snaps.append(x)
            so.push(x)
            G = so.gram()
            c = min(t + 1, 5)
            assert G.shape == (c, c)
            win = snaps[-c:]
            for j in range(c):
                ref = (int(np.dot(win[j].astype(np.int64), x.astype(np.int64))) if kind == "u8"
                       else float(np.dot(win[j].astype(np.float64), x.astype(np.float64))))
                assert G[j, c - 1] == pytest.approx(ref, rel=1e-13, abs=1e-12)
            if prev is not None:
                # BLAS may block the FP64 sums differently per shape: equal to
                # rounding for floats, exactly equal for integers
                same = ((lambda a, b: np.array_equal(a, b)) if kind == "u8"
                        else (lambda a, b: np.allclose(a, b, rtol=1e-13, atol=0)))
                if t >= 5:
                    assert same(G[:-1, :-1], prev[1:, 1:])
                else:   # ramp-up: nothing evicted yet
                    assert same(G[:-1, :-1], prev)
            prev = G


# ------------------------------------------------------ method of snapshots -

@pytest.mark.parametrize("cplx", [False, True])
def test_mos_svd_matches_numpy_svd(cplx):
    rng = np.random.default_rng(10 + cplx)
    X = rng.standard_normal((40, 7))
    if cplx:
        X = X + 1j * rng.standard_normal((40, 7))
    lam, sigma, V, rank = oracle.mos_svd(oracle.gram_dense(X))
    U_ref, s_ref, Vh_ref = np.linalg.svd(X, full_matrices=False)
    assert rank == 7
    # sigma agrees to ~eps * sigma_1^2 / sigma_i (the MoS accuracy, cf. Fig. 1)
    tol = 50 * np.finfo(float).eps * s_ref[0] ** 2 / s_ref
    assert (np.abs(sigma - s_ref) <= tol).all()
    assert (np.diff(sigma) <= 0).all()
    # U = X V Sigma^-1 (Eq. 4) reproduces the SVD's left singular vectors
    U = X @ V / sigma
    for k in range(7):
        assert abs(abs(np.vdot(U[:, k], U_ref[:, k])) - 1.0) < 1e-10
    assert np.allclose(U.conj().T @ U, np.eye(7), atol=1e-10)


def test_mos_svd_rank_deficient_window():
    rng = np.random.default_rng(12)
    B = rng.standard_normal((30, 3))
    X = B @ rng.standard_normal((3, 8))        # rank 3
    lam, sigma, V, rank = oracle.mos_svd(oracle.gram_dense(X))
    assert rank == 3
    res = oracle.exact_dmd(np.concatenate([X, X[:, :1]], axis=1), r=8)
    assert res.r <= 3


# ------------------------------------------------------------ exact DMD ---

def test_exact_dmd_scalar_closed_form():
    # x_k = lam^k u: X has rank 1, sigma_1 = |u| sqrt(sum_k lam^2k),
    # the single DMD eigenvalue is lam and Phi is parallel to u.
    lam0 = 0.9
    rng = np.random.default_rng(20)
    u = rng.standard_normal(25)
    c = 6
    W = np.stack([lam0 ** k * u for k in range(c)], axis=1)
    res = oracle.exact_dmd(W, r=4)
    assert res.r == 1
    s1 = np.linalg.norm(u) * math.sqrt(sum(lam0 ** (2 * k) for k in range(c - 1)))
    assert abs(res.sigma[0] - s1) < 1e-12 * s1
    assert abs(res.lam[0] - lam0) < 1e-13
    phi = res.Phi[:, 0]
    assert abs(abs(np.vdot(phi, u)) / (np.linalg.norm(phi) * np.linalg.norm(u)) - 1) < 1e-13


def test_exact_dmd_rotation_closed_form():
    # x_k = Q R(theta)^k x0 in a 2-D subspace: eigenvalues exp(+-i theta).
    theta = 0.7
    rng = np.random.default_rng(21)
    Q, _ = np.linalg.qr(rng.standard_normal((30, 2)))
    R = np.array([[math.cos(theta), -math.sin(theta)], [math.sin(theta), math.cos(theta)]])
    z = np.array([1.0, 0.3])
    cols = []
    for _ in range(8):
        cols.append(Q @ z)
        z = R @ z
    res = oracle.exact_dmd(np.stack(cols, axis=1), r=5)
    assert res.r == 2
    want = sorted([cmath.exp(1j * theta), cmath.exp(-1j * theta)], key=lambda v: v.imag)
    got = sorted(res.lam.tolist(), key=lambda v: v.imag)
    assert all(abs(a - b) < 1e-12 for a, b in zip(got, want))


def test_exact_dmd_planted_linear_system_noise_free():
    ps = synth.PlantedStream(side=16, noise_var=0.0, seed=30)
    W = np.stack([ps.snapshot(t).astype(np.float64) for t in range(12)], axis=1)
    # regenerate in FP64 to keep the system exactly linear
    F = ps.fields
    W = np.zeros((ps.n, 12))
    for t in range(12):
        for p in range(ps.n_pairs):
            zz = ps.c_pairs[p] * ps.lam_pairs[p] ** t
            W[:, t] += zz.real * F[:, 2 * p] + zz.imag * F[:, 2 * p + 1]
        W[:, t] += ps.c_real[0] * ps.lam_real[0] ** t * F[:, 4]
    res = oracle.exact_dmd(W, r=10)
    assert res.r == 5
    planted = ps.planted_lambdas()
    for lp in planted:
        assert np.min(np.abs(res.lam - lp)) < 1e-10
    modes = ps.planted_modes()
    for k in range(5):
        j = int(np.argmin(np.abs(planted - res.lam[k])))
        a, b = res.Phi[:, k], modes[:, j]
        cosang = abs(np.vdot(a, b)) / (np.linalg.norm(a) * np.linalg.norm(b))
        assert cosang > 1 - 1e-10


def test_exact_dmd_eigs_equal_full_operator_eigs_and_phi_are_eigenvectors():
    # Eq. 6-9: A = X' X^+ ; A~ has A's nonzero eigenvalues and exact DMD
    # modes satisfy A Phi = Phi Lambda.
    rng = np.random.default_rng(40)
    W = rng.standard_normal((10, 7))
    X, Xp = W[:, :-1], W[:, 1:]
    A = Xp @ np.linalg.pinv(X)
    evA = np.linalg.eigvals(A)
    evA = evA[np.abs(evA) > 1e-8]
    res = oracle.exact_dmd(W, r=6)
    assert res.r == 6
    assert len(evA) == 6
    for lam in res.lam:
        assert np.min(np.abs(evA - lam)) < 1e-9
    assert np.allclose(A @ res.Phi, res.Phi * res.lam[None, :], atol=1e-9)


def test_exact_dmd_complex_window():
    rng = np.random.default_rng(41)
    W = rng.standard_normal((12, 6)) + 1j * rng.standard_normal((12, 6))
    X, Xp = W[:, :-1], W[:, 1:]
    A = Xp @ np.linalg.pinv(X)
    res = oracle.exact_dmd(W, r=5)
    assert np.allclose(A @ res.Phi, res.Phi * res.lam[None, :], atol=1e-9)


def test_u8_window_dmd_equals_float_window_dmd():
    rng = np.random.default_rng(42)
    W = rng.integers(0, 256, (300, 9), dtype=np.uint8)
    r8 = oracle.exact_dmd(W, r=6)
    rf = oracle.exact_dmd(W.astype(np.float64), r=6)
    assert np.allclose(r8.lam, rf.lam, atol=1e-10)
    assert np.allclose(r8.sigma, rf.sigma, rtol=1e-12)


# ---------------------------------------------------- amplitudes / Alg. 3 --

def test_pod_amplitudes_equal_least_squares_and_reconstruct():
    # Sec. 3.3: b from POD coefficients equals b = Phi^+ x_1 (Eq. 13) when the
    # data are exactly linear, and Phi Lambda^k b reproduces x_{k+1}.
    theta = 0.4
    rng = np.random.default_rng(50)
    Q, _ = np.linalg.qr(rng.standard_normal((40, 3)))
    z = np.array([1.0, -0.5, 2.0])
    Rm = np.array([[math.cos(theta), -math.sin(theta), 0],
                   [math.sin(theta), math.cos(theta), 0], [0, 0, 0.97]])
    cols = []
    for _ in range(9):
        cols.append(Q @ z)
        z = Rm @ z
    W = np.stack(cols, axis=1)
    res = oracle.exact_dmd(W, r=3)
    b_pod = oracle.pod_amplitudes(res)
    b_ls = oracle.lstsq_amplitudes(res, W[:, 0])
    assert np.allclose(b_pod, b_ls, atol=1e-10)
    for k in range(8):
        rec = res.Phi @ (b_pod * res.lam ** k)
        assert np.allclose(rec, W[:, k], atol=1e-9)
    # background: the slowest mode is the |lambda| = 0.97 real one
    idx = oracle.background_index(res.lam)
    assert abs(res.lam[idx] - 0.97) < 1e-10
    l5 = oracle.background_column(res, b_pod, 5)
    assert np.allclose(l5, b_pod[idx] * res.Phi[:, idx] * 0.97 ** 5)


def _planted_rotation_window(steps, static=None, seed=50):
    # x_k = B + Q R^k z: a rotation by theta (|lambda| = 1) and a decay 0.97
    theta = 0.4
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((40, 4)))
    z = np.array([1.0, -0.5, 2.0])
    Rm = np.array([[math.cos(theta), -math.sin(theta), 0],
                   [math.sin(theta), math.cos(theta), 0], [0, 0, 0.97]])
    B = np.zeros(40) if static is None else static * Q[:, 3]
    cols = []
    for _ in range(steps):
        cols.append(B + Q[:, :3] @ z)
        z = Rm @ z
    return np.stack(cols, axis=1), B


def test_reconstruct_reproduces_window_and_extrapolates_planted_dynamics():
    # Eq. 11 with every mode: x_hat(t) = x_{t+1} inside the window (t = 0 is
    # x_1), and beyond it the planted dynamics continue (exactly linear data).
    W_all, _ = _planted_rotation_window(12)
    W = W_all[:, :9]
    res = oracle.exact_dmd(W, r=3)
    b = oracle.pod_amplitudes(res)
    for t in range(12):
        assert np.allclose(oracle.reconstruct(res, b, t).real, W_all[:, t], atol=1e-9)
        assert np.abs(oracle.reconstruct(res, b, t).imag).max() < 1e-9


def test_background_and_foreground_of_planted_static_scene():
    # A static part B is the lambda = 1 mode: Algorithm 3's background column
    # is B at every t and the foreground is the dynamic part x_t - B.
    W, B = _planted_rotation_window(10, static=3.0, seed=51)
    res = oracle.exact_dmd(W, r=4)
    b = oracle.pod_amplitudes(res)
    idx = oracle.background_index(res.lam)
    assert abs(res.lam[idx] - 1.0) < 1e-10
    for t in (0, 4, 9):
        assert np.allclose(oracle.background_column(res, b, t).real, B, atol=1e-9)
        assert np.allclose(oracle.foreground_column(W, res, b, t), W[:, t] - B, atol=1e-9)


def test_slow_modes_background_is_the_planted_slow_part():
    # Planted scene: static B (lambda = 1), a rotation (|log lambda| = 0.4)
    # and a decay (lambda = 0.97, |log lambda| = 0.030). Slow modes with
    # tol = 0.1 are the static and the decaying ones: their background is
    # B + the decaying component, known in closed form; tol below 0.03 leaves
    # the single background mode, tol above 0.4 every mode (the window).
    W, B = _planted_rotation_window(10, static=3.0, seed=51)
    rng = np.random.default_rng(51)
    Q, _ = np.linalg.qr(rng.standard_normal((40, 4)))
    res = oracle.exact_dmd(W, r=4)
    b = oracle.pod_amplitudes(res)
    assert sorted(oracle.slow_modes(res.lam, 0.1).tolist()) == sorted(
        [int(np.argmin(np.abs(res.lam - 1.0))), int(np.argmin(np.abs(res.lam - 0.97)))])
    for t in (0, 3, 9):
        decay = Q[:, 2] * 2.0 * 0.97 ** t
        assert np.allclose(oracle.slow_background_column(res, b, t, 0.1).real, B + decay, atol=1e-9)
        assert np.allclose(oracle.slow_foreground_column(W, res, b, t, 0.1), W[:, t] - B - decay, atol=1e-9)
        assert np.allclose(oracle.slow_background_column(res, b, t, 0.01), oracle.background_column(res, b, t),
                           atol=1e-12)
        assert np.allclose(oracle.slow_background_column(res, b, t, 0.5).real, W[:, t], atol=1e-9)


def test_pod_modes_are_the_left_singular_vectors():
    # U = X V Sigma^-1 (Eq. 4) against numpy's SVD of X: same sigma, columns
    # equal up to sign, orthonormal; X (not X') is the operand.
    rng = np.random.default_rng(70)
    W = rng.standard_normal((30, 8)) * np.array([5, 4, 3, 2.5, 2, 1.5, 1, 0.5])[None, :]
    U, sigma = oracle.pod_modes(W, 5)
    Us, ss, _ = np.linalg.svd(W[:, :-1], full_matrices=False)
    assert np.allclose(sigma, ss[:5], rtol=1e-12)
    for k in range(5):
        assert abs(abs(U[:, k] @ Us[:, k]) - 1.0) < 1e-10
    assert np.allclose(U.T @ U, np.eye(5), atol=1e-10)
    Uu, _ = oracle.pod_modes(rng.integers(0, 256, (50, 6), dtype=np.uint8), 3)   # exact-u8 Gram route
    assert np.allclose(Uu.T @ Uu, np.eye(3), atol=1e-9)


def test_fourier_domain_dmd_equals_physical_dmd():
    # DMD in coefficient space (Sec. 3.5): the orthonormal transform leaves G,
    # and so lambda and M, unchanged (Parseval), and Phi-hat maps to the
    # physical-space modes by the inverse transform: Phi = ifft2(Phi-hat).
    fs = synth.FourierSparseStream(side=16, nnz=40, churn=0.1, seed=5)
    c, r = 9, 5
    snaps = [fs.snapshot(t) for t in range(c)]
    res_f = oracle.fourier_dmd(snaps, r)
    Wp = np.stack([fs.physical(t) for t in range(c)], axis=1)
    res_p = oracle.exact_dmd(Wp, r)
    assert res_f.r == res_p.r == r
    assert np.abs(res_f.lam - res_p.lam).max() < 1e-10
    sup = oracle.fourier_support(snaps)
    rows = oracle.fourier_phi_rows(snaps, res_f.M, sup)
    Phi_hat = np.zeros((fs.N, r), dtype=np.complex128)
    Phi_hat[sup] = rows
    dense_hat = np.stack([fs.dense_coeffs(t) for t in range(1, c)], axis=1) @ res_f.M
    assert np.allclose(Phi_hat, dense_hat, atol=1e-12)               # zero off the support
    Phi_phys = np.stack([np.fft.ifft2(Phi_hat[:, k].reshape(16, 16), norm="ortho").reshape(-1)
                         for k in range(r)], axis=1)
    for k in range(r):                                                # same columns up to phase
        a, b = Phi_phys[:, k], res_p.Phi[:, k]
        ph = np.vdot(a, b) / abs(np.vdot(a, b))
        assert np.linalg.norm(a * ph - b) <= 1e-8 * np.linalg.norm(b)


def test_background_index_principal_log():
    lam = np.array([0.5, 1.0001 * cmath.exp(0.001j), 0.9 * cmath.exp(2j), -1.0])
    # |log(-1)| = pi: a unit-modulus but fast mode is not background
    assert oracle.background_index(lam) == 1


# -------------------------------------------- mutations the pins must catch --

def test_pins_catch_wrong_phi_operand(monkeypatch):
    # Planting Phi = X vsi W (X instead of X') must break A Phi = Phi Lambda.
    rng = np.random.default_rng(60)
    W = rng.standard_normal((10, 7))
    X, Xp = W[:, :-1], W[:, 1:]
    A = Xp @ np.linalg.pinv(X)
    res = oracle.exact_dmd(W, r=6)
    bad_phi = X @ res.M
    assert not np.allclose(A @ bad_phi, bad_phi * res.lam[None, :], atol=1e-6)


def test_pins_catch_unpermuted_eigenvectors(monkeypatch):
    # If V were not permuted along with the sorted sigma, U = X V Sigma^-1
    # would not be orthonormal.
    real_eigh = np.linalg.eigh

    def eigh_then_unsorted(G):
        lam, V = real_eigh(G)
        return lam, V[:, ::-1]  # planted mistake: vectors in the wrong order

    rng = np.random.default_rng(61)
    X = rng.standard_normal((40, 6))
    monkeypatch.setattr(odmd.np.linalg, "eigh", eigh_then_unsorted)
    lam, sigma, V, rank = oracle.mos_svd(oracle.gram_dense(X))
    monkeypatch.undo()
    U = X @ V / sigma
    assert not np.allclose(U.conj().T @ U, np.eye(6), atol=1e-6)


def test_pins_catch_wrong_atilde_block(monkeypatch):
    # A~ built from X^H X instead of X^H X' must miss A's eigenvalues.
    rng = np.random.default_rng(62)
    W = rng.standard_normal((10, 7))
    X, Xp = W[:, :-1], W[:, 1:]
    evA = np.linalg.eigvals(Xp @ np.linalg.pinv(X))
    evA = evA[np.abs(evA) > 1e-8]
    real_cross = odmd.cross_gram

    def swapped(A, B):
        return real_cross(A, A)   # planted mistake

    monkeypatch.setattr(odmd, "cross_gram", swapped)
    res = oracle.exact_dmd(W, r=6)
    monkeypatch.undo()
    miss = max(np.min(np.abs(evA - lam)) for lam in res.lam)
    assert miss > 1e-3


# --------------------------------------- pins of the building blocks -------

def test_cross_gram_brute_force_conjugates_first_operand():
    # A^H B entry (i, j) = sum_k conj(A_ki) B_kj: a missing conjugate or a
    # transposed operand fails (A and B differ in column count on purpose)
    rng = np.random.default_rng(71)
    A = rng.standard_normal((9, 3)) + 1j * rng.standard_normal((9, 3))
    B = rng.standard_normal((9, 4)) + 1j * rng.standard_normal((9, 4))
    C = oracle.cross_gram(A, B)
    assert C.shape == (3, 4)
    for i in range(3):
        for j in range(4):
            re = math.fsum((A[k, i].conjugate() * B[k, j]).real for k in range(9))
            im = math.fsum((A[k, i].conjugate() * B[k, j]).imag for k in range(9))
            assert abs(C[i, j] - complex(re, im)) <= 1e-13
    Ar, Br = A.real, B.real
    Cr = oracle.cross_gram(Ar, Br)
    for i in range(3):
        for j in range(4):
            assert Cr[i, j] == pytest.approx(math.fsum(Ar[k, i] * Br[k, j] for k in range(9)), abs=1e-13)


def test_gram_u8_cols_brute_force_python_ints():
    rng = np.random.default_rng(72)
    cols = [rng.integers(0, 256, 301, dtype=np.uint8) for _ in range(5)]
    cols[2][:] = 255                                   # the largest products
    G = oracle.gram_u8_cols(cols)
    ref = _brute_gram([[int(v) for v in c] for c in cols])
    assert [[int(x) for x in row] for row in G] == ref


def test_densify_sparse_round_trip_and_parseval_inner():
    rng = np.random.default_rng(73)
    n = 50
    ia = np.sort(rng.choice(n, 12, replace=False)).astype(np.int32)
    ib = np.sort(rng.choice(n, 15, replace=False)).astype(np.int32)
    va = (rng.standard_normal(12) + 1j * rng.standard_normal(12)).astype(np.complex64)
    vb = (rng.standard_normal(15) + 1j * rng.standard_normal(15)).astype(np.complex64)
    da = oracle.densify_sparse(ia, va, n)
    assert da.shape == (n,) and da.dtype == np.complex128
    assert np.array_equal(da[ia], va.astype(np.complex128))
    mask = np.ones(n, bool)
    mask[ia] = False
    assert not da[mask].any()
    db = oracle.densify_sparse(ib, vb, n)
    assert abs(oracle.sparse_inner(ia, va, ib, vb) - np.vdot(da, db)) <= 1e-12


def test_numerical_rank_threshold_hand_built():
    # rule: lambda_k > lambda_1 * 64 * p * eps64, strictly
    p = 10
    thr = 1.0 * odmd.RANK_RTOL_FACTOR * p * odmd.EPS64
    assert oracle.numerical_rank([1.0, 1e-3, 1e-16], p) == 2
    assert oracle.numerical_rank([1.0, thr * 1.0000001, thr * 0.5], p) == 2
    assert oracle.numerical_rank([1.0, thr, 0.0], p) == 1          # at the threshold: dropped
    assert oracle.numerical_rank([2.0, 1.0, 0.5], p) == 3
    assert oracle.numerical_rank([0.0, 0.0], p) == 0
    assert oracle.numerical_rank([-1.0, -2.0], p) == 0
    assert oracle.numerical_rank([], p) == 0


def test_dmd_from_gram_planted_system_from_gram_blocks_only():
    # the small-matrix part given only G_X = X^T X and G_XY = X^T X' of a
    # planted noise-free linear system recovers the planted eigenvalues and,
    # through X' M, the modes; the transposed cross block (X'^T X) gives
    # A~ transposed: the same eigenvalues but left eigenvectors, so modes that
    # are not the planted ones
    ps = synth.PlantedStream(side=16, noise_var=0.0, seed=31)
    F = ps.fields
    W = np.zeros((ps.n, 12))
    for t in range(12):
        for q in range(ps.n_pairs):
            zz = ps.c_pairs[q] * ps.lam_pairs[q] ** t
            W[:, t] += zz.real * F[:, 2 * q] + zz.imag * F[:, 2 * q + 1]
        W[:, t] += ps.c_real[0] * ps.lam_real[0] ** t * F[:, 4]
    X, Xp = W[:, :-1], W[:, 1:]
    GX = X.T @ X
    GXY = X.T @ Xp
    res = oracle.dmd_from_gram(GX, GXY, 10)
    assert res.r == 5 and res.Phi is None
    planted = ps.planted_lambdas()
    for lp in planted:
        assert np.min(np.abs(res.lam - lp)) < 1e-10
    # M = vsi W maps X' to the modes: X' M equals exact_dmd's Phi
    ref = oracle.exact_dmd(W, 10)
    assert np.allclose(Xp @ res.M, ref.Phi, rtol=0, atol=1e-10 * np.abs(ref.Phi).max())
    modes = ps.planted_modes()

    def worst_cos(res_):
        Phi = Xp @ res_.M
        worst = 1.0
        for k in range(res_.r):
            j = int(np.argmin(np.abs(planted - res_.lam[k])))
            a, b = Phi[:, k], modes[:, j]
            worst = min(worst, abs(np.vdot(a, b)) / (np.linalg.norm(a) * np.linalg.norm(b)))
        return worst

    assert worst_cos(res) > 1 - 1e-10
    wrong = oracle.dmd_from_gram(GX, GXY.T, 10)
    assert worst_cos(wrong) < 1 - 1e-6
