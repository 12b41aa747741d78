"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: a library routine the
operation reduces to (numpy's FFT and SVD), a closed form, a theorem of the paper, an
invariant, or brute force on tiny inputs.  A plausible mistake in the oracle (a dropped
term, a wrong sign or index, a transposed operand, a missing conjugate pairing, a wrong
dual scaling) fails at least one of them.
"""
import numpy as np
import pytest

from helpers import bcirc, lowrank_fourier, relerr, rse_db, svt_matrix

import oracle
from paper_1407_1785_gb300 import synth

pytestmark = pytest.mark.usefixtures("oracle_lib")


def _rng(seed=0):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- DFT (Sec. 2.1, Algorithm 1)

@pytest.mark.parametrize("shape", [(3, 4, 1), (3, 4, 2), (2, 3, 7), (4, 2, 8), (2, 2, 3, 4),
                                   (3, 2, 5, 3), (2, 3, 2, 3, 4), (2, 2, 3, 2, 2, 3)])
def test_dft_matches_numpy_fft(shape):
    x = _rng(1).standard_normal(shape)
    axes = tuple(range(2, len(shape)))
    assert np.allclose(oracle.dft(x), np.fft.fftn(x, axes=axes), atol=1e-12)
    X = oracle.dft(x)
    assert np.allclose(oracle.idft(X), x, atol=1e-13)


def test_dft_closed_forms():
    n = 9
    delta = np.zeros((1, 1, n))
    delta[0, 0, 0] = 1.0
    assert np.allclose(oracle.dft(delta), np.ones((1, 1, n)), atol=1e-15)
    const = np.full((1, 1, n), 2.5)
    D = oracle.dft(const)
    assert abs(D[0, 0, 0] - n * 2.5) < 1e-12
    assert np.abs(D[0, 0, 1:]).max() < 1e-12
    shifted = np.zeros((1, 1, n))
    shifted[0, 0, 2] = 1.0          # delta at t = 2: X[k] = exp(-2 pi i 2k / n)
    k = np.arange(n)
    assert np.allclose(oracle.dft(shifted)[0, 0], np.exp(-2j * np.pi * 2 * k / n), atol=1e-14)


@pytest.mark.parametrize("n3", [5, 6])
def test_dft_conjugate_symmetry_of_real_input(n3):
    X = oracle.dft(_rng(2).standard_normal((3, 2, n3)))
    for k in range(1, n3):
        assert np.allclose(X[:, :, n3 - k], np.conj(X[:, :, k]), atol=1e-13)
    assert np.abs(X[:, :, 0].imag).max() < 1e-13


# ---------------------------------------------------------------- matrix SVD (Algorithm 1)

@pytest.mark.parametrize("m,n", [(5, 3), (3, 5), (4, 4), (1, 4), (6, 1)])
def test_svd_matches_numpy(m, n):
    r = _rng(3)
    A = r.standard_normal((m, n)) + 1j * r.standard_normal((m, n))
    U, s, V = oracle.svd(A)
    assert np.allclose(s, np.linalg.svd(A, compute_uv=False), atol=1e-13)
    assert np.allclose(U.conj().T @ U, np.eye(m), atol=1e-13)
    assert np.allclose(V.conj().T @ V, np.eye(n), atol=1e-13)
    k = min(m, n)
    assert np.allclose((U[:, :k] * s) @ V[:, :k].conj().T, A, atol=1e-13)
    assert np.all(np.diff(s) <= 1e-15)


def test_svd_rank_deficient_and_real():
    r = _rng(4)
    A = r.standard_normal((6, 2)) @ r.standard_normal((2, 5))   # rank 2, real
    U, s, V = oracle.svd(A)
    assert np.allclose(s, np.linalg.svd(A, compute_uv=False), atol=1e-12)
    assert s[2:].max() < 1e-12
    assert np.abs(U.imag).max() == 0 and np.abs(V.imag).max() == 0
    assert np.allclose(U.T @ U, np.eye(6), atol=1e-12)
    assert np.allclose(V.T @ V, np.eye(5), atol=1e-12)
    assert np.allclose((U[:, :5] * s) @ V.T, A, atol=1e-12)


# ---------------------------------------------------------------- tensor algebra (Sec. 2.1)

def _tproduct_bruteforce(A, B):
    """Def. 2.1.1 literally: C(i,j,:) = sum_k A(i,k,:) o B(k,j,:), o = circular convolution."""
    n1, n2, n3 = A.shape
    n4 = B.shape[1]
    C = np.zeros((n1, n4, n3))
    for i in range(n1):
        for j in range(n4):
            for k in range(n2):
                a, b = A[i, k, :], B[k, j, :]
                for t in range(n3):
                    C[i, j, t] += sum(a[s] * b[(t - s) % n3] for s in range(n3))
    return C


@pytest.mark.parametrize("n3", [1, 2, 5])
def test_tproduct_equals_circular_convolution(n3):
    r = _rng(5)
    A = r.standard_normal((3, 4, n3))
    B = r.standard_normal((4, 2, n3))
    assert np.allclose(oracle.tproduct(A, B), _tproduct_bruteforce(A, B), atol=1e-12)
    # the generator's t-product follows the same definition
    assert np.allclose(synth.circular_tproduct(A, B), _tproduct_bruteforce(A, B), atol=1e-12)


def test_transpose_and_identity():
    r = _rng(6)
    A = r.standard_normal((3, 4, 5))
    B = r.standard_normal((4, 2, 5))
    lhs = oracle.ttranspose(oracle.tproduct(A, B))
    rhs = oracle.tproduct(oracle.ttranspose(B), oracle.ttranspose(A))
    assert np.allclose(lhs, rhs, atol=1e-12)             # (A*B)^T = B^T * A^T
    I = np.zeros((3, 3, 5))
    I[:, :, 0] = np.eye(3)                               # Def. 2.1.3
    assert np.allclose(oracle.tproduct(I, A), A, atol=1e-12)
    assert np.allclose(oracle.ttranspose(oracle.ttranspose(A)), A)


def _tproduct_bruteforce_nd(A, B):
    """Order-N t-product by its definition as a circular convolution of the tubes over every
    mode from 3 on: C(i, j, t) = sum_l sum_s A(i, l, s) B(l, j, (t - s) mod dims)."""
    modes = A.shape[2:]
    C = np.zeros((A.shape[0], B.shape[1]) + modes)
    for t in np.ndindex(*modes):
        for s_ in np.ndindex(*modes):
            d = tuple((a - b) % n for a, b, n in zip(t, s_, modes))
            C[(slice(None), slice(None)) + t] += (A[(slice(None), slice(None)) + s_]
                                                  @ B[(slice(None), slice(None)) + d])
    return C


@pytest.mark.parametrize("modes", [(2, 3), (3, 2, 2), (2, 2, 1, 3)])
def test_tproduct_order_4_to_6_is_circular_convolution(modes):
    r = _rng(8)
    A = r.standard_normal((3, 2) + modes)
    B = r.standard_normal((2, 4) + modes)
    assert np.allclose(oracle.tproduct(A, B), _tproduct_bruteforce_nd(A, B), atol=1e-12)


@pytest.mark.parametrize("modes", [(3, 4), (2, 3, 2), (2, 2, 3, 2)])
def test_transpose_and_identity_order_4_to_6(modes):
    """(A*B)^T = B^T * A^T, I * A = A, (A^T)^T = A, and the transpose is the conjugate
    transpose of every Fourier slice."""
    r = _rng(9)
    A = r.standard_normal((3, 4) + modes)
    B = r.standard_normal((4, 2) + modes)
    lhs = oracle.ttranspose(oracle.tproduct(A, B))
    rhs = oracle.tproduct(oracle.ttranspose(B), oracle.ttranspose(A))
    assert np.allclose(lhs, rhs, atol=1e-12)
    I = np.zeros((3, 3) + modes)
    I[(slice(None), slice(None)) + (0,) * len(modes)] = np.eye(3)
    assert np.allclose(oracle.tproduct(I, A), A, atol=1e-12)
    assert np.allclose(oracle.ttranspose(oracle.ttranspose(A)), A)
    axes = tuple(range(2, A.ndim))
    Ah, ATh = np.fft.fftn(A, axes=axes), np.fft.fftn(oracle.ttranspose(A), axes=axes)
    assert np.allclose(ATh, np.conj(np.swapaxes(Ah, 0, 1)), atol=1e-12)


# ---------------------------------------------------------------- t-SVD (Theorem 2.2.1)

@pytest.mark.parametrize("shape", [(4, 3, 5), (3, 4, 6), (3, 3, 1), (2, 4, 2)])
def test_tsvd_reconstruction_and_orthogonality(shape):
    M = _rng(7).standard_normal(shape)
    U, S, V = oracle.tsvd(M)
    n1, n2, n3 = shape
    rec = oracle.tproduct(oracle.tproduct(U, S), oracle.ttranspose(V))
    assert np.allclose(rec, M, atol=1e-11)
    I1 = np.zeros((n1, n1, n3)); I1[:, :, 0] = np.eye(n1)
    I2 = np.zeros((n2, n2, n3)); I2[:, :, 0] = np.eye(n2)
    assert np.allclose(oracle.tproduct(oracle.ttranspose(U), U), I1, atol=1e-11)
    assert np.allclose(oracle.tproduct(oracle.ttranspose(V), V), I2, atol=1e-11)
    # S is f-diagonal: every frontal slice is diagonal
    off = S.copy()
    for i in range(min(n1, n2)):
        off[i, i, :] = 0
    assert np.abs(off).max() < 1e-12


@pytest.mark.parametrize("shape", [(4, 3, 2, 3), (3, 4, 3, 2, 2), (3, 2, 2, 2, 1, 3)])
def test_tsvd_order_4_to_6(shape):
    """Algorithm 1 over modes 3..N: U * S * V^T = M, U^T * U = I, V^T * V = I, S f-diagonal,
    and the diagonal of every Fourier slice of S is numpy's singular values of that slice of M
    (decreasing)."""
    M = _rng(17).standard_normal(shape)
    U, S, V = oracle.tsvd(M)
    n1, n2, modes = shape[0], shape[1], shape[2:]
    rec = oracle.tproduct(oracle.tproduct(U, S), oracle.ttranspose(V))
    assert np.allclose(rec, M, atol=1e-11)
    for X, n in ((U, n1), (V, n2)):
        I = np.zeros((n, n) + modes)
        I[(slice(None), slice(None)) + (0,) * len(modes)] = np.eye(n)
        assert np.allclose(oracle.tproduct(oracle.ttranspose(X), X), I, atol=1e-11)
    off = S.copy()
    for i in range(min(n1, n2)):
        off[i, i] = 0
    assert np.abs(off).max() < 1e-12
    axes = tuple(range(2, M.ndim))
    Mh, Sh = np.fft.fftn(M, axes=axes), np.fft.fftn(S, axes=axes)
    for idx in np.ndindex(*modes):
        sl = (slice(None), slice(None)) + idx
        sv = np.linalg.svd(Mh[sl], compute_uv=False)
        assert np.allclose(np.diagonal(Sh[sl])[:sv.size], sv, atol=1e-10)


def test_truncated_tsvd_theorem_2_3_1():
    n1, n2, n3, k = 5, 4, 6, 2
    M = _rng(8).standard_normal((n1, n2, n3))
    U, S, V = oracle.tsvd(M)
    Mk = oracle.tproduct(oracle.tproduct(U[:, :k, :], S[:k, :k, :]),
                         oracle.ttranspose(V[:, :k, :]))
    err2 = np.linalg.norm((M - Mk).ravel()) ** 2
    # Parseval: the error is (1/n3) sum over Fourier slices of the dropped sigma_i^2
    Mh = np.fft.fft(M, axis=2)
    dropped = sum((np.linalg.svd(Mh[:, :, j], compute_uv=False)[k:] ** 2).sum()
                  for j in range(n3))
    assert abs(err2 - dropped / n3) < 1e-9 * max(1.0, err2)
    # no random X * Y with inner dimension k does better
    r = _rng(9)
    for _ in range(20):
        X = r.standard_normal((n1, k, n3))
        Y = r.standard_normal((k, n2, n3))
        C = oracle.tproduct(X, Y)
        alpha = np.vdot(C.ravel(), M.ravel()) / max(np.vdot(C.ravel(), C.ravel()), 1e-300)
        assert np.linalg.norm((M - alpha * C).ravel()) ** 2 >= err2 - 1e-9


# ---------------------------------------------------------------- compression (Sec. 3)

def _fourier_svals(M):
    axes = tuple(range(2, M.ndim))
    Mh = np.fft.fftn(M, axes=axes)
    return np.stack([np.linalg.svd(Mh[(slice(None), slice(None)) + idx], compute_uv=False)
                     for idx in np.ndindex(*M.shape[2:])], axis=1)   # (min(n1, n2), slices)


def test_truncated_tsvd_theorem_2_3_1_order_5():
    """Theorem 2.3.1 with the DFT over modes 3 to 5: M_k's error is the Parseval sum of the
    dropped Fourier singular values, and no scaled random X * Y of inner size k does better."""
    shape, k = (5, 4, 2, 3, 2), 2
    M = _rng(22).standard_normal(shape)
    U, S, V = oracle.tsvd(M)
    Mk = oracle.tproduct(oracle.tproduct(U[:, :k], S[:k, :k]), oracle.ttranspose(V[:, :k]))
    err2 = np.linalg.norm((M - Mk).ravel()) ** 2
    sv = _fourier_svals(M)
    assert abs(err2 - np.sum(sv[k:] ** 2) / sv.shape[1]) < 1e-9 * max(1.0, err2)
    r = _rng(23)
    for _ in range(20):
        X = r.standard_normal((shape[0], k) + shape[2:])
        Y = r.standard_normal((k, shape[1]) + shape[2:])
        C = oracle.tproduct(X, Y)
        alpha = np.vdot(C.ravel(), M.ravel()) / max(np.vdot(C.ravel(), C.ravel()), 1e-300)
        assert np.linalg.norm((M - alpha * C).ravel()) ** 2 >= err2 - 1e-9


@pytest.mark.parametrize("shape", [(6, 5, 7), (5, 7, 8), (4, 5, 2, 3, 4)])
def test_compress_tubal_is_truncated_tsvd(shape):
    """Method 2 with k tubes is M_k of Theorem 2.3.1: the first k columns of U, S, V
    multiplied back, and its error energy is the discarded singular values' (Parseval, the
    squares summed over every Fourier slice divided by their number)."""
    M = _rng(18).standard_normal(shape)
    k = 2
    Z, kept = oracle.compress(M, oracle.COMPRESS_TUBAL, k)
    assert kept == k * int(np.prod(shape[2:]))
    U, S, V = oracle.tsvd(M)
    Mk = oracle.tproduct(oracle.tproduct(U[:, :k], S[:k, :k]), oracle.ttranspose(V[:, :k]))
    assert np.allclose(Z, Mk, atol=1e-11)
    sv = _fourier_svals(M)
    nsl = sv.shape[1]
    assert np.sum((M - Z) ** 2) == pytest.approx(np.sum(sv[k:] ** 2) / nsl, rel=1e-10)
    Zall, _ = oracle.compress(M, oracle.COMPRESS_TUBAL, min(shape[:2]))
    assert np.allclose(Zall, M, atol=1e-11)


@pytest.mark.parametrize("shape,k", [((6, 5, 7), 9), ((5, 7, 8), 17), ((4, 5, 2, 3, 4), 30),
                                     ((4, 5, 2, 3, 4), 96)])
def test_compress_global_keeps_the_largest_entries(shape, k):
    """Method 1 keeps every Fourier singular value at least as large as the k-th largest
    (numpy's SVD of every slice), so at least k entries, and the error energy is that of the
    rest (Parseval); keeping all of them returns M."""
    M = _rng(19).standard_normal(shape)
    Z, kept = oracle.compress(M, oracle.COMPRESS_GLOBAL, k)
    sv = _fourier_svals(M)
    flat = np.sort(sv.ravel())[::-1]
    thr = flat[k - 1]
    expect = int(np.sum(sv >= thr * (1 - 1e-12)))
    assert kept >= k and kept == expect
    nsl = sv.shape[1]
    assert np.sum((M - Z) ** 2) == pytest.approx(np.sum(flat[kept:] ** 2) / nsl, rel=1e-9,
                                                 abs=1e-12)
    if k == flat.size:
        assert np.allclose(Z, M, atol=1e-11)


# ---------------------------------------------------------------- TNN and t-SVT (Thm 2.4.1, Lemma)

@pytest.mark.parametrize("shape", [(3, 4, 5), (4, 3, 4), (2, 2, 1), (3, 2, 2)])
def test_tnn_is_nuclear_norm_of_block_circulant(shape):
    Y = _rng(10).standard_normal(shape)
    _, _, tnn = oracle.tsvt(Y, 0.0, with_info=True)
    assert abs(tnn - np.linalg.svd(bcirc(Y), compute_uv=False).sum()) < 1e-10 * tnn


@pytest.mark.parametrize("shape,tau", [((3, 4, 5), 0.7), ((4, 3, 4), 2.0), ((2, 3, 1), 0.3),
                                       ((3, 3, 2), 5.0), ((4, 4, 6), 0.0)])
def test_tsvt_is_matrix_svt_of_block_circulant(shape, tau):
    """bcirc is unitarily equivalent to blkdiag of the unnormalised DFT slices, so the t-SVT
    with threshold tau on those slices is the textbook SVT of bcirc(Y)."""
    Y = _rng(11).standard_normal(shape)
    Z = oracle.tsvt(Y, tau)
    assert np.allclose(bcirc(Z), svt_matrix(bcirc(Y), tau), atol=1e-10)


@pytest.mark.parametrize("shape,tau", [((5, 4, 6), 1.5), ((3, 5, 7), 0.8), ((3, 4, 3, 4), 1.0),
                                       ((2, 3, 4, 5), 0.5), ((3, 3, 2, 1), 0.4),
                                       ((3, 4, 2, 3, 4), 1.0), ((4, 3, 3, 2, 2, 3), 0.8)])
def test_tsvt_matches_library_fft_svd(shape, tau):
    """Same result through numpy's FFT over the tube modes and numpy's SVD per slice."""
    Y = _rng(12).standard_normal(shape)
    axes = tuple(range(2, Y.ndim))
    Yh = np.fft.fftn(Y, axes=axes)
    Zh = np.zeros_like(Yh)
    for idx in np.ndindex(*Y.shape[2:]):
        Zh[(slice(None), slice(None)) + idx] = svt_matrix(Yh[(slice(None), slice(None)) + idx], tau)
    Zref = np.fft.ifftn(Zh, axes=axes)
    assert np.abs(Zref.imag).max() < 1e-12
    Z, rk, _ = oracle.tsvt(Y, tau, with_info=True)
    assert np.allclose(Z, Zref.real, atol=1e-11)
    for idx in np.ndindex(*Y.shape[2:]):
        s = np.linalg.svd(Yh[(slice(None), slice(None)) + idx], compute_uv=False)
        assert rk[idx] == int((s > tau).sum())


@pytest.mark.parametrize("shape", [(4, 3, 5), (3, 4, 2, 3, 2)])
def test_tsvt_is_a_firmly_nonexpansive_prox(shape):
    """The t-SVT is the proximal map of a convex function (Thm 2.4.1 with the Lemma), so it
    is firmly non-expansive: ||P(X) - P(Y)||^2 <= <P(X) - P(Y), X - Y>; and its result's TNN
    is the sum of the thresholded singular values."""
    r = _rng(24)
    for _ in range(5):
        X = r.standard_normal(shape)
        Y = X + 0.3 * r.standard_normal(shape)
        tau = 0.8
        PX, PY = oracle.tsvt(X, tau), oracle.tsvt(Y, tau)
        d = (PX - PY).ravel()
        assert d @ d <= d @ (X - Y).ravel() + 1e-12
    sv = []
    Xh = np.fft.fftn(X, axes=tuple(range(2, X.ndim)))
    for idx in np.ndindex(*shape[2:]):
        sv.append(np.linalg.svd(Xh[(slice(None), slice(None)) + idx], compute_uv=False))
    _, _, tnn = oracle.tsvt(PX, 0.0, with_info=True)
    assert tnn == pytest.approx(np.sum(np.maximum(np.concatenate(sv) - tau, 0.0)), rel=1e-10)


def test_svt_lemma_optimality_and_certificate():
    """D_tau(Y) minimises 1/2 ||X - Y||^2 + tau ||X||_* (Lemma of Sec. 4.1); n3 = 1 makes the
    t-SVT the matrix SVT of the single frontal slice."""
    r = _rng(13)
    Y = r.standard_normal((5, 4, 1))
    tau = 1.2
    Z = oracle.tsvt(Y, tau)[:, :, 0]
    Y2 = Y[:, :, 0]
    f = lambda X: 0.5 * np.linalg.norm(X - Y2) ** 2 + tau * np.linalg.svd(X, compute_uv=False).sum()
    f0 = f(Z)
    for _ in range(200):
        E = r.standard_normal(Z.shape)
        for eps in (1e-1, 1e-3):
            assert f(Z + eps * E) >= f0 - 1e-12
    # subgradient certificate: Y - D_tau(Y) = tau (U_r V_r^H + W), ||W||_2 <= 1, U_r^H W = 0
    U, s, Vh = np.linalg.svd(Y2, full_matrices=False)
    r_ = int((s > tau).sum())
    G = (Y2 - Z) / tau
    W = G - U[:, :r_] @ Vh[:r_]
    assert np.linalg.norm(W, 2) <= 1 + 1e-12
    assert np.abs(U[:, :r_].T @ W).max() < 1e-12


def test_tubal_shrinkage_via_convolution():
    """Sec. 4.1: Z = U * (S * T) * V^T with T f-diagonal, T(i,i,:) = iFFT of
    (1 - tau / Shat(i,i,:))_+, equals the t-SVT."""
    Y = _rng(14).standard_normal((4, 3, 5))
    tau = 1.1
    U, S, V = oracle.tsvd(Y)
    Sh = oracle.dft(S)
    Th = np.zeros_like(Sh)
    for i in range(3):
        d = Sh[i, i, :].real
        Th[i, i, :] = np.where(d > 0, np.maximum(1.0 - tau / np.where(d > 0, d, 1.0), 0.0), 0.0)
    T = oracle.idft(Th)
    assert np.abs(T.imag).max() < 1e-12
    Z = oracle.tproduct(oracle.tproduct(U, oracle.tproduct(S, T.real[:3, :3, :])),
                        oracle.ttranspose(V))
    assert np.allclose(Z, oracle.tsvt(Y, tau), atol=1e-11)


# ---------------------------------------------------------------- shrink operators (Sec. 5)

def test_shrink_entry_closed_form():
    D = np.array([-3.0, -1.0, -0.5, 0.0, 0.2, 0.5, 2.0]).reshape(1, 1, 7)
    S = oracle.shrink(D, 0.5, oracle.SPARSE_ENTRY)
    assert np.allclose(S.ravel(), [-2.5, -0.5, 0.0, 0.0, 0.0, 0.0, 1.5])


def test_shrink_tube_is_group_prox():
    """eq. sparse2 is the prox of kappa * sum_ij ||S(i,j,:)||_2: brute force over the scale of
    each tube (the minimiser is a nonnegative multiple of the tube)."""
    r = _rng(15)
    D = r.standard_normal((2, 3, 4))
    D[1, 2, :] = 0.0
    kappa = 1.3
    S = oracle.shrink(D, kappa, oracle.SPARSE_TUBE)
    grid = np.linspace(0.0, 1.0, 200001)
    for i in range(2):
        for j in range(3):
            d = D[i, j, :]
            nd = np.linalg.norm(d)
            obj = kappa * grid * nd + 0.5 * (1 - grid) ** 2 * nd ** 2
            a = grid[np.argmin(obj)]
            assert np.allclose(S[i, j, :], a * d, atol=1e-5)
    assert np.all(S[1, 2, :] == 0)


def test_shrink_tube_groups_every_mode_from_3_on():
    """For order 5 the tube of (i, j) is S(i, j, :, :, :): the group soft threshold (the
    closed form of the prox above) with norms over modes 3 to 5."""
    D = _rng(16).standard_normal((3, 2, 2, 3, 4))
    D[2, 1] = 0.0
    kappa = 4.65
    nrm = np.sqrt((D ** 2).sum(axis=(2, 3, 4), keepdims=True))
    expect = np.where(nrm > kappa, 1.0 - kappa / np.where(nrm > 0, nrm, 1.0), 0.0) * D
    assert np.allclose(oracle.shrink(D, kappa, oracle.SPARSE_TUBE), expect, atol=1e-14)
    assert np.any(nrm > kappa) and np.any((nrm < kappa) & (nrm > 0))


# ---------------------------------------------------------------- ADMM completion (Sec. 4)

def test_completion_exact_recovery_lowrank():
    X, om = synth.workload_lowrank_completion(seed=1)
    Xr, Z = oracle.tnn_complete(X * om, om, 100)
    assert np.array_equal(Xr[om == 1], X[om == 1])               # P_Omega(X) = P_Omega(M)
    assert rse_db(Xr, X) < -60.0
    # the ground truth is feasible, so the minimiser's TNN is not above it
    _, _, tnn_rec = oracle.tsvt(Xr, 0.0, with_info=True)
    _, _, tnn_true = oracle.tsvt(X, 0.0, with_info=True)
    assert tnn_rec <= tnn_true * (1 + 1e-6)


def test_completion_scaled_dual_is_subgradient():
    """After each Z-step, rho_{k+1} Q_{k+1} = rho_k (X + Q_k - Z) lies in the subdifferential
    of TNN/P at Z, so every Fourier slice of it has spectral norm <= 1 with equality on the
    slices where Z is nonzero.  This fixes the scaled-dual update and its rescaling by
    rho_k / rho_{k+1} when rho grows."""
    X, om = synth.workload_lowrank_completion(seed=2, n1=8, n2=7, n3=5, rank=2, p=0.6)
    for iters in (3, 12):
        _, Z, Q, rho = oracle.tnn_complete(X * om, om, iters, rho0=0.05, mu=1.3,
                                           with_dual=True)
        G = np.fft.fft(rho * Q, axis=2)
        Zh = np.fft.fft(Z, axis=2)
        norms = [np.linalg.norm(G[:, :, k], 2) for k in range(5)]
        assert max(norms) <= 1 + 1e-8
        for k in range(5):
            if np.linalg.norm(Zh[:, :, k]) > 1e-8:
                assert abs(norms[k] - 1.0) < 1e-8


def test_completion_sum_scaling_is_avg_with_scaled_penalty():
    """TNN scaling SUM thresholds at P/rho: the same iterates as AVG with rho0 / P."""
    X, om = synth.workload_lowrank_completion(seed=3, n1=6, n2=5, n3=4, rank=2, p=0.5)
    a = oracle.tnn_complete(X * om, om, 7, rho0=0.4, tnn_scale=oracle.SCALE_SUM)
    b = oracle.tnn_complete(X * om, om, 7, rho0=0.1, tnn_scale=oracle.SCALE_AVG)
    assert np.allclose(a[0], b[0], atol=1e-12) and np.allclose(a[1], b[1], atol=1e-12)


def test_completion_zero_iterations_is_projection():
    X, om = synth.workload_lowrank_completion(seed=4, n1=4, n2=3, n3=2, rank=1)
    Xr, Z = oracle.tnn_complete(X, om, 0)
    assert np.array_equal(Xr, np.where(om == 1, X, 0.0))
    assert np.all(Z == 0)


@pytest.mark.parametrize("shape", [(12, 10, 2, 3, 4), (14, 12, 2, 2, 3, 3)])
def test_completion_order_5_and_6(shape):
    """Orders 5 and 6: a low-tubal-rank tensor (built with numpy's FFT) is recovered from 60%
    of its entries, and the scaled dual stays a subgradient of the TNN in every slice of the
    multi-dimensional DFT (spectral norm <= 1)."""
    X = lowrank_fourier(shape, 2, 17)
    om = synth.sampling_mask(shape, 0.6, seed=17)
    Xr, _ = oracle.tnn_complete(X * om, om, 80)
    assert np.array_equal(Xr[om == 1], X[om == 1])
    assert rse_db(Xr, X) < -80.0
    _, Z, Q, rho = oracle.tnn_complete(X * om, om, 6, rho0=0.05, mu=1.3, with_dual=True)
    axes = tuple(range(2, len(shape)))
    G = np.fft.fftn(rho * Q, axes=axes)
    Zh = np.fft.fftn(Z, axes=axes)
    for idx in np.ndindex(*shape[2:]):
        sl = (slice(None), slice(None)) + idx
        g = np.linalg.norm(G[sl], 2)
        assert g <= 1 + 1e-8
        if np.linalg.norm(Zh[sl]) > 1e-8:
            assert abs(g - 1) < 1e-8


# ---------------------------------------------------------------- tensor RPCA (Sec. 5)

def test_rpca_without_corruption_recovers_input():
    M = synth.lowrank_tensor(10, 9, 6, 2, seed=5)
    L, S = oracle.trpca(M, 1.0 / np.sqrt(10 * 6), 150)
    assert relerr(L, M) < 1e-6
    assert np.abs(S).max() < 1e-6 * np.abs(M).max()


@pytest.mark.parametrize("mode", [oracle.SPARSE_ENTRY, oracle.SPARSE_TUBE])
def test_rpca_scaled_dual_bounds(mode):
    """After the S-step, rho_{k+1} W_{k+1} = -rho_k (D - S) is -lambda times a subgradient of
    the sparse penalty at S: |.| <= lambda entrywise (entry mode) or per tube (tube mode),
    with equality on the support of S."""
    M = synth.lowrank_tensor(7, 6, 5, 2, seed=6)
    Sx, _ = synth.sparse_corruption(M.shape, 0.15, seed=6)
    lam = 0.3
    for iters in (4, 15):
        L, S, W, rho = oracle.trpca(M + Sx, lam, iters, rho0=0.05, mu=1.3, sparse_mode=mode,
                                    with_dual=True)
        G = rho * W
        if mode == oracle.SPARSE_ENTRY:
            assert np.abs(G).max() <= lam * (1 + 1e-9)
            on = S != 0
            assert np.allclose(G[on], -lam * np.sign(S[on]), rtol=1e-9, atol=1e-12)
        else:
            gn = np.linalg.norm(G, axis=2)
            sn = np.linalg.norm(S, axis=2)
            assert gn.max() <= lam * (1 + 1e-9)
            on = sn > 0
            assert np.allclose(G[on], -lam * S[on] / sn[on][:, None], rtol=1e-8, atol=1e-12)


@pytest.mark.parametrize("mode", [oracle.SPARSE_ENTRY, oracle.SPARSE_TUBE])
def test_rpca_order_5_duals(mode):
    """Order 5: after the S-step rho W is -lambda times a subgradient of the sparse penalty
    at S (entrywise, or per tube with the tube of (i, j) spanning modes 3 to 5)."""
    shape = (7, 6, 2, 3, 2)
    M = lowrank_fourier(shape, 2, 21)
    Sx, _ = synth.sparse_corruption(shape, 0.15, seed=21)
    lam = 0.3
    L, S, W, rho = oracle.trpca(M + Sx, lam, 8, rho0=0.05, mu=1.3, sparse_mode=mode,
                                with_dual=True)
    G = rho * W
    axes = (2, 3, 4)
    if mode == oracle.SPARSE_ENTRY:
        assert np.abs(G).max() <= lam * (1 + 1e-9)
        on = S != 0
        assert on.any()
        assert np.allclose(G[on], -lam * np.sign(S[on]), rtol=1e-9, atol=1e-12)
    else:
        gn = np.sqrt((G ** 2).sum(axis=axes))
        sn = np.sqrt((S ** 2).sum(axis=axes))
        assert gn.max() <= lam * (1 + 1e-9)
        on = sn > 0
        assert on.any()
        assert np.allclose(G[on], -lam * S[on] / sn[on][:, None, None, None], rtol=1e-8,
                           atol=1e-12)


def test_rpca_separates_sparse_corruption():
    L0 = synth.lowrank_tensor(20, 18, 8, 2, seed=7)
    S0, sup = synth.sparse_corruption(L0.shape, 0.05, seed=7, lo=-20, hi=20)
    lam = 1.0 / np.sqrt(20 * 8)
    L, S = oracle.trpca(L0 + S0, lam, 300)
    assert relerr(L, L0) < 1e-4
    assert relerr(S, S0) < 1e-3


def test_rpca_tube_mode_finds_corrupted_tubes():
    L0 = synth.lowrank_tensor(16, 14, 10, 2, seed=8)
    S0, sup = synth.tube_corruption(L0.shape, 0.08, seed=8, block=10, std=3.0)
    lam = 1.0 / np.sqrt(16)
    L, S = oracle.trpca(L0 + S0, lam, 300, sparse_mode=oracle.SPARSE_TUBE)
    assert relerr(L, L0) < 1e-2
    tube_found = np.linalg.norm(S, axis=2) > 1e-3
    tube_true = np.linalg.norm(S0, axis=2) > 0
    assert np.array_equal(tube_found, tube_true)


def test_rpca_tube_workload_generator():
    """The tube-sparse RPCA workload (Sec. 5 setting): noisy pixel locations constant within
    each 10-frame block, about 10% of the tubes per block, lambda = 1/sqrt(max(n1, n2)), and
    L the panning video itself."""
    M, L0, S0, sup, lam = synth.workload_rpca_tube(seed=3, n1=24, n2=40, n3=25)
    assert M.shape == (24, 40, 25) and lam == 1.0 / np.sqrt(40)
    assert np.array_equal(M, L0 + S0)
    assert np.array_equal(L0, synth.translating_texture(24, 40, 25, 3))
    for b0 in (0, 10, 20):
        blk = sup[:, :, b0:min(b0 + 10, 25)]
        assert np.all(blk == blk[:, :, :1])            # same pixels for the whole block
        assert 0.05 < blk[:, :, 0].mean() < 0.15
    assert np.array_equal(S0 != 0, sup.astype(bool))
