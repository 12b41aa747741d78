"""tsvd_factor(): the truncated t-SVD (Algorithm 1, Theorem 2.3.1), and tsvd_compress(): the
t-SVD compression of Sec. 3 (Methods 1 and 2), through the C ABI.

The factors are unique only up to a phase per (Fourier slice, column), so the tests compare
what is unique -- U * S * V^T against Y and against the FP64 oracle's truncated t-SVD M_k, the
singular tubes against an SVD of every Fourier slice -- and check that the rest is valid:
U^T * U = I and S f-diagonal.  Tolerances: reconstructions and singular values 2e-5 relative
(the per-call t-SVT budget), orthogonality 2e-5, M_k 1e-4 where the k-th singular value gap
is at least 1e-2 of the largest.
"""
import numpy as np
import pytest

from helpers import colmajor, relerr, uncolmajor

import oracle
from paper_1407_1785_gb300 import libtsvd, synth

pytestmark = pytest.mark.gpu

TOL = 2e-5


def _torch():
    import torch
    return torch


def factor_shapes(shape, k):
    n1, n2, rest = shape[0], shape[1], tuple(shape[2:])
    kk = k or min(n1, n2)
    return (n1, kk) + rest, (kk, kk) + rest, (n2, kk) + rest


def gpu_factor(ctx, Y, k):
    torch = _torch()
    su, ss, sv = factor_shapes(Y.shape, k)
    y = torch.from_numpy(colmajor(Y)).cuda()
    U = torch.empty(int(np.prod(su)), device="cuda")
    S = torch.empty(int(np.prod(ss)), device="cuda")
    V = torch.empty(int(np.prod(sv)), device="cuda")
    ctx.factor(y, Y.shape, k, U, S, V)
    torch.cuda.synchronize()
    return (uncolmajor(U.cpu().numpy(), su), uncolmajor(S.cpu().numpy(), ss),
            uncolmajor(V.cpu().numpy(), sv))


def fourier(X):
    return np.fft.fftn(np.asarray(X, np.float64), axes=tuple(range(2, X.ndim)))


def _by_slice(Xh):
    """(a, b, slices...) -> (slices, a, b)."""
    return np.moveaxis(Xh.reshape(Xh.shape[0], Xh.shape[1], -1), 2, 0)


def product_fourier(U, S, V):
    """U * S * V^T through the Fourier domain (the t-product of Def. 2.1.1 per slice)."""
    Uh, Sh, Vh = (_by_slice(fourier(X)) for X in (U, S, V))
    Rh = Uh @ Sh @ np.conj(np.swapaxes(Vh, 1, 2))
    Rh = np.moveaxis(Rh, 0, 2).reshape((U.shape[0], V.shape[0]) + U.shape[2:])
    return np.real(np.fft.ifftn(Rh, axes=tuple(range(2, U.ndim))))


def gram_fourier(U):
    """U^T * U in the Fourier domain: per slice U-hat^H U-hat, as (k, k, slices)."""
    Uh = _by_slice(fourier(U))
    return np.moveaxis(np.conj(np.swapaxes(Uh, 1, 2)) @ Uh, 0, 2)


def slice_svals(Y):
    Yh = fourier(Y)
    out = np.empty((min(Y.shape[:2]),) + Y.shape[2:])
    for idx in np.ndindex(*Y.shape[2:]):
        out[(slice(None),) + idx] = np.linalg.svd(Yh[(slice(None), slice(None)) + idx],
                                                   compute_uv=False)
    return out


def check_valid(Y, U, S, V, k):
    kk = k or min(Y.shape[:2])
    # S is f-diagonal: its off-diagonal tubes are the inverse DFT of exact zeros
    off = S.copy()
    for i in range(kk):
        off[i, i] = 0.0
    assert np.all(off == 0.0)
    # U^T * U = I and V^T * V = I (the identity tensor: I in every Fourier slice)
    eye = np.eye(kk)[:, :, None]
    assert np.abs(gram_fourier(U) - eye).max() <= TOL * 10
    assert np.abs(gram_fourier(V) - eye).max() <= TOL * 10
    # singular tubes: the diagonal of S-hat is each slice's singular values, decreasing
    Sh = fourier(S)
    diag = np.stack([Sh[i, i] for i in range(kk)])
    sv = slice_svals(Y)[:kk]
    assert np.abs(np.imag(diag)).max() <= TOL * sv.max()
    assert np.abs(np.real(diag) - sv).max() <= TOL * sv.max()


@pytest.fixture(scope="module")
def fctx():
    torch = _torch()
    ctx = libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream)
    yield ctx
    ctx.close()


@pytest.mark.parametrize("shape", [(30, 20, 9), (20, 33, 8), (24, 24, 5), (40, 28, 1), (1, 9, 5),
                                   (9, 1, 4), (64, 48, 13)])
def test_full_factorisation_reproduces_and_matches_oracle(fctx, shape):
    """k = min(n1, n2): U * S * V^T = Y (by the t-product of the oracle, Def. 2.1.1), the
    factors valid, and the same product as the oracle's full t-SVD (Alg. 1)."""
    Y = synth.normal(61, 0, int(np.prod(shape))).reshape(shape, order="F").astype(np.float32)
    U, S, V = gpu_factor(fctx, Y, 0)
    R = oracle.tproduct(oracle.tproduct(U, S), oracle.ttranspose(V))
    assert relerr(R, Y) <= TOL
    check_valid(Y, U, S, V, 0)
    Uo, So, Vo = oracle.tsvd(Y.astype(np.float64))
    Ro = oracle.tproduct(oracle.tproduct(Uo, So), oracle.ttranspose(Vo))
    assert relerr(R, Ro) <= TOL


@pytest.mark.parametrize("shape,k", [((36, 28, 7), 3), ((28, 44, 6), 3), ((50, 50, 4), 5)])
def test_truncated_factorisation_is_oracle_mk(fctx, shape, k):
    """k < min(n1, n2): U * S * V^T is M_k of Theorem 2.3.1, compared with the oracle's full
    t-SVD truncated to its first k singular tubes (a tubal-rank-k tensor plus noise, so the
    k-th gap is wide), and its error is the Parseval sum of the discarded singular values."""
    n1, n2, n3 = shape
    Y = synth.lowrank_tensor(n1, n2, n3, k, seed=62)
    Y = (Y + 0.05 * synth.normal(63, 5, Y.size).reshape(shape, order="F")).astype(np.float32)
    sv = slice_svals(Y)
    assert np.min(sv[k - 1] - sv[k]) >= 1e-2 * sv.max()
    U, S, V = gpu_factor(fctx, Y, k)
    check_valid(Y, U, S, V, k)
    R = oracle.tproduct(oracle.tproduct(U, S), oracle.ttranspose(V))
    Uo, So, Vo = oracle.tsvd(Y.astype(np.float64))
    Mk = oracle.tproduct(oracle.tproduct(Uo[:, :k], So[:k, :k]), oracle.ttranspose(Vo[:, :k]))
    assert relerr(R, Mk) <= 1e-4
    # Theorem 2.3.1: ||Y - M_k||_F^2 = (1/n3) sum over slices of the discarded sigma^2
    err2 = np.sum((Y.astype(np.float64) - R) ** 2)
    assert abs(err2 - np.sum(sv[k:] ** 2) / n3) <= 1e-3 * err2


@pytest.mark.parametrize("shape,k", [((12, 10, 3, 6), 0), ((9, 14, 4, 5), 0), ((16, 12, 3, 4), 4)])
def test_four_way_factorisation(fctx, shape, k):
    """4-way tensors (DFT along modes 3 and 4): reconstruction through the Fourier domain and
    valid factors; for k < min(n1, n2) the per-slice best rank-k approximation."""
    Y = synth.normal(64, 0, int(np.prod(shape))).reshape(shape, order="F").astype(np.float32)
    U, S, V = gpu_factor(fctx, Y, k)
    check_valid(Y, U, S, V, k)
    R = product_fourier(U, S, V)
    if k == 0:
        assert relerr(R, Y) <= TOL
    else:
        Yh = fourier(Y)
        Rh = np.empty_like(Yh)
        for idx in np.ndindex(*shape[2:]):
            sl = (slice(None), slice(None)) + idx
            u, s, vh = np.linalg.svd(Yh[sl])
            Rh[sl] = (u[:, :k] * s[:k]) @ vh[:k]
        Rb = np.real(np.fft.ifftn(Rh, axes=(2, 3)))
        # compared where the k-th gap allows it: the error scales with sigma_max / gap
        sv = slice_svals(Y)
        gap = np.min(sv[k - 1] - sv[k]) / sv.max()
        assert relerr(R, Rb) <= max(1e-4, 1e-6 / gap)


def test_cluster_plans_and_host_buffers(fctx):
    """Slices spread over a cluster of CTAs (converged vectors gathered from every CTA), and
    host buffers staged by the library give the same bits as device buffers."""
    torch = _torch()
    shape = (130, 150, 4)
    Y = synth.normal(65, 0, int(np.prod(shape))).reshape(shape, order="F").astype(np.float32)
    with libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream,
                         ctas_per_slice=4) as ctx:
        U, S, V = gpu_factor(ctx, Y, 0)
        su, ss, sv = factor_shapes(shape, 0)
        hu, hs, hv = (np.empty(int(np.prod(x)), np.float32) for x in (su, ss, sv))
        ctx.factor(colmajor(Y), shape, 0, hu, hs, hv)
    assert np.array_equal(uncolmajor(hu, su), U)
    assert np.array_equal(uncolmajor(hs, ss), S)
    assert np.array_equal(uncolmajor(hv, sv), V)
    R = oracle.tproduct(oracle.tproduct(U, S), oracle.ttranspose(V))
    assert relerr(R, Y) <= TOL
    check_valid(Y, U, S, V, 0)


def test_video_full_size_sampled(fctx):
    """The 144 x 176 x 100 video: full and truncated (k = 20) factorisations; reconstruction
    and the singular values of sampled Fourier slices against numpy."""
    X, om = synth.workload_video_completion(seed=1)
    Y = X.astype(np.float32)
    U, S, V = gpu_factor(fctx, Y, 0)
    assert relerr(product_fourier(U, S, V), Y) <= TOL
    Uk, Sk, Vk = gpu_factor(fctx, Y, 20)
    Yh, Sh = fourier(Y), fourier(Sk)
    for q in (0, 1, 17, 50):
        s = np.linalg.svd(Yh[:, :, q], compute_uv=False)
        assert np.abs(np.real(np.diagonal(Sh[:, :, q])) - s[:20]).max() <= TOL * s[0]
    # M_20 is at least as close to Y as the first 20 tubes of the full factorisation
    e20 = relerr(product_fourier(Uk, Sk, Vk), Y)
    assert abs(e20 - relerr(product_fourier(U[:, :20], S[:20, :20], V[:, :20]), Y)) <= 1e-4


def test_factor_argument_errors(fctx):
    torch = _torch()
    y = torch.zeros(6 * 5 * 3, device="cuda")
    u = torch.zeros(6 * 5 * 3, device="cuda")
    s = torch.zeros(5 * 5 * 3, device="cuda")
    v = torch.zeros(5 * 5 * 3, device="cuda")
    dims = (6, 5, 3)
    assert fctx.raw_factor(y, dims, 6, u, s, v) == libtsvd.TSVD_EINVAL      # k > min(n1, n2)
    assert fctx.raw_factor(y, dims, -1, u, s, v) == libtsvd.TSVD_EINVAL
    assert fctx.raw_factor(y, dims, 0, u, u, v) == libtsvd.TSVD_EINVAL      # aliasing outputs
    assert fctx.raw_factor(y, dims, 0, y, s, v) == libtsvd.TSVD_EINVAL      # output aliases Y
    assert fctx.raw_factor(y, (6, 0, 3), 0, u, s, v) == libtsvd.TSVD_EINVAL
    assert fctx.raw_factor(y, dims, 0, u, s, v) == libtsvd.TSVD_OK


# ------------------------------------------------------------------ compression (Sec. 3)

def gpu_compress(ctx, Y, method, k):
    torch = _torch()
    y = torch.from_numpy(colmajor(Y)).cuda()
    z = torch.empty_like(y)
    kept, ratio = ctx.compress(y, Y.shape, method, k, z)
    return uncolmajor(z.cpu().numpy(), Y.shape), kept, ratio


def oracle_compress(Y, method, k):
    """Sec. 3 on the oracle's t-SVD (Algorithm 1, 3-way): the f-diagonal of S-hat over all n3
    slices; Method 1 keeps the k largest entries (all entries equal to the k-th), Method 2 the
    first k of every slice.  Returns (Z, entries kept)."""
    Uo, So, Vo = oracle.tsvd(np.asarray(Y, np.float64))
    Uh, Sh, Vh = (np.fft.fft(X, axis=2) for X in (Uo, So, Vo))
    n1, n2, n3 = Y.shape
    n0 = min(n1, n2)
    sig = np.real(np.stack([np.diagonal(Sh[:, :, q])[:n0] for q in range(n3)], axis=1))
    if method == libtsvd.COMPRESS_TUBAL:
        keep = np.zeros_like(sig, dtype=bool)
        keep[:k] = True
    else:
        thr = np.sort(sig.ravel())[::-1][k - 1]
        keep = sig >= thr
    Zh = np.zeros((n1, n2, n3), complex)
    for q in range(n3):
        idx = np.nonzero(keep[:, q])[0]
        Zh[:, :, q] = (Uh[:, idx, q] * sig[idx, q]) @ np.conj(Vh[:, idx, q]).T
    return np.real(np.fft.ifft(Zh, axis=2)), int(keep.sum())


@pytest.mark.parametrize("shape", [(36, 28, 7), (28, 44, 8)])
def test_compression_methods_match_oracle(fctx, shape):
    """A tubal-rank-3 tensor plus noise: Method 1 with k = 3 n3 and Method 2 with k = 3 keep
    the signal terms (a wide gap at the cut) and equal the oracle's compression; the ratios are
    the formulas of Sec. 3."""
    n1, n2, n3 = shape
    Y = synth.lowrank_tensor(n1, n2, n3, 3, seed=66)
    Y = (Y + 0.05 * synth.normal(67, 5, Y.size).reshape(shape, order="F")).astype(np.float32)
    for method, k in ((libtsvd.COMPRESS_GLOBAL, 3 * n3), (libtsvd.COMPRESS_TUBAL, 3)):
        Z, kept, ratio = gpu_compress(fctx, Y, method, k)
        Zo, kept_o = oracle_compress(Y, method, k)
        assert relerr(Z, Zo) <= 1e-4, method
        if method == libtsvd.COMPRESS_GLOBAL:
            assert kept == kept_o == k
            assert ratio == pytest.approx(n1 * n2 * n3 / (k * (n1 + n2 + 1)), rel=1e-12)
        else:
            assert kept == k
            assert ratio == pytest.approx(n1 * n2 / (k * (n1 + n2 + 1)), rel=1e-12)
    # Method 2 is the truncated t-SVD of tsvd_factor
    U, S, V = gpu_factor(fctx, Y, 3)
    Z2, _, _ = gpu_compress(fctx, Y, libtsvd.COMPRESS_TUBAL, 3)
    assert relerr(Z2, product_fourier(U, S, V)) <= TOL


@pytest.mark.parametrize("shape,k", [((30, 20, 9), 1), ((30, 20, 9), 57), ((20, 33, 8), 100),
                                     ((12, 10, 3, 6), 90), ((30, 20, 9), 180)])
def test_global_compression_keeps_the_largest_entries(fctx, shape, k):
    """Method 1 on Gaussian tensors (3-way and 4-way), any k: at least k entries kept (ties at
    the cut kept whole), and the error energy is the energy of the discarded Fourier singular
    values (Parseval, Theorem 2.3.1's identity per entry): Z keeps the largest ones.  k = n0 n3
    keeps everything."""
    Y = synth.normal(68, 0, int(np.prod(shape))).reshape(shape, order="F").astype(np.float32)
    Z, kept, ratio = gpu_compress(fctx, Y, libtsvd.COMPRESS_GLOBAL, k)
    sv = np.sort(slice_svals(Y).ravel())[::-1]
    nsl = int(np.prod(shape[2:]))
    assert k <= kept <= k + 2
    assert ratio == pytest.approx(shape[0] * shape[1] * nsl / (kept * (shape[0] + shape[1] + 1)),
                                  rel=1e-12)
    err2 = np.sum((Y.astype(np.float64) - Z) ** 2)
    assert err2 == pytest.approx(np.sum(sv[kept:] ** 2) / nsl, rel=1e-3, abs=1e-6 * np.sum(sv ** 2))
    if kept == sv.size:
        assert relerr(Z, Y) <= TOL


def test_compression_host_buffers_in_place_and_errors(fctx):
    """Host buffers, Z aliasing Y, and the argument checks."""
    shape = (24, 18, 6)
    Y = synth.normal(69, 0, int(np.prod(shape))).reshape(shape, order="F").astype(np.float32)
    Zd, kept_d, _ = gpu_compress(fctx, Y, libtsvd.COMPRESS_GLOBAL, 40)
    h = colmajor(Y).copy()
    kept_h, _ = fctx.compress(h, shape, libtsvd.COMPRESS_GLOBAL, 40, h)     # in place, host
    assert kept_h == kept_d
    assert np.array_equal(uncolmajor(h, shape), Zd)
    torch = _torch()
    y = torch.from_numpy(colmajor(Y)).cuda()
    z = torch.empty_like(y)
    n0 = min(shape[:2])
    assert fctx.raw_compress(y, shape, 3, 1, z) == libtsvd.TSVD_EINVAL
    assert fctx.raw_compress(y, shape, libtsvd.COMPRESS_GLOBAL, 0, z) == libtsvd.TSVD_EINVAL
    assert fctx.raw_compress(y, shape, libtsvd.COMPRESS_GLOBAL, n0 * 6 + 1, z) == libtsvd.TSVD_EINVAL
    assert fctx.raw_compress(y, shape, libtsvd.COMPRESS_TUBAL, n0 + 1, z) == libtsvd.TSVD_EINVAL
    assert fctx.raw_compress(y, shape, libtsvd.COMPRESS_TUBAL, n0, z) == libtsvd.TSVD_OK
