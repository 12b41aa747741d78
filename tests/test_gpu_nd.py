"""Tensors of order 5 and 6 through the C ABI, against the FP64 oracle.

The t-SVD of an order-N tensor takes the DFT along every mode from 3 to N (Sec. 2, the
order-p extension of Algorithm 1) and an SVD of each of the n3 n4 ... nN Fourier slices.  The
library takes the half spectrum along mode N and the full multi-dimensional DFT over modes
3..N-1 (at most 64 entries per tube section for N >= 5).  Tolerances are those of the 3-way and
4-way parity tests: one t-SVT 2e-5 relative, an ADMM solve 1e-3 relative to the oracle's,
factorisations 2e-5.
"""
import math

import numpy as np
import pytest

from helpers import colmajor, lowrank_fourier as lowrank_nd, relerr, uncolmajor

import oracle
from paper_1407_1785_gb300 import libtsvd, synth

pytestmark = pytest.mark.gpu

TSVT_TOL = 2e-5
ADMM_TOL = 1e-3
TOL = 2e-5


def _torch():
    import torch
    return torch


def dev(x, dtype=np.float32):
    return _torch().from_numpy(colmajor(x, dtype)).cuda()


def host(t, shape):
    _torch().cuda.synchronize()
    return uncolmajor(t.cpu().numpy(), shape)


def fourier(X):
    return np.fft.fftn(np.asarray(X, np.float64), axes=tuple(range(2, X.ndim)))


def slice_svals(Y):
    """Singular values of every Fourier slice, (min(n1, n2),) + dims[2:]."""
    Yh = fourier(Y)
    out = np.empty((min(Y.shape[:2]),) + Y.shape[2:])
    for idx in np.ndindex(*Y.shape[2:]):
        out[(slice(None),) + idx] = np.linalg.svd(Yh[(slice(None), slice(None)) + idx],
                                                   compute_uv=False)
    return out


def gap_threshold(sv, q):
    u = np.unique(sv.ravel())
    i = min(max(int(q * len(u)), 1), len(u) - 1)
    return float(0.5 * (u[i - 1] + u[i]))


@pytest.fixture(scope="module")
def ctx():
    torch = _torch()
    c = libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream)
    yield c
    c.close()


def gpu_tsvt(c, Y, tau):
    y = dev(Y)
    z = _torch().empty_like(y)
    mr = np.zeros(int(np.prod(Y.shape[2:])), np.int32)
    _, tnn = c.tsvt(y, z, Y.shape, tau, multirank=mr, with_tnn=True)
    return host(z, Y.shape), uncolmajor(mr, Y.shape[2:]), tnn


def check_tsvt(c, Y, tau):
    Y32 = np.asarray(Y, np.float32)
    Zo, rko, tnno = oracle.tsvt(Y32.astype(np.float64), tau, with_info=True)
    Zg, rkg, tnng = gpu_tsvt(c, Y32, tau)
    floor = 1e-3 * np.linalg.norm(Y32.astype(np.float64).ravel())
    assert relerr(Zg, Zo, floor=floor) <= TSVT_TOL
    assert abs(tnng - tnno) <= 1e-4 * max(tnno, 1e-30)
    sv = slice_svals(Y32)
    smax = sv.max()
    for idx in np.ndindex(*Y.shape[2:]):
        s = sv[(slice(None),) + idx]
        if np.min(np.abs(s - tau)) > 1e-4 * smax:
            assert rkg[idx] == rko[idx], (idx, rkg[idx], rko[idx])


# modes 3..N-1 with 6 to 64 entries per tube section, odd and even sizes on every mode (odd:
# no self-conjugate index but 0; even: index n/2 pairs with itself), long and short last modes
ND_SHAPES = [(5, 4, 2, 3, 4), (4, 6, 3, 2, 5), (6, 5, 3, 4, 6), (7, 5, 2, 2, 3), (4, 3, 8, 8, 3),
             (9, 7, 3, 3, 17), (3, 4, 2, 2, 2, 2), (5, 3, 2, 3, 2, 4), (6, 4, 4, 4, 2, 3),
             (4, 5, 3, 1, 2, 5), (6, 5, 2, 3, 1), (24, 20, 2, 3, 4)]


@pytest.mark.parametrize("shape", ND_SHAPES)
def test_tsvt_parity_nd(ctx, shape):
    Y = synth.normal(81, 0, int(np.prod(shape))).reshape(shape, order="F")
    sv = slice_svals(Y.astype(np.float32))
    for q in (0.0, 0.4, 0.8):
        check_tsvt(ctx, Y, 0.0 if q == 0.0 else gap_threshold(sv, q))


@pytest.mark.parametrize("shape,ctas", [((40, 50, 2, 3, 3), 2), ((70, 60, 3, 2, 2, 2), 4)])
def test_tsvt_parity_nd_cluster(shape, ctas):
    torch = _torch()
    with libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream,
                         ctas_per_slice=ctas) as c:
        Y = synth.normal(82, 0, int(np.prod(shape))).reshape(shape, order="F")
        sv = slice_svals(Y.astype(np.float32))
        check_tsvt(c, Y, gap_threshold(sv, 0.5))


def test_tsvt_nd_mixed_form():
    """The rank-adaptive randomized form (3xTF32 products) on a 5-way low-tubal-rank tensor
    plus noise, with tau above the noise."""
    torch = _torch()
    shape = (40, 36, 3, 2, 5)
    Y = lowrank_nd(shape, 3, 83) + 0.01 * synth.normal(84, 0, int(np.prod(shape))).reshape(
        shape, order="F")
    Y = Y.astype(np.float32)
    sv = slice_svals(Y)
    tau = float(0.5 * (sv[2].min() + sv[3].max()))
    assert sv[2].min() > 2 * sv[3].max()
    Zo = oracle.tsvt(Y.astype(np.float64), tau)
    with libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream,
                         precision=3) as c:
        Zg, _, _ = gpu_tsvt(c, Y, tau)
    assert relerr(Zg, Zo) <= 1e-4


def test_nd_limits(ctx):
    torch = _torch()
    y = torch.zeros(4 * 3 * 9 * 8 * 3, device="cuda")
    z = torch.zeros_like(y)
    with pytest.raises(libtsvd.TsvdError) as e:          # 72 entries per section of modes 3..4
        ctx.tsvt(y, z, (4, 3, 9, 8, 3), 1.0)
    assert e.value.status == libtsvd.TSVD_EUNSUPPORTED
    with pytest.raises(libtsvd.TsvdError) as e:          # order 7
        ctx.tsvt(y, z, (4, 3, 2, 2, 2, 2, 3), 1.0)
    assert e.value.status == libtsvd.TSVD_EINVAL
    u = torch.zeros(4 * 3 * 2 * 2 * 2 * 2 * 3, device="cuda")
    s = torch.zeros_like(u)
    v = torch.zeros_like(u)
    assert ctx.raw_factor(y, (4, 3, 2, 2, 2, 2, 3), 0, u, s, v) == libtsvd.TSVD_EINVAL
    assert ctx.raw_compress(y, (4, 3, 2, 2, 2, 2, 3), libtsvd.COMPRESS_TUBAL, 1, z) == \
        libtsvd.TSVD_EINVAL


# ------------------------------------------------------------------ ADMM solves (Secs. 4, 5)

@pytest.mark.parametrize("shape", [(16, 12, 3, 2, 5), (10, 14, 2, 2, 3, 4)])
def test_completion_nd(ctx, shape):
    X = lowrank_nd(shape, 2, 85)
    om = synth.sampling_mask(shape, 0.6, seed=85)
    M = (X * om).astype(np.float32)
    iters = 40
    Xo, Zo = oracle.tnn_complete(M.astype(np.float64), om, iters)
    m = dev(M)
    o = _torch().from_numpy(colmajor(om, np.uint8)).cuda()
    x, zz = _torch().empty_like(m), _torch().empty_like(m)
    st = ctx.tnn_complete(m, o, shape, iters, x, zz, stats=True)
    Xg, Zg = host(x, shape), host(zz, shape)
    assert np.array_equal(Xg[om == 1], M[om == 1])
    assert relerr(Xg, Xo) <= ADMM_TOL
    assert relerr(Zg, Zo) <= ADMM_TOL
    e_g, e_o = relerr(Xg, X), relerr(Xo, X)
    assert abs(e_g - e_o) <= 0.01 * e_o + 1e-5, (e_g, e_o)
    assert st["nonconverged"] == 0


@pytest.mark.parametrize("mode", ["entry", "tube"])
def test_rpca_nd(mode):
    torch = _torch()
    shape = (18, 14, 2, 3, 4)
    L0 = lowrank_nd(shape, 2, 86)
    if mode == "entry":
        S0, _ = synth.sparse_corruption(shape, 0.08, seed=86)
        sm, om_ = libtsvd.SPARSE_ENTRY, oracle.SPARSE_ENTRY
        lam = 1.0 / math.sqrt(max(shape[:2]) * int(np.prod(shape[2:])))
    else:
        sup = synth.sampling_mask(shape[:2], 0.1, seed=87)
        val = 3.0 * synth.normal(87, 3, int(np.prod(shape))).reshape(shape, order="F")
        S0 = val * sup.reshape(shape[:2] + (1,) * (len(shape) - 2))
        sm, om_ = libtsvd.SPARSE_TUBE, oracle.SPARSE_TUBE
        lam = 1.0 / math.sqrt(max(shape[:2]))
    M = (L0 + S0).astype(np.float32)
    iters = 40
    Lo, So = oracle.trpca(M.astype(np.float64), lam, iters, sparse_mode=om_)
    with libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream,
                         sparse_mode=sm) as c:
        m = dev(M)
        a, b = torch.empty_like(m), torch.empty_like(m)
        st = c.trpca(m, shape, lam, iters, a, b, stats=True)
        Lg, Sg = host(a, shape), host(b, shape)
    floor = 1e-3 * np.linalg.norm(M)
    assert relerr(Lg, Lo, floor=floor) <= ADMM_TOL
    assert relerr(Sg, So, floor=floor) <= ADMM_TOL
    assert st["nonconverged"] == 0


# -------------------------------------------------- t-SVD export and compression (Sec. 3)

def factor_shapes(shape, k):
    n1, n2, rest = shape[0], shape[1], tuple(shape[2:])
    kk = k or min(n1, n2)
    return (n1, kk) + rest, (kk, kk) + rest, (n2, kk) + rest


def _by_slice(Xh):
    return np.moveaxis(Xh.reshape(Xh.shape[0], Xh.shape[1], -1), 2, 0)


def product_fourier(U, S, V):
    Uh, Sh, Vh = (_by_slice(fourier(X)) for X in (U, S, V))
    Rh = Uh @ Sh @ np.conj(np.swapaxes(Vh, 1, 2))
    Rh = np.moveaxis(Rh, 0, 2).reshape((U.shape[0], V.shape[0]) + U.shape[2:])
    return np.real(np.fft.ifftn(Rh, axes=tuple(range(2, U.ndim))))


@pytest.mark.parametrize("shape,k", [((8, 6, 2, 3, 4), 0), ((5, 9, 3, 2, 2, 3), 0),
                                     ((12, 10, 2, 3, 5), 3)])
def test_factor_nd(ctx, shape, k):
    torch = _torch()
    Y = synth.normal(88, 0, int(np.prod(shape))).reshape(shape, order="F").astype(np.float32)
    su, ss, sv_ = factor_shapes(shape, k)
    U, S, V = (torch.empty(int(np.prod(x)), device="cuda") for x in (su, ss, sv_))
    ctx.factor(dev(Y), shape, k, U, S, V)
    U, S, V = host(U, su), host(S, ss), host(V, sv_)
    kk = k or min(shape[:2])
    # f-diagonal S, orthogonal U and V in every Fourier slice, singular values decreasing
    off = S.copy()
    for i in range(kk):
        off[i, i] = 0.0
    assert np.all(off == 0.0)
    for X in (U, V):
        Xh = _by_slice(fourier(X))
        G = np.conj(np.swapaxes(Xh, 1, 2)) @ Xh
        assert np.abs(G - np.eye(kk)).max() <= 10 * TOL
    sv = slice_svals(Y)
    Sh = fourier(S)
    diag = np.stack([Sh[i, i] for i in range(kk)])
    assert np.abs(np.real(diag) - sv[:kk]).max() <= TOL * sv.max()
    # the singular tubes of the oracle's order-N t-SVD (Algorithm 1 over modes 3..N)
    So = fourier(oracle.tsvd(Y.astype(np.float64))[1])
    diag_o = np.stack([So[i, i] for i in range(kk)])
    assert np.abs(diag - diag_o).max() <= TOL * sv.max()
    R = product_fourier(U, S, V)
    if k == 0:
        assert relerr(R, Y) <= TOL
        # and the oracle's order-N t-product multiplies the factors back to Y
        assert relerr(oracle.tproduct(oracle.tproduct(U, S), oracle.ttranspose(V)), Y) <= TOL
    else:
        # per-slice best rank-k approximation: error energy = discarded sigma^2 / #slices
        nsl = int(np.prod(shape[2:]))
        err2 = np.sum((Y.astype(np.float64) - R) ** 2)
        assert err2 == pytest.approx(np.sum(sv[k:] ** 2) / nsl, rel=1e-3)


@pytest.mark.parametrize("shape,method,k", [((8, 6, 2, 3, 4), "global", 70),
                                            ((7, 9, 3, 2, 2, 3), "global", 200),
                                            ((8, 6, 2, 3, 4), "tubal", 2)])
def test_compress_nd(ctx, shape, method, k):
    """Method 1 keeps the k largest Fourier singular values over all slices (ties at the cut
    whole), Method 2 the first k of every slice; either way the error energy is that of the
    discarded values (Parseval over the multi-dimensional DFT)."""
    Y = synth.normal(89, 0, int(np.prod(shape))).reshape(shape, order="F").astype(np.float32)
    m = libtsvd.COMPRESS_GLOBAL if method == "global" else libtsvd.COMPRESS_TUBAL
    y = dev(Y)
    z = _torch().empty_like(y)
    kept, ratio = ctx.compress(y, shape, m, k, z)
    Z = host(z, shape)
    sv = slice_svals(Y)
    nsl = int(np.prod(shape[2:]))
    n1, n2 = shape[:2]
    if method == "global":
        assert k <= kept <= k + 2
        disc = np.sort(sv.ravel())[::-1][kept:]
        assert ratio == pytest.approx(n1 * n2 * nsl / (kept * (n1 + n2 + 1)), rel=1e-12)
    else:
        assert kept == k
        disc = sv[k:].ravel()
        assert ratio == pytest.approx(n1 * n2 / (k * (n1 + n2 + 1)), rel=1e-12)
    err2 = np.sum((Y.astype(np.float64) - Z) ** 2)
    assert err2 == pytest.approx(np.sum(disc ** 2) / nsl, rel=1e-3)
