"""tsvd_tproduct(): the t-product of Def. 2.1.1 through the C ABI, against the FP64 oracle.

3-way: the oracle's t-product (the literal sum of circular convolutions, itself pinned to a
brute-force convolution).  Order 4 to 6: the oracle's DFT over modes 3..N, the slice products
and its inverse DFT.  Tolerance 2e-5 relative (Frobenius) for FP32 slice products, the per-call
t-SVT budget; 3xTF32 products 1e-4, TF32 1e-3, BF16 1e-2.
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


def dev(x):
    return _torch().from_numpy(colmajor(x)).cuda()


def host(t, shape):
    _torch().cuda.synchronize()
    return uncolmajor(t.cpu().numpy(), shape)


def rand(shape, seed):
    return synth.normal(seed, 0, int(np.prod(shape))).reshape(shape, order="F").astype(np.float32)


def oracle_tproduct(A, B):
    """A * B by the oracle: its t-product for order 3; for higher orders its DFT over modes
    3..N, the product of every Fourier slice and its inverse DFT."""
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    if A.ndim == 3:
        return oracle.tproduct(A, B)
    Ah, Bh = oracle.dft(A), oracle.dft(B)
    Ch = np.empty((A.shape[0], B.shape[1]) + A.shape[2:], complex)
    for idx in np.ndindex(*A.shape[2:]):
        sl = (slice(None), slice(None)) + idx
        Ch[sl] = Ah[sl] @ Bh[sl]
    C = oracle.idft(Ch)
    assert np.abs(np.imag(C)).max() <= 1e-9 * max(np.abs(C).max(), 1.0)
    return np.real(C)


def gpu_tproduct(ctx, A, B):
    torch = _torch()
    sc = (A.shape[0], B.shape[1]) + A.shape[2:]
    C = torch.empty(int(np.prod(sc)), device="cuda")
    ctx.tproduct(dev(A), dev(B), C, A.shape, B.shape[1])
    return host(C, sc)


@pytest.fixture(scope="module")
def ctx():
    torch = _torch()
    c = libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream)
    yield c
    c.close()


@pytest.mark.parametrize("sa,n4", [((5, 4, 7), 6), ((1, 3, 4), 1), ((3, 1, 5), 2), ((17, 33, 8), 12),
                                   ((64, 48, 13), 40), ((3, 5, 1), 4), ((9, 7, 100), 5),
                                   ((6, 5, 3, 4), 7), ((4, 3, 5, 40), 2), ((5, 4, 2, 3, 4), 3),
                                   ((4, 6, 3, 2, 2, 3), 5), ((3, 2, 8, 8, 3), 2)])
def test_tproduct_matches_oracle(ctx, sa, n4):
    A = rand(sa, 71)
    B = rand((sa[1], n4) + sa[2:], 72)
    C = gpu_tproduct(ctx, A, B)
    assert relerr(C, oracle_tproduct(A, B)) <= TOL


def test_tproduct_slices_beyond_the_svd_limits(ctx):
    """The t-product runs no slice SVD: 600 x 700 slices (larger than any slice the t-SVT
    takes) are fine."""
    A = rand((600, 700, 3), 78)
    B = rand((700, 30, 3), 79)
    assert relerr(gpu_tproduct(ctx, A, B), oracle_tproduct(A, B)) <= TOL


def test_tproduct_identity_and_host_buffers(ctx):
    """A * I = A for the identity tensor (first frontal slice I, the rest 0; Def. 2.1.3), and
    host buffers give the bits of device buffers."""
    shape = (12, 9, 10)
    A = rand(shape, 73)
    I = np.zeros((9, 9, 10), np.float32)
    I[:, :, 0] = np.eye(9)
    assert relerr(gpu_tproduct(ctx, A, I), A) <= TOL
    B = rand((9, 4, 10), 74)
    Cd = gpu_tproduct(ctx, A, B)
    Ch = np.empty(12 * 4 * 10, np.float32)
    ctx.tproduct(colmajor(A), colmajor(B), Ch, shape, 4)
    assert np.array_equal(uncolmajor(Ch, (12, 4, 10)), Cd)


def test_tsvd_factors_multiply_back(ctx):
    """U * S * V^T = Y with the factors of tsvd_factor and the products of tsvd_tproduct
    (V^T: the tensor transpose of Def. 2.1.2, taken by the oracle)."""
    torch = _torch()
    shape = (20, 14, 9)
    Y = rand(shape, 75)
    k = 14
    U = torch.empty(20 * k * 9, device="cuda")
    S = torch.empty(k * k * 9, device="cuda")
    V = torch.empty(14 * k * 9, device="cuda")
    y = dev(Y)
    ctx.factor(y, shape, 0, U, S, V)
    US = torch.empty(20 * k * 9, device="cuda")
    ctx.tproduct(U, S, US, (20, k, 9), k)
    Vt = dev(oracle.ttranspose(host(V, (14, k, 9))).astype(np.float32))
    R = torch.empty_like(y)
    ctx.tproduct(US, Vt, R, (20, k, 9), 14)
    assert relerr(host(R, shape), Y) <= TOL


@pytest.mark.parametrize("prec,tol", [(3, 1e-4), (1, 1e-3), (2, 1e-2)], ids=["3xtf32", "tf32", "bf16"])
def test_tproduct_tensor_core_products(prec, tol):
    torch = _torch()
    A = rand((48, 40, 6), 76)
    B = rand((40, 36, 6), 77)
    with libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream,
                         precision=prec) as c:
        C = gpu_tproduct(c, A, B)
    assert relerr(C, oracle_tproduct(A, B)) <= tol


def test_tproduct_argument_errors(ctx):
    torch = _torch()
    a = torch.zeros(4 * 3 * 5, device="cuda")
    b = torch.zeros(3 * 2 * 5, device="cuda")
    c = torch.zeros(4 * 2 * 5, device="cuda")
    dims = (4, 3, 5)
    assert ctx.raw_tproduct(a, b, a, dims, 2) == libtsvd.TSVD_EINVAL       # C aliases A
    assert ctx.raw_tproduct(a, b, c, dims, 0) == libtsvd.TSVD_EINVAL       # n4 < 1
    assert ctx.raw_tproduct(a, b, c, (4, 3), 2) == libtsvd.TSVD_EINVAL     # order 2
    assert ctx.raw_tproduct(a, b, c, (4, 3, 5, 1, 1, 1, 1), 2) == libtsvd.TSVD_EINVAL
    assert ctx.raw_tproduct(a, b, c, dims, 2) == libtsvd.TSVD_OK
