"""Batched complex slice products (tsvd_cgemm) on every engine against an FP64 product.

The bound per engine is a multiple of its unit roundoff times the size of the terms:
relative Frobenius error of C against the FP64 product, normalised by
|| |A| |B| ||_F (the magnitudes a rounding error can scale with), must be below
  FP32 (CUDA cores) 1e-6, 3XTF32 4e-6, TF32 2e-3, BF16 1.6e-2.
"""
import numpy as np
import pytest

from paper_1407_1785_gb300 import synth

pytestmark = pytest.mark.gpu

ENGINES = [("fp32", 0, 1e-6), ("rand_fp32", 4, 1e-6), ("3xtf32", 3, 4e-6), ("tf32", 1, 2e-3),
           ("bf16", 2, 1.6e-2)]


def crandn(seed, stream, shape):
    n = int(np.prod(shape))
    re = synth.normal(seed, stream, n)
    im = synth.normal(seed, stream + 1, n)
    return (re + 1j * im).reshape(shape, order="F")


def op(X, t):
    return X if t == 0 else (X.T if t == 1 else X.conj().T)


def run(prec, transa, transb, m, n, k, batch, seed=3):
    import torch
    from paper_1407_1785_gb300 import libtsvd
    ra, ca = (m, k) if transa == 0 else (k, m)
    rb, cb = (k, n) if transb == 0 else (n, k)
    lda, ldb, ldc = ra + 3, rb + 1, m + 2
    A = [crandn(seed + b, 0, (lda, ca)) for b in range(batch)]
    B = [crandn(seed + b, 2, (ldb, cb)) for b in range(batch)]

    def pack(mats, ld, cols):
        buf = np.zeros((batch, ld * cols), np.complex64)
        for b, X in enumerate(mats):
            buf[b] = X.reshape(-1, order="F")
        return buf

    Ad = torch.from_numpy(pack(A, lda, ca).view(np.float32).ravel()).cuda()
    Bd = torch.from_numpy(pack(B, ldb, cb).view(np.float32).ravel()).cuda()
    Cd = torch.full((batch * ldc * n * 2,), 7.0, device="cuda")
    with libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream,
                         precision=prec) as ctx:
        ctx.cgemm(transa, transb, m, n, k, Ad, lda, lda * ca, Bd, ldb, ldb * cb, Cd, ldc,
                  ldc * n, batch)
        torch.cuda.synchronize()
    Cg = Cd.cpu().numpy().view(np.complex64).reshape(batch, n, ldc).transpose(0, 2, 1)
    errs = []
    for b in range(batch):
        Ao = op(A[b].astype(np.complex64).astype(np.complex128)[:ra, :], transa)
        Bo = op(B[b].astype(np.complex64).astype(np.complex128)[:rb, :], transb)
        ref = Ao @ Bo
        scale = np.linalg.norm(np.abs(Ao) @ np.abs(Bo))
        errs.append(np.linalg.norm(Cg[b, :m, :] - ref) / scale)
        # rows of C beyond m (padding up to ldc) are untouched
        pad = Cg[b, m:, :]
        assert np.all(pad.real == 7.0) and np.all(pad.imag == 7.0)
    return max(errs)


@pytest.mark.parametrize("name,prec,tol", [pytest.param(*e, id=e[0]) for e in ENGINES])
@pytest.mark.parametrize("transa,transb,m,n,k,batch", [
    (0, 0, 128, 64, 32, 1),         # one tile, one chunk
    (0, 0, 200, 37, 333, 3),        # ragged M, N and K over several tiles and chunks
    (1, 2, 145, 70, 90, 2),         # transposed / conjugated operands
    (2, 1, 64, 130, 17, 2),
    (0, 2, 300, 24, 176, 4),        # the sketch shape: N = k
])
def test_cgemm_matches_fp64(name, prec, tol, transa, transb, m, n, k, batch):
    err = run(prec, transa, transb, m, n, k, batch)
    print(f"{name} {transa}{transb} {m}x{n}x{k}: {err:.3e}")
    assert err <= tol, f"{name}: {err:.3e}"
