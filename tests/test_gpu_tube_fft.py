"""The two forms of the tube pass's half-mode transform through the C ABI against the FP64
oracle (Algorithm 1's DFT along the tubes, the Lemma of Sec. 4.1 per Fourier slice, and the
Sec. 4 / Sec. 5 ADMM loops): the real-input Stockham FFT (even nh >= 128 whose half length
has no prime factor above 5: 128, 160, 200, 250 here) and the DFT products (the other lengths,
including 130 = 2 x 65 = 2 x 5 x 13 and odd 255, next to them)."""
import math

import numpy as np
import pytest

from helpers import colmajor, relerr, uncolmajor

import oracle
from paper_1407_1785_gb300 import libtsvd, synth

pytestmark = pytest.mark.gpu

TSVT_TOL = 2e-5
ADMM_TOL = 1e-3


def _torch():
    import torch
    return torch


def _ctx(**kw):
    torch = _torch()
    return libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream, **kw)


def _host(t, shape):
    _torch().cuda.synchronize()
    return uncolmajor(t.cpu().numpy(), shape)


@pytest.mark.parametrize("shape", [(6, 5, 128), (5, 7, 160), (4, 6, 200), (3, 5, 250),
                                   (6, 5, 130), (4, 3, 255), (5, 4, 3, 128), (3, 4, 2, 160)])
def test_tsvt_long_tubes_match_oracle(shape):
    Y = synth.normal(71, 0, int(np.prod(shape))).reshape(shape, order="F").astype(np.float32)
    for tau in (0.0, 2.0):
        Zo = oracle.tsvt(Y.astype(np.float64), tau)
        with _ctx() as ctx:
            y = _torch().from_numpy(colmajor(Y)).cuda()
            z = _torch().empty_like(y)
            ctx.tsvt(y, z, shape, tau)
            Zg = _host(z, shape)
        floor = max(np.linalg.norm(Zo), 1e-3 * np.linalg.norm(Y))
        assert relerr(Zg, Zo, floor=floor) <= TSVT_TOL, (shape, tau)


def test_completion_long_tubes_match_oracle():
    iters = 20
    X, om = synth.workload_lowrank_completion(seed=72, n1=20, n2=16, n3=200, rank=2, p=0.5)
    M = (X * om).astype(np.float32)
    Xo, _ = oracle.tnn_complete(M.astype(np.float64), om, iters)
    with _ctx() as ctx:
        m = _torch().from_numpy(colmajor(M)).cuda()
        o = _torch().from_numpy(colmajor(om, np.uint8)).cuda()
        x = _torch().empty_like(m)
        ctx.tnn_complete(m, o, M.shape, iters, x)
        Xg = _host(x, M.shape)
    assert relerr(Xg, Xo, floor=1e-6) <= ADMM_TOL
    obs = om.astype(bool)
    assert np.array_equal(Xg[obs], M[obs])


@pytest.mark.parametrize("mode", ["entry", "tube"])
def test_rpca_long_tubes_match_oracle(mode):
    iters = 20
    n1, n2, n3 = 18, 14, 160
    L0 = synth.lowrank_tensor(n1, n2, n3, 2, seed=73)
    S0, _ = synth.sparse_corruption(L0.shape, 0.1, seed=73)
    M = (L0 + S0).astype(np.float32)
    if mode == "entry":
        lam = 1.0 / math.sqrt(max(n1, n2) * n3)
        Lo, So = oracle.trpca(M.astype(np.float64), lam, iters)
        opts = {}
    else:
        lam = 1.0 / math.sqrt(max(n1, n2))
        Lo, So = oracle.trpca(M.astype(np.float64), lam, iters, sparse_mode=oracle.SPARSE_TUBE)
        opts = {"sparse_mode": libtsvd.SPARSE_TUBE}
    with _ctx(**opts) as ctx:
        m = _torch().from_numpy(colmajor(M)).cuda()
        l = _torch().empty_like(m)
        s = _torch().empty_like(m)
        ctx.trpca(m, M.shape, lam, iters, l, s)
        Lg, Sg = _host(l, M.shape), _host(s, M.shape)
    assert relerr(Lg, Lo, floor=1e-6) <= ADMM_TOL
    assert relerr(Sg, So, floor=1e-3 * np.linalg.norm(M)) <= ADMM_TOL
