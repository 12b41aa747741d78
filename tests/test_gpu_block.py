"""The block form of the plain slice SVT (each round of vector blocks computed on the Gram of
a CTA's vectors) against the FP64 oracle, forced through the slice_form option: one t-SVT
call per shape (Lemma of Sec. 4.1 on every Fourier slice, Algorithm 1's DFT along modes 3..N),
on one CTA and on clusters of 2 to 8 CTAs, vectors as columns and as rows, real
(self-conjugate) slices, the accumulated-V rebuild, and short ADMM solves of both methods
(Sec. 4 and Sec. 5) with and without the warm start."""
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


def _ctx(**opts):
    torch = _torch()
    return libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream,
                           slice_form=libtsvd.SLICE_BLOCK, autotune=0, **opts)


def _tsvt(ctx, Y, tau):
    torch = _torch()
    y = torch.from_numpy(colmajor(Y)).cuda()
    z = torch.empty_like(y)
    ctx.tsvt(y, z, Y.shape, tau)
    torch.cuda.synchronize()
    return uncolmajor(z.cpu().numpy(), Y.shape)


def _thresholds(Y):
    axes = tuple(range(2, Y.ndim))
    Yh = np.fft.fftn(Y.astype(np.float64), axes=axes)
    sv = []
    for idx in np.ndindex(*Y.shape[2:]):
        sv.append(np.linalg.svd(Yh[(slice(None), slice(None)) + idx], compute_uv=False))
    u = np.unique(np.concatenate(sv))
    out = [0.0]
    for q in (0.3, 0.7):
        i = min(max(int(q * len(u)), 1), len(u) - 1)
        out.append(float(0.5 * (u[i - 1] + u[i])))
    return out


@pytest.mark.parametrize("shape,ctas", [((32, 32, 16), 0), ((33, 17, 7), 1), ((17, 33, 8), 1),
                                        ((64, 48, 13), 2), ((48, 64, 6), 4), ((150, 20, 9), 0),
                                        ((144, 176, 4), 8), ((200, 190, 3), 4), ((40, 50, 5), 8),
                                        ((9, 7, 3, 6), 0), ((16, 12, 3, 5), 2)])
def test_block_form_tsvt_matches_oracle(shape, ctas):
    Y = synth.normal(31, 0, int(np.prod(shape))).reshape(shape, order="F").astype(np.float32)
    with _ctx(ctas_per_slice=ctas) as ctx:
        for tau in _thresholds(Y):
            Zo = oracle.tsvt(Y.astype(np.float64), tau)
            Zg = _tsvt(ctx, Y, tau)
            floor = 1e-3 * np.linalg.norm(Y)
            assert relerr(Zg, Zo, floor=floor) <= TSVT_TOL, (shape, ctas, tau)


@pytest.mark.parametrize("shape,ctas", [((40, 50, 5), 1), ((130, 150, 4), 4), ((150, 130, 4), 2)])
def test_block_form_accumulated_v(shape, ctas):
    """The V-form rebuild (rotations accumulated into V inside the block update)."""
    Y = synth.normal(32, 0, int(np.prod(shape))).reshape(shape, order="F").astype(np.float32)
    with _ctx(ctas_per_slice=ctas, accumulate_v=1) as ctx:
        for tau in _thresholds(Y)[1:]:
            Zo = oracle.tsvt(Y.astype(np.float64), tau)
            assert relerr(_tsvt(ctx, Y, tau), Zo, floor=1e-3 * np.linalg.norm(Y)) <= TSVT_TOL


def test_block_form_matches_pairwise_rank_and_sweeps():
    """Both forms run the same rotations in exact arithmetic: the same multi-rank and the same
    result to the t-SVT tolerance."""
    torch = _torch()
    X = synth.lowrank_tensor(96, 80, 12, 6, seed=33)
    Y = (X + 0.01 * synth.normal(33, 5, X.size).reshape(X.shape, order="F")).astype(np.float32)
    y = torch.from_numpy(colmajor(Y)).cuda()
    res = {}
    for form in (libtsvd.SLICE_PAIRWISE, libtsvd.SLICE_BLOCK):
        with libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream,
                             slice_form=form, autotune=0) as ctx:
            z = torch.empty_like(y)
            mr = np.zeros(Y.shape[2], np.int32)
            ctx.tsvt(y, z, Y.shape, 5.0, multirank=mr)
            torch.cuda.synchronize()
            res[form] = (uncolmajor(z.cpu().numpy(), Y.shape), mr.copy())
    (zp, rp), (zb, rb) = res[libtsvd.SLICE_PAIRWISE], res[libtsvd.SLICE_BLOCK]
    assert np.array_equal(rp, rb)
    assert relerr(zb, zp, floor=1e-3 * np.linalg.norm(Y)) <= TSVT_TOL


@pytest.mark.parametrize("warm", [libtsvd.WARM_OFF, libtsvd.WARM_ON])
def test_block_form_completion_matches_oracle(warm):
    torch = _torch()
    X = synth.lowrank_tensor(60, 44, 10, 3, seed=34)
    om = synth.sampling_mask(X.shape, 0.5, seed=34)
    M = (X * om).astype(np.float32)
    iters = 40
    Xo, _ = oracle.tnn_complete(M.astype(np.float64), om, iters)
    with _ctx(warm_start=warm) as ctx:
        m = torch.from_numpy(colmajor(M)).cuda()
        o = torch.from_numpy(colmajor(om, np.uint8)).cuda()
        x = torch.empty_like(m)
        st = ctx.tnn_complete(m, o, X.shape, iters, x, stats=True)
        torch.cuda.synchronize()
        Xg = uncolmajor(x.cpu().numpy(), X.shape)
    assert st["nonconverged"] == 0
    assert relerr(Xg, Xo, floor=1e-6) <= ADMM_TOL
    obs = om.astype(bool)
    assert np.array_equal(Xg[obs], M[obs])


def test_block_form_rpca_matches_oracle():
    torch = _torch()
    L0 = synth.lowrank_tensor(70, 52, 8, 3, seed=35)
    S0, _ = synth.sparse_corruption(L0.shape, 0.1, seed=35)
    M = (L0 + S0).astype(np.float32)
    lam = 1.0 / math.sqrt(70 * 8)
    iters = 40
    Lo, So = oracle.trpca(M.astype(np.float64), lam, iters)
    with _ctx() as ctx:
        m = torch.from_numpy(colmajor(M)).cuda()
        l = torch.empty_like(m)
        s = torch.empty_like(m)
        ctx.trpca(m, M.shape, lam, iters, l, s)
        torch.cuda.synchronize()
        Lg = uncolmajor(l.cpu().numpy(), M.shape)
        Sg = uncolmajor(s.cpu().numpy(), M.shape)
    assert relerr(Lg, Lo, floor=1e-6) <= ADMM_TOL
    assert relerr(Sg, So, floor=1e-3 * np.linalg.norm(M)) <= ADMM_TOL


def test_block_form_deterministic():
    Y = synth.normal(36, 0, 80 * 70 * 6).reshape((80, 70, 6), order="F").astype(np.float32)
    with _ctx(ctas_per_slice=2) as ctx:
        a = _tsvt(ctx, Y, 3.0)
        b = _tsvt(ctx, Y, 3.0)
    assert np.array_equal(a, b)
