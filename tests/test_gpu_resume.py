"""Resuming the ADMM solves of Sec. 4 (completion: eq. proj, eq. shrink, dual ascent) and
Sec. 5 (RPCA: eq. low_rank, eq. sparse, eq. dual) from a returned state: k1 iterations, then
k2 more from (Z, Q, rho) or (S, W, rho), against the oracle's k1 + k2 iterations; the final
scaled duals against the oracle's."""
import math

import numpy as np
import pytest

from helpers import colmajor, relerr, uncolmajor

import oracle
from paper_1407_1785_gb300 import libtsvd, synth

pytestmark = pytest.mark.gpu

ADMM_TOL = 1e-3


def _torch():
    import torch
    return torch


def _host(t, shape):
    torch = _torch()
    torch.cuda.synchronize()
    return uncolmajor(t.cpu().numpy(), shape)


@pytest.mark.parametrize("k1,k2", [(10, 15), (1, 1)])
def test_completion_resume_matches_one_long_run(gpu_ctx, k1, k2):
    torch = _torch()
    X0 = synth.lowrank_tensor(40, 36, 10, 3, seed=51)
    om = synth.sampling_mask(X0.shape, 0.5, seed=51)
    M = (X0 * om).astype(np.float32)
    shape = M.shape
    Xo1, Zo1, Qo1, rho1 = oracle.tnn_complete(M.astype(np.float64), om, k1, with_dual=True)
    Xo, Zo = oracle.tnn_complete(M.astype(np.float64), om, k1 + k2)
    m = torch.from_numpy(colmajor(M)).cuda()
    o = torch.from_numpy(colmajor(om, np.uint8)).cuda()
    x, z, q = torch.empty_like(m), torch.empty_like(m), torch.empty_like(m)
    st = gpu_ctx.tnn_complete_resume(m, o, shape, k1, x, Z_out=z, Q_out=q, stats=True)
    assert abs(st["rho_final"] - rho1) <= 1e-12 * rho1
    assert relerr(_host(q, shape), Qo1, floor=1e-3 * np.linalg.norm(M)) <= ADMM_TOL
    assert relerr(_host(z, shape), Zo1, floor=1e-6) <= ADMM_TOL
    x2, z2 = torch.empty_like(m), torch.empty_like(m)
    gpu_ctx.tnn_complete_resume(m, o, shape, k2, x2, Z_out=z2, Z0=z, Q0=q, rho=st["rho_final"])
    assert relerr(_host(x2, shape), Xo, floor=1e-6) <= ADMM_TOL
    assert relerr(_host(z2, shape), Zo, floor=1e-6) <= ADMM_TOL
    obs = om.astype(bool)
    assert np.array_equal(_host(x2, shape)[obs], M[obs])


@pytest.mark.parametrize("mode", [libtsvd.SPARSE_ENTRY, libtsvd.SPARSE_TUBE])
def test_rpca_resume_matches_one_long_run(mode):
    torch = _torch()
    L0 = synth.lowrank_tensor(44, 38, 8, 3, seed=52)
    S0, _ = synth.sparse_corruption(L0.shape, 0.1, seed=52)
    M = (L0 + S0).astype(np.float32)
    shape = M.shape
    lam = 1.0 / math.sqrt(44 * (8 if mode == libtsvd.SPARSE_ENTRY else 1))
    k1, k2 = 12, 18
    om = oracle.SPARSE_TUBE if mode == libtsvd.SPARSE_TUBE else oracle.SPARSE_ENTRY
    Lo1, So1, Wo1, rho1 = oracle.trpca(M.astype(np.float64), lam, k1, sparse_mode=om,
                                       with_dual=True)
    Lo, So = oracle.trpca(M.astype(np.float64), lam, k1 + k2, sparse_mode=om)
    nm = np.linalg.norm(M)
    with libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream,
                         sparse_mode=mode) as ctx:
        m = torch.from_numpy(colmajor(M)).cuda()
        l, s, w = torch.empty_like(m), torch.empty_like(m), torch.empty_like(m)
        st = ctx.trpca_resume(m, shape, lam, k1, l, s, W_out=w, stats=True)
        assert abs(st["rho_final"] - rho1) <= 1e-12 * rho1
        assert relerr(_host(w, shape), Wo1, floor=1e-3 * nm) <= ADMM_TOL
        assert relerr(_host(s, shape), So1, floor=1e-3 * nm) <= ADMM_TOL
        l2, s2 = torch.empty_like(m), torch.empty_like(m)
        ctx.trpca_resume(m, shape, lam, k2, l2, s2, S0=s, W0=w, rho=st["rho_final"])
    assert relerr(_host(l2, shape), Lo, floor=1e-6) <= ADMM_TOL
    assert relerr(_host(s2, shape), So, floor=1e-3 * nm) <= ADMM_TOL


def test_resume_rejects_host_state_and_zero_iterations(gpu_ctx):
    torch = _torch()
    M = np.ones((8, 6, 4), np.float32)
    om = np.ones((8, 6, 4), np.uint8)
    m = torch.from_numpy(colmajor(M)).cuda()
    o = torch.from_numpy(colmajor(om, np.uint8)).cuda()
    x = torch.empty_like(m)
    zh = colmajor(M)                       # host memory
    with pytest.raises(libtsvd.TsvdError) as ei:
        gpu_ctx.tnn_complete_resume(m, o, M.shape, 3, x, Z0=zh)
    assert ei.value.status == libtsvd.TSVD_EINVAL
    with pytest.raises(libtsvd.TsvdError) as ei:
        gpu_ctx.tnn_complete_resume(m, o, M.shape, 0, x, Z0=m)
    assert ei.value.status == libtsvd.TSVD_EINVAL
