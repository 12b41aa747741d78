"""The two stopping tests of the plain-form Jacobi (tsvd_opts.jacobi_stop) against the FP64
oracle through the C ABI.

STOP_RELATIVE stops a vector pair once |x^H y| <= tol ||x|| ||y||; STOP_SVT (the default)
also once |x^H y| <= tol min(||x||, ||y||) ||B||_F / nv, which leaves the FP32-noise
tail of a nearly low-rank slice unrotated.  Both must reach the oracle's t-SVT (Lemma of
Sec. 4.1 per Fourier slice) within the per-call tolerance and its ADMM iterates (Sec. 4 and
Sec. 5) within the run tolerance; the SVT test may only save sweeps; the factorisation
(Sec. 2 t-SVD) always uses the relative test, so its output does not depend on the option."""
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


def _dev(x, dtype=np.float32):
    return _torch().from_numpy(colmajor(x, dtype)).cuda()


def _host(t, shape):
    _torch().cuda.synchronize()
    return uncolmajor(t.cpu().numpy(), shape)


def _nearly_lowrank(n1, n2, n3, rank, noise, seed):
    L = synth.lowrank_tensor(n1, n2, n3, rank, seed=seed)
    E = synth.normal(seed, 7, n1 * n2 * n3).reshape((n1, n2, n3), order="F")
    return (L + noise * np.linalg.norm(L) / math.sqrt(L.size) * E).astype(np.float32)


@pytest.mark.parametrize("shape,ctas", [((48, 40, 9), 0), ((96, 80, 6), 0), ((120, 100, 5), 4),
                                        ((40, 130, 4), 2)])
@pytest.mark.parametrize("noise", [1e-6, 1e-3])
def test_tsvt_both_stopping_tests_match_oracle(shape, ctas, noise):
    """A rank-4 tensor plus noise at 1e-6 / 1e-3 of its RMS entry, with the threshold in the
    gap between the signal and the noise singular values and, separately, inside the noise."""
    Y = _nearly_lowrank(*shape, 4, noise, seed=31 + shape[0])
    Yh = np.fft.fft(Y.astype(np.float64), axis=2)
    s = np.concatenate([np.linalg.svd(Yh[:, :, k], compute_uv=False) for k in range(shape[2])])
    s = np.sort(s)[::-1]
    nsig = 4 * shape[2]
    taus = [float(math.sqrt(s[nsig - 1] * s[nsig])), float(0.5 * s[nsig + 2])]
    for tau in taus:
        Zo = oracle.tsvt(Y.astype(np.float64), tau)
        floor = max(np.linalg.norm(Zo), 1e-3 * np.linalg.norm(Y))
        for stop in (libtsvd.STOP_SVT, libtsvd.STOP_RELATIVE):
            with _ctx(jacobi_stop=stop, ctas_per_slice=ctas) as ctx:
                y = _dev(Y)
                z = _torch().empty_like(y)
                ctx.tsvt(y, z, shape, tau)
                Zg = _host(z, shape)
            err = relerr(Zg, Zo, floor=floor)
            assert err <= TSVT_TOL, (stop, tau, err)


@pytest.mark.parametrize("warm", [libtsvd.WARM_OFF, libtsvd.WARM_ON])
@pytest.mark.parametrize("ctas", [0, 4])
def test_rpca_stopping_tests_match_oracle_and_svt_saves_sweeps(warm, ctas):
    """Exact-recovery RPCA (rank 3, 10% corruption) over 120 iterations: the late iterations'
    slices are rank 3 plus an FP32-level residual, the case the SVT test is for."""
    iters = 120
    n1, n2, n3 = 72, 64, 8
    L0 = synth.lowrank_tensor(n1, n2, n3, 3, seed=41)
    S0, _ = synth.sparse_corruption(L0.shape, 0.1, seed=41)
    M = (L0 + S0).astype(np.float32)
    lam = 1.0 / math.sqrt(max(n1, n2) * n3)
    Lo, So = oracle.trpca(M.astype(np.float64), lam, iters)
    e_orc = relerr(Lo, L0)
    out = {}
    for stop in (libtsvd.STOP_SVT, libtsvd.STOP_RELATIVE):
        with _ctx(jacobi_stop=stop, warm_start=warm, ctas_per_slice=ctas) as ctx:
            m = _dev(M)
            l = _torch().empty_like(m)
            s = _torch().empty_like(m)
            st = ctx.trpca(m, M.shape, lam, iters, l, s, stats=True)
            Lg, Sg = _host(l, M.shape), _host(s, M.shape)
        assert st["nonconverged"] == 0
        assert relerr(Lg, Lo, floor=1e-6) <= ADMM_TOL, stop
        assert relerr(Sg, So, floor=1e-3 * np.linalg.norm(M)) <= ADMM_TOL, stop
        e = relerr(Lg, L0)
        # exact recovery: the FP32 floor of these solves, as the full-size RPCA test states
        assert e <= (1e-4 if e_orc < 1e-6 else 1.01 * e_orc + 1e-5), (stop, e, e_orc)
        out[stop] = (st["total_sweeps"], e)
    (sw_svt, e_svt), (sw_rel, e_rel) = out[libtsvd.STOP_SVT], out[libtsvd.STOP_RELATIVE]
    assert sw_svt <= sw_rel
    # the stopped pairs move each t-SVT by ~tol ||B||_F at most: the recovery error stays at
    # the relative test's FP32 level
    assert e_svt <= 1.5 * e_rel + 2e-6, (e_svt, e_rel)


def test_completion_stopping_tests_match_oracle():
    iters = 80
    X, om = synth.workload_lowrank_completion(seed=5, n1=64, n2=56, n3=10, rank=4, p=0.4)
    M = (X * om).astype(np.float32)
    Xo, _ = oracle.tnn_complete(M.astype(np.float64), om, iters)
    for stop in (libtsvd.STOP_SVT, libtsvd.STOP_RELATIVE):
        with _ctx(jacobi_stop=stop) as ctx:
            m = _dev(M)
            o = _torch().from_numpy(colmajor(om, np.uint8)).cuda()
            x = _torch().empty_like(m)
            ctx.tnn_complete(m, o, M.shape, iters, x)
            Xg = _host(x, M.shape)
        assert relerr(Xg, Xo, floor=1e-6) <= ADMM_TOL, stop
        assert abs(relerr(Xg, X) - relerr(Xo, X)) <= 0.01 * relerr(Xo, X) + 1e-5, stop


def test_factor_ignores_the_option():
    """tsvd_factor keeps every direction, so it always runs the relative test: its outputs are
    bit-identical under both settings (the autotuner off, so both take the same plan)."""
    shape, k = (50, 40, 6), 40
    Y = _nearly_lowrank(*shape, 3, 1e-6, seed=51)
    res = []
    for stop in (libtsvd.STOP_SVT, libtsvd.STOP_RELATIVE):
        torch = _torch()
        with _ctx(jacobi_stop=stop, autotune=0) as ctx:
            y = _dev(Y)
            U = torch.empty(shape[0] * k * shape[2], device="cuda")
            S = torch.empty(k * k * shape[2], device="cuda")
            V = torch.empty(shape[1] * k * shape[2], device="cuda")
            ctx.factor(y, shape, k, U, S, V)
            torch.cuda.synchronize()
            res.append([t.cpu().numpy() for t in (U, S, V)])
    for a, b in zip(*res):
        assert np.array_equal(a, b)


def test_invalid_stop_value_is_refused():
    with pytest.raises(libtsvd.TsvdError):
        _ctx(jacobi_stop=2)
