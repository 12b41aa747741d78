"""The batched solvers through the C ABI against the FP64 oracle: the single-method entry
points tnn_complete_batched / trpca_batched (Sec. 4 and Sec. 5 ADMM loops over a list of
uneven tensors), their kind checks, and the measured FP32 peak used by the rooflines."""
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


def dev(x, dtype=np.float32):
    return _torch().from_numpy(colmajor(x, dtype)).cuda()


def host(t, shape):
    torch = _torch()
    torch.cuda.synchronize()
    return uncolmajor(t.cpu().numpy(), shape)


def _completion_problems(specs, iters, seed0):
    torch = _torch()
    probs, refs = [], []
    for i, (shape, rank, p) in enumerate(specs):
        L0 = synth.lowrank_tensor(shape[0], shape[1], shape[2], rank, seed=seed0 + i)
        om = synth.sampling_mask(shape, p, seed=seed0 + i)
        M = (L0 * om).astype(np.float32)
        refs.append(oracle.tnn_complete(M.astype(np.float64), om, iters)[0])
        q = dict(kind="complete", dims=shape, M=dev(M),
                 omega=torch.from_numpy(colmajor(om, np.uint8)).cuda())
        q["out0"] = torch.empty_like(q["M"])
        q["out1"] = torch.empty_like(q["M"])
        probs.append(q)
    return probs, refs


def _rpca_problems(specs, iters, seed0):
    torch = _torch()
    probs, refs = [], []
    for i, (shape, rank, frac) in enumerate(specs):
        L0 = synth.lowrank_tensor(shape[0], shape[1], shape[2], rank, seed=seed0 + i)
        S0, _ = synth.sparse_corruption(shape, frac, seed=seed0 + i)
        M = (L0 + S0).astype(np.float32)
        lam = 1.0 / math.sqrt(max(shape[0], shape[1]) * shape[2])
        refs.append((oracle.trpca(M.astype(np.float64), lam, iters), np.linalg.norm(M)))
        q = dict(kind="rpca", dims=shape, M=dev(M), lam=lam)
        q["out0"] = torch.empty_like(q["M"])
        q["out1"] = torch.empty_like(q["M"])
        probs.append(q)
    return probs, refs


def test_tnn_complete_batched_matches_oracle(gpu_ctx):
    iters = 30
    probs, refs = _completion_problems([((30, 41, 8), 3, 0.5), ((64, 20, 11), 4, 0.5),
                                        ((48, 48, 5), 2, 0.4)], iters, seed0=300)
    gpu_ctx.tnn_complete_batched(probs, iters)
    for q, Xo in zip(probs, refs):
        assert relerr(host(q["out0"], q["dims"]), Xo, floor=1e-6) <= ADMM_TOL


def test_trpca_batched_matches_oracle(gpu_ctx):
    iters = 30
    probs, refs = _rpca_problems([((52, 36, 6), 2, 0.1), ((20, 70, 9), 2, 0.08),
                                  ((40, 40, 4), 3, 0.1)], iters, seed0=320)
    gpu_ctx.trpca_batched(probs, iters)
    for q, ((Lo, So), nm) in zip(probs, refs):
        assert relerr(host(q["out0"], q["dims"]), Lo, floor=1e-6) <= ADMM_TOL
        assert relerr(host(q["out1"], q["dims"]), So, floor=1e-3 * nm) <= ADMM_TOL


def test_single_kind_entry_points_reject_the_other_kind(gpu_ctx):
    cp, _ = _completion_problems([((12, 10, 4), 2, 0.5)], 1, seed0=340)
    rp, _ = _rpca_problems([((12, 10, 4), 2, 0.1)], 1, seed0=341)
    st, _ = gpu_ctx.raw_solve_batched(cp + rp, 5, entry="tnn_complete_batched")
    assert st == libtsvd.TSVD_EINVAL
    assert "trpca" not in gpu_ctx.last_error() and "kind" in gpu_ctx.last_error()
    st, _ = gpu_ctx.raw_solve_batched(cp + rp, 5, entry="trpca_batched")
    assert st == libtsvd.TSVD_EINVAL
    # the mixed entry point takes both
    st, _ = gpu_ctx.raw_solve_batched(cp + rp, 5, entry="tsvd_solve_batched")
    assert st == libtsvd.TSVD_OK


def test_measured_fp32_peak_is_plausible():
    """The FMA-loop probe behind the FP32 rooflines: positive, and below twice the count
    SMs x 128 lanes x 2 flop x 2.2 GHz (a probe whose loop were optimised away would read
    far above it)."""
    torch = _torch()
    fma, fma2 = libtsvd.measure_fp32_peak(0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    bound = sms * 128 * 2 * 2.2e9 / 1e12
    for v in (fma, fma2):
        assert 0.1 * bound < v < 2.0 * bound


def test_forced_plan_a_tensor_cannot_take_fails_cleanly():
    """A forced ctas_per_slice = 2 cannot hold a 288 x 352 complex slice (two CTAs' shared
    memory is far below the slice's 811 KB): the batched call refuses it with EUNSUPPORTED
    naming the tensor before anything is enqueued, and neither that context (on tensors that
    do fit) nor a fresh one inherits an error from it."""
    torch = _torch()
    iters = 3
    probs, refs = _completion_problems([((30, 41, 8), 3, 0.5), ((288, 352, 4), 5, 0.5),
                                        ((24, 20, 6), 2, 0.5)], iters, seed0=360)
    stream = torch.cuda.current_stream().cuda_stream
    with libtsvd.Context(device=0, stream=stream, ctas_per_slice=2) as ctx:
        st, _ = ctx.raw_solve_batched(probs, iters, entry="tnn_complete_batched")
        assert st == libtsvd.TSVD_EUNSUPPORTED
        assert "problem 1" in ctx.last_error()
        small = [probs[0], probs[2]]
        ctx.tnn_complete_batched(small, iters)
        for q, Xo in zip(small, [refs[0], refs[2]]):
            assert relerr(host(q["out0"], q["dims"]), Xo, floor=1e-6) <= ADMM_TOL
    with libtsvd.Context(device=0, stream=stream) as ctx:
        ctx.tnn_complete_batched(probs, iters)
        for q, Xo in zip(probs, refs):
            assert relerr(host(q["out0"], q["dims"]), Xo, floor=1e-6) <= ADMM_TOL


def test_fewest_ctas_plan_matches_oracle():
    """ctas_per_slice = CTAS_FEWEST (each slice on the fewest CTAs that hold it, for launches
    that share the GPU): the batched solves still reach the oracle's iterates."""
    torch = _torch()
    iters = 20
    probs, refs = _completion_problems([((64, 48, 7), 3, 0.5), ((120, 100, 4), 4, 0.5)], iters,
                                       seed0=380)
    rp, rrefs = _rpca_problems([((90, 70, 6), 2, 0.1)], iters, seed0=381)
    with libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream,
                         ctas_per_slice=libtsvd.CTAS_FEWEST) as ctx:
        st = ctx.solve_batched(probs + rp, iters, stats=True)
    assert st["nonconverged"] == 0
    for q, Xo in zip(probs, refs):
        assert relerr(host(q["out0"], q["dims"]), Xo, floor=1e-6) <= ADMM_TOL
    for q, ((Lo, So), nm) in zip(rp, rrefs):
        assert relerr(host(q["out0"], q["dims"]), Lo, floor=1e-6) <= ADMM_TOL
        assert relerr(host(q["out1"], q["dims"]), So, floor=1e-3 * nm) <= ADMM_TOL
