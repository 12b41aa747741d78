"""Full-length ADMM parity at the benchmark workloads, against values the FP64 oracle stored
in tests/golden/ (written by tests/golden/make_golden.py, which calls only oracle/; the GPU
tests never run the oracle at these sizes).

For each workload the library runs the whole solve through the C ABI on the same seeded
inputs (paper_1407_1785_gb300.synth), and every output tensor must match the oracle's:
  * sampled entries: ||x[idx] - x_oracle[idx]|| <= 1e-3 ||x_oracle[idx]|| at the stored sample
    of entries (sample size 1024, 64 per tensor for the batch);
  * Frobenius norm within 1e-3 relative;
  * recovery error against the ground truth within 1% of the oracle's (+1e-5); where the
    oracle recovers the truth to below 1e-6 (an exact-recovery problem: its FP64 error is below
    anything FP32 can represent of it), the recovery error must instead be at most 1e-4, the
    FP32 floor of these solves (measured 2e-5 to 5e-5 on the 240 x 320 x 60 RPCA, against the
    oracle's 4.6e-15);
  * completion: the observed entries of X bit-exact (X = P_Omega(M) + P_Omega^c(Z - Q)).
The mixed form (3xTF32 / TF32 products) is held to the equal-error rule instead: its recovery
error no worse than the oracle's beyond 1% (+1e-5).

Sec. 4 (eq. proj, eq. shrink, dual ascent) and Sec. 5 (eq. low_rank, eq. sparse, eq. dual).
"""
import json
import math
import os

import numpy as np
import pytest

from helpers import colmajor, uncolmajor

from paper_1407_1785_gb300 import libtsvd, synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
ADMM_TOL = 1e-3


def _golden(name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        return json.load(f)


def _torch():
    import torch
    return torch


def _host(t, shape):
    torch = _torch()
    torch.cuda.synchronize()
    return uncolmajor(t.cpu().numpy(), shape)


def _check(out, gold, truth=None, what="", scale=None):
    """The checks of the module docstring for one output tensor against its stored summary.
    scale (the RPCA S part): the tensor whose size the error is measured against, M for the
    sparse part of the split M = L + S, since an error in L moves to S with the opposite
    sign (default: the output itself)."""
    flat = np.asfortranarray(out).ravel(order="F").astype(np.float64)
    idx = np.asarray(gold["sample_idx"], np.int64)
    ref = np.asarray(gold["sample"], np.float64)
    if scale is None:
        den, nden = np.linalg.norm(ref), gold["norm"]
    else:
        sflat = np.asfortranarray(scale).ravel(order="F").astype(np.float64)
        den, nden = np.linalg.norm(sflat[idx]), np.linalg.norm(sflat)
    samp = np.linalg.norm(flat[idx] - ref) / max(den, 1e-30)
    assert samp <= ADMM_TOL, f"{what}: sampled entries differ by {samp:.3e}"
    nrm = np.linalg.norm(flat)
    assert abs(nrm - gold["norm"]) <= ADMM_TOL * max(nden, 1e-30), \
        f"{what}: norm {nrm} vs {gold['norm']}"
    if truth is not None and "rse" in gold:
        e = np.linalg.norm(out - truth) / np.linalg.norm(truth)
        assert rse_matches(e, gold["rse"]), \
            f"{what}: recovery error {e:.6e} vs oracle {gold['rse']:.6e}"
    return samp


FP32_RSE_FLOOR = 1e-4     # recovery error an FP32 solve may keep where FP64 recovers exactly
EXACT = 1e-6              # oracle recovery errors below this are exact recoveries


def rse_matches(e, e_orc):
    """Recovery error within 1% (+1e-5) of the oracle's, or below the FP32 floor when the
    oracle's recovery is exact."""
    if e_orc < EXACT:
        return e <= FP32_RSE_FLOOR
    return abs(e - e_orc) <= 0.01 * e_orc + 1e-5


def _equal_error(out, gold, truth, what=""):
    """Equal error for the mixed form: no worse than the oracle's beyond 1% (+1e-5), or below
    the FP32 floor on an exact recovery."""
    e = np.linalg.norm(out - truth) / np.linalg.norm(truth)
    ok = e <= FP32_RSE_FLOOR if gold["rse"] < EXACT else e <= gold["rse"] + 0.01 * gold["rse"] + 1e-5
    assert ok, f"{what}: recovery error {e:.6e} vs oracle {gold['rse']:.6e}"


def _completion(ctx, X, om, iters):
    torch = _torch()
    M = (X * om).astype(np.float32)
    m = torch.from_numpy(colmajor(M)).cuda()
    o = torch.from_numpy(colmajor(om, np.uint8)).cuda()
    x = torch.empty_like(m)
    st = ctx.tnn_complete(m, o, X.shape, iters, x, stats=True)
    Xg = _host(x, X.shape)
    obs = om.astype(bool)
    assert np.array_equal(Xg[obs], M[obs])
    return Xg, st


def _rpca(ctx, M, lam, iters):
    torch = _torch()
    m = torch.from_numpy(colmajor(M.astype(np.float32))).cuda()
    l = torch.empty_like(m)
    s = torch.empty_like(m)
    st = ctx.trpca(m, M.shape, lam, iters, l, s, stats=True)
    return _host(l, M.shape), _host(s, M.shape), st


def _ctx(precision=libtsvd.PRECISION_FP32):
    torch = _torch()
    return libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream,
                           precision=precision)


def test_video_completion_150_iterations_matches_oracle():
    g = _golden("video_completion_144x176x100")
    X, om = synth.workload_video_completion(seed=1)
    with _ctx() as ctx:
        Xg, st = _completion(ctx, X, om, g["iters"])
    assert st["nonconverged"] == 0
    _check(Xg, g["X"], X, "video X")


def test_rpca_200_iterations_matches_oracle():
    g = _golden("rpca_240x320x60")
    M, L0, S0, sup, lam = synth.workload_rpca(seed=1)
    assert abs(lam - g["lambda"]) <= 1e-15
    with _ctx() as ctx:
        Lg, Sg, st = _rpca(ctx, M, lam, g["iters"])
    _check(Lg, g["L"], L0, "RPCA L")
    # the recovery-error rule is the recovered tensor's (L); S, the rest of the split, is
    # checked entry by entry and in norm on the scale of M
    _check(Sg, g["S"], None, "RPCA S", scale=M)


@pytest.mark.parametrize("fp64", [0, 1])
def test_rpca_mixed_full_run_equal_error(fp64):
    """The mixed form with split-TF32 (3xTF32) products at the 240 x 320 x 60 RPCA size:
    recovery error no worse than the oracle's beyond 1% (+1e-5), here the FP32 floor since
    the oracle recovers L exactly; k x k solves in FP32 / double-single or FP64."""
    g = _golden("rpca_240x320x60")
    M, L0, S0, sup, lam = synth.workload_rpca(seed=1)
    torch = _torch()
    with libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream,
                         precision=libtsvd.PRECISION_3XTF32, rsvt_small_fp64=fp64) as ctx:
        Lg, Sg, st = _rpca(ctx, M, lam, g["iters"])
    _equal_error(Lg, g["L"], L0, "RPCA L (3xTF32)")


def test_rpca_tf32_full_run_recovery_bound():
    """Plain TF32 products (an 11-bit significand, unit roundoff 4.9e-4) cannot follow an
    exact recovery to the FP32 floor: the 240 x 320 x 60 RPCA stops near 5e-3 (-46 dB)
    instead of 1e-4.  TF32 is therefore outside the equal-error rule on exact-recovery
    problems; this checks that it still recovers L to 1e-2."""
    g = _golden("rpca_240x320x60")
    M, L0, S0, sup, lam = synth.workload_rpca(seed=1)
    with _ctx(libtsvd.PRECISION_TF32) as ctx:
        Lg, Sg, st = _rpca(ctx, M, lam, g["iters"])
    e = np.linalg.norm(Lg - L0) / np.linalg.norm(L0)
    assert e <= 1e-2, f"TF32 RPCA recovery error {e:.3e}"


def test_video_mixed_full_run_equal_error():
    """The 3xTF32 mixed form on the 144 x 176 x 100 video (150 iterations): equal error, and
    its X also within 1e-3 of the oracle's at the stored sample."""
    g = _golden("video_completion_144x176x100")
    X, om = synth.workload_video_completion(seed=1)
    with _ctx(libtsvd.PRECISION_3XTF32) as ctx:
        Xg, st = _completion(ctx, X, om, g["iters"])
    _equal_error(Xg, g["X"], X, "video X (3xTF32)")
    _check(Xg, g["X"], None, "video X (3xTF32)")


# ---- the mixed form, one t-SVT call at the benchmark sizes, against the oracle's t-SVT ----
_TSVT_CASES = {}


def _config_tsvt_case(name):
    """(Y, tau, oracle's t-SVT) at a benchmark size, tau where the ADMM's late iterations put
    it: the RPCA input M (tubal rank 10 plus sparse corruption) with tau in the gap between
    its 10 signal singular values and the corruption's flat floor (the geometric mean of the
    10th and 11th singular values of the DC slice); the colour video itself (a smooth
    texture plus N(0, 0.01^2) noise) with tau = 2% of the largest singular value (about 18
    directions of the DC slice above it, a few in the low frequencies, none in the rest)."""
    import oracle
    if name in _TSVT_CASES:
        return _TSVT_CASES[name]
    if name == "rpca_240x320x60":
        M, L0, S0, sup, lam = synth.workload_rpca(seed=1)
        Y = M.astype(np.float32)
    else:
        X, om = synth.workload_color_video(seed=1)
        Y = X.astype(np.float32)
    axes = tuple(range(2, Y.ndim))
    dc = np.sum(Y.astype(np.float64), axis=axes)       # the DC Fourier slice
    s = np.linalg.svd(dc, compute_uv=False)
    tau = float(math.sqrt(s[9] * s[10])) if name == "rpca_240x320x60" else float(0.02 * s[0])
    Zo = oracle.tsvt(Y.astype(np.float64), tau)
    _TSVT_CASES[name] = (Y, tau, Zo)
    return _TSVT_CASES[name]


@pytest.mark.parametrize("name", ["rpca_240x320x60", "color_video_288x352x3x60"])
@pytest.mark.parametrize("prec,tol,fp64", [(libtsvd.PRECISION_3XTF32, 1e-4, 0),
                                           (libtsvd.PRECISION_3XTF32, 1e-4, 1),
                                           (libtsvd.PRECISION_TF32, 1e-3, 0)])
def test_mixed_tsvt_at_config_size(name, prec, tol, fp64):
    """One mixed-form t-SVT call at the RPCA (240 x 320 x 60) and colour-video (288 x 352 x 3 x
    60) sizes within 1e-3 of the FP64 oracle (TF32 products) or 1e-4 (split 3xTF32), with the
    k x k CholeskyQR2 and eigen-solve in FP32 / double-single or in FP64 (fp64 = 1)."""
    torch = _torch()
    Y, tau, Zo = _config_tsvt_case(name)
    with libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream,
                         precision=prec, rsvt_small_fp64=fp64) as ctx:
        y = torch.from_numpy(colmajor(Y)).cuda()
        z = torch.empty_like(y)
        ctx.tsvt(y, z, Y.shape, tau)
        Zg = _host(z, Y.shape)
    den = max(np.linalg.norm(Zo), 1e-3 * np.linalg.norm(Y))
    err = np.linalg.norm(Zg - Zo) / den
    assert err <= tol, f"{name}: mixed t-SVT error {err:.3e}"


@pytest.mark.parametrize("persistent", [0, 1])
def test_batch_64_uneven_100_iterations_matches_oracle(persistent):
    """The 64-tensor uneven batch (half completion, half RPCA) in one batched call, as
    per-tensor stream branches and as one persistent launch per iteration: every tensor's
    outputs against the oracle's solve of that tensor alone."""
    torch = _torch()
    g = _golden("batch_64_uneven")
    items = synth.workload_batch(seed=1)
    assert len(items) == len(g["tensors"])
    probs = []
    for it, gt in zip(items, g["tensors"]):
        assert list(it["dims"]) == gt["dims"] and it["kind"] == gt["kind"]
        q = dict(kind=it["kind"], dims=it["dims"],
                 M=torch.from_numpy(colmajor(it["M"])).cuda())
        if it["kind"] == "complete":
            q["omega"] = torch.from_numpy(colmajor(it["omega"], np.uint8)).cuda()
        else:
            q["lam"] = it["lam"]
            assert abs(it["lam"] - gt["lambda"]) <= 1e-15
        q["out0"] = torch.empty_like(q["M"])
        q["out1"] = torch.empty_like(q["M"])
        probs.append(q)
    with libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream,
                         batch_persistent=persistent) as ctx:
        st = ctx.solve_batched(probs, g["iters"], stats=True)
    assert st["nonconverged"] == 0
    for b, (it, gt, q) in enumerate(zip(items, g["tensors"], probs)):
        out0 = _host(q["out0"], it["dims"])
        if it["kind"] == "complete":
            obs = it["omega"].astype(bool)
            assert np.array_equal(out0[obs], it["M"][obs]), b
            _check(out0, gt["X"], it["truth"], f"tensor {b} X")
        else:
            _check(out0, gt["L"], it["truth"], f"tensor {b} L")
            _check(_host(q["out1"], it["dims"]), gt["S"], None, f"tensor {b} S", scale=it["M"])


def test_color_video_150_iterations_matches_oracle():
    """The 288 x 352 x 3 x 60 colour video (DFT along modes 3 and 4, 93 stored / 91 distinct
    Fourier slices), 150 iterations of the plain form against the oracle's solve."""
    g = _golden("color_video_completion_288x352x3x60")
    X, om = synth.workload_color_video(seed=1)
    with _ctx() as ctx:
        Xg, st = _completion(ctx, X, om, g["iters"])
    assert st["nonconverged"] == 0
    _check(Xg, g["X"], X, "colour video X")


MIXED_X_TOL = 5e-3   # the mixed form's final X against the exact method's (measured 1.6e-3)


def test_color_video_mixed_full_run_equal_error():
    """The 3xTF32 mixed form on the colour video: equal error against the oracle.  Its final X
    follows a different trajectory from the exact method's (early iterations whose spectrum
    above the threshold is wider than the sketch are thresholded only in the sketched
    subspace), so it is compared with the oracle's X at 5e-3 (measured 1.6e-3); one mixed
    t-SVT call is held to 1e-4 (test_mixed_tsvt_at_config_size)."""
    g = _golden("color_video_completion_288x352x3x60")
    X, om = synth.workload_color_video(seed=1)
    with _ctx(libtsvd.PRECISION_3XTF32) as ctx:
        Xg, st = _completion(ctx, X, om, g["iters"])
    _equal_error(Xg, g["X"], X, "colour video X (3xTF32)")
    flat = np.asfortranarray(Xg).ravel(order="F").astype(np.float64)
    idx = np.asarray(g["X"]["sample_idx"], np.int64)
    ref = np.asarray(g["X"]["sample"], np.float64)
    assert np.linalg.norm(flat[idx] - ref) / np.linalg.norm(ref) <= MIXED_X_TOL
