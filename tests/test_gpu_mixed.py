"""The mixed form (randomized, rank-adaptive slice SVT) against the FP64 oracle, through the
C ABI.

Its result is D_tau(Q Q^H A) per Fourier slice, which equals the t-SVT when the sketch covers
every singular direction above tau, so each case compares with the oracle's exact t-SVT:
  * one t-SVT call on a low-rank-plus-noise tensor with tau above the noise: relative
    Frobenius error <= 1e-3 for every precision but BF16 (FP32-level products: <= 1e-4);
  * a full-rank slice set: the sketch grows to the whole slice and the result is exact;
  * ADMM solves: recovery error within 1% (+1e-5) of the oracle's ("equal error").
"""
import math

import numpy as np
import pytest

from helpers import colmajor, relerr, uncolmajor

import oracle
from paper_1407_1785_gb300 import synth

pytestmark = pytest.mark.gpu

# (name, precision value, per-call tolerance, equal-error slack of the recovery error)
FORMS = [("rand_fp32", 4, 1e-4, 0.01), ("3xtf32", 3, 1e-4, 0.01), ("tf32", 1, 1e-3, 0.01),
         ("bf16", 2, 1e-2, 0.05)]
IMPLEMENTED = {"rand_fp32", "3xtf32", "tf32", "bf16"}


def _forms():
    return [pytest.param(*f, id=f[0]) for f in FORMS]


def _ctx(prec, **kw):
    import torch
    from paper_1407_1785_gb300 import libtsvd
    if FORMS and prec not in [f[1] for f in FORMS if f[0] in IMPLEMENTED]:
        pytest.skip("engine not built")
    return libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream,
                           precision=prec, **kw)


def dev(x, dtype=np.float32):
    import torch
    return torch.from_numpy(colmajor(x, dtype)).cuda()


def host(t, shape):
    import torch
    torch.cuda.synchronize()
    return uncolmajor(t.cpu().numpy(), shape)


def lowrank_plus_noise(shape, rank, noise, seed):
    L = synth.lowrank_tensor(shape[0], shape[1], shape[2], rank, seed=seed)
    E = synth.normal(seed, 9, int(np.prod(shape))).reshape(shape, order="F")
    return L + noise * E


def slice_svals(Y):
    Yh = np.fft.fft(np.asarray(Y, np.float64), axis=2)
    return [np.linalg.svd(Yh[:, :, k], compute_uv=False) for k in range(Y.shape[2])]


@pytest.mark.parametrize("name,prec,tol,slack", _forms())
@pytest.mark.parametrize("shape", [(60, 50, 8), (48, 90, 7), (130, 150, 6)])
def test_mixed_tsvt_lowrank_plus_noise(name, prec, tol, slack, shape):
    Y = lowrank_plus_noise(shape, 4, 1e-2, seed=21).astype(np.float32)
    sv = slice_svals(Y)
    # tau between the largest noise singular value and the smallest signal one
    top_noise = max(s[4] for s in sv)
    low_signal = min(s[3] for s in sv)
    assert top_noise < low_signal
    tau = float(math.sqrt(top_noise * low_signal))
    Zo = oracle.tsvt(Y.astype(np.float64), tau)
    with _ctx(prec) as ctx:
        y = dev(Y)
        z = y.clone()
        ctx.tsvt(y, z, shape, tau)
        Zg = host(z, shape)
    err = relerr(Zg, Zo, floor=1e-3 * np.linalg.norm(Y))
    assert err <= tol, f"{name}: {err:.3e}"


@pytest.mark.parametrize("name,prec,tol,slack", _forms())
def test_mixed_tsvt_full_rank_grows_sketch(name, prec, tol, slack):
    """A dense random tensor with a small tau: every slice keeps all 30 singular values, so the
    sketch must grow from its initial width to the whole slice (k = min(n1, n2) = 30)."""
    shape = (40, 30, 5)
    Y = synth.normal(5, 3, int(np.prod(shape))).reshape(shape, order="F").astype(np.float32)
    tau = 0.05
    Zo = oracle.tsvt(Y.astype(np.float64), tau)
    with _ctx(prec) as ctx:
        y = dev(Y)
        z = y.clone()
        ctx.tsvt(y, z, shape, tau)
        Zg = host(z, shape)
    full = {"rand_fp32": 2e-5, "3xtf32": 2e-5, "tf32": 2e-3, "bf16": 2e-2}[name]
    assert relerr(Zg, Zo) <= full


@pytest.mark.parametrize("name,prec,tol,slack", _forms())
def test_mixed_completion_equal_error(name, prec, tol, slack):
    X, om = synth.workload_video_completion(seed=1, n1=72, n2=88, n3=40)
    Mobs = (X * om).astype(np.float32)
    iters = 80
    Xo, _ = oracle.tnn_complete(Mobs.astype(np.float64), om, iters)
    import torch
    with _ctx(prec) as ctx:
        m = dev(Mobs)
        o = torch.from_numpy(colmajor(om, np.uint8)).cuda()
        x = torch.empty_like(m)
        st = ctx.tnn_complete(m, o, Mobs.shape, iters, x, stats=True)
        Xg = host(x, Mobs.shape)
    assert np.array_equal(Xg[om == 1], Mobs[om == 1])
    e_g, e_o = relerr(Xg, X), relerr(Xo, X)
    assert abs(e_g - e_o) <= slack * e_o + 1e-5, (name, e_g, e_o)
    assert st["iters"] == iters and 8 <= st["rsvt_k_last"] <= 72
    assert st["slice_launches"] == iters


@pytest.mark.parametrize("name,prec,tol,slack", _forms())
def test_mixed_rpca_matches_oracle(name, prec, tol, slack):
    L0 = synth.lowrank_tensor(40, 36, 8, 2, seed=31)
    S0, _ = synth.sparse_corruption(L0.shape, 0.1, seed=31)
    M = (L0 + S0).astype(np.float32)
    lam = 1.0 / math.sqrt(40 * 8)
    iters = 60
    Lo, So = oracle.trpca(M.astype(np.float64), lam, iters)
    import torch
    with _ctx(prec) as ctx:
        m = dev(M)
        l = torch.empty_like(m)
        s = torch.empty_like(m)
        ctx.trpca(m, M.shape, lam, iters, l, s)
        Lg = host(l, M.shape)
    e_g, e_o = relerr(Lg, L0), relerr(Lo, L0)
    lim = {"rand_fp32": 1e-3, "3xtf32": 1e-3, "tf32": 2e-2, "bf16": 1e-1}[name]
    assert relerr(Lg, Lo) <= lim, (name, relerr(Lg, Lo))
    assert e_g <= e_o + lim


@pytest.mark.parametrize("name,prec,tol,slack", [f for f in _forms() if f.id in ("3xtf32", "tf32")])
def test_mixed_batched_matches_oracle(name, prec, tol, slack):
    """Uneven tensors, completion and RPCA, in one batched call of the mixed form (the sketch
    width chosen on the device, the whole batch in one CUDA graph): each tensor recovers its
    ground truth as well as the oracle's solve does (within the slack), and a second call
    replays the graph bit for bit."""
    import torch
    specs = [("complete", (48, 40, 8), 3, 0.5), ("rpca", (36, 52, 6), 2, 0.1),
             ("complete", (70, 30, 9), 4, 0.6), ("rpca", (40, 44, 5), 3, 0.08)]
    iters = 40
    probs, truths, oracle_err = [], [], []
    for i, (kind, shape, rank, frac) in enumerate(specs):
        L0 = synth.lowrank_tensor(shape[0], shape[1], shape[2], rank, seed=70 + i)
        if kind == "complete":
            om = synth.sampling_mask(shape, frac, seed=70 + i)
            M = (L0 * om).astype(np.float32)
            Xo, _ = oracle.tnn_complete(M.astype(np.float64), om, iters)
            q = dict(kind=kind, dims=shape, M=dev(M),
                     omega=torch.from_numpy(colmajor(om, np.uint8)).cuda())
        else:
            S0, _ = synth.sparse_corruption(shape, frac, seed=70 + i)
            M = (L0 + S0).astype(np.float32)
            lam = 1.0 / math.sqrt(max(shape[0], shape[1]) * shape[2])
            Xo, _ = oracle.trpca(M.astype(np.float64), lam, iters)
            q = dict(kind=kind, dims=shape, M=dev(M), lam=lam)
        q["out0"] = torch.empty_like(q["M"])
        q["out1"] = torch.empty_like(q["M"])
        probs.append(q)
        truths.append(L0)
        oracle_err.append(relerr(Xo, L0))
    with _ctx(prec) as ctx:
        first = None
        for call in range(2):
            st = ctx.solve_batched(probs, iters, stats=True)
            got = [host(q["out0"], q["dims"]) for q in probs]
            if first is None:
                first = got
            else:
                for a, b in zip(got, first):
                    assert np.array_equal(a, b)
        assert st["slice_launches"] == iters * len(specs)
        assert 8 <= st["rsvt_k_last"] <= 44
    # these instances recover their ground truth almost exactly, so the TF32 products' own
    # rounding (~5e-4 relative per product) sets the floor of that engine's recovery error
    floor = {"3xtf32": 1e-4, "tf32": 2e-3}[name]
    for X, L0, eo in zip(first, truths, oracle_err):
        eg = relerr(X, L0)
        assert eg <= eo + slack * eo + floor, (name, eg, eo)
