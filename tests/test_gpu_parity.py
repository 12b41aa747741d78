"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on seeded inputs.

Tolerances:
  * one t-SVT call: relative Frobenius error <= 2e-5, normalised by
    max(||Z_oracle||_F, 1e-3 ||Y||_F) (early ADMM thresholds can zero almost everything);
  * an ADMM run: final tensor within 1e-3 relative of the oracle's, and a recovery error
    against the ground truth within 1% (+1e-5) of the oracle's;
  * masks and the observed entries of X: bit-exact.
"""
import math

import numpy as np
import pytest

from helpers import colmajor, relerr, uncolmajor

import oracle
from paper_1407_1785_gb300 import synth

pytestmark = pytest.mark.gpu

TSVT_TOL = 2e-5
ADMM_TOL = 1e-3


def _torch():
    import torch
    return torch


def dev(x, dtype=np.float32):
    torch = _torch()
    return torch.from_numpy(colmajor(x, dtype)).cuda()


def host(t, shape):
    torch = _torch()
    torch.cuda.synchronize()
    return uncolmajor(t.cpu().numpy(), shape)


def gpu_tsvt(ctx, Y, tau, allow_notconv=False):
    y = dev(Y)
    z = _torch().empty_like(y)
    ns = int(np.prod(Y.shape[2:]))
    mr = np.zeros(ns, np.int32)
    st, tnn = ctx.tsvt(y, z, Y.shape, tau, multirank=mr, with_tnn=True,
                       allow_notconv=allow_notconv)
    return host(z, Y.shape), uncolmajor(mr, Y.shape[2:]), tnn


def slice_singular_values(Y):
    axes = tuple(range(2, Y.ndim))
    Yh = np.fft.fftn(np.asarray(Y, np.float64), axes=axes)
    out = {}
    for idx in np.ndindex(*Y.shape[2:]):
        out[idx] = np.linalg.svd(Yh[(slice(None), slice(None)) + idx], compute_uv=False)
    return out


def check_tsvt(ctx, Y, tau):
    Y32 = np.asarray(Y, np.float32)
    Zo, rko, tnno = oracle.tsvt(Y32.astype(np.float64), tau, with_info=True)
    Zg, rkg, tnng = gpu_tsvt(ctx, Y32, tau)
    floor = 1e-3 * np.linalg.norm(Y32.astype(np.float64).ravel())
    err = relerr(Zg, Zo, floor=floor)
    assert err <= TSVT_TOL, f"t-SVT relative error {err:.3e}"
    # the TNN (sum of every Fourier slice's singular values) at 1e-5: measured 4.9e-7 on the
    # 144 x 176 x 100 video and 4.7e-6 on the 240 x 320 x 60 RPCA input (each singular value
    # carries the Jacobi's FP32 rounding, ~eps_32 sqrt(sweeps) relative)
    assert abs(tnng - tnno) <= 1e-5 * max(tnno, 1e-30)
    # multi-rank: exact wherever no singular value sits within 1e-4 sigma_max of tau
    sv = slice_singular_values(Y32)
    smax = max(s.max() for s in sv.values()) if sv else 0.0
    for idx, s in sv.items():
        if s.size and np.min(np.abs(s - tau)) > 1e-4 * max(smax, 1e-30):
            assert rkg[idx] == rko[idx], (idx, rkg[idx], rko[idx])
    return err


def gap_threshold(allsv, q):
    """A threshold at quantile q of the singular values, placed in the middle of the gap
    between two consecutive distinct values (a threshold within rounding distance of a
    singular value makes the result ill-conditioned in any precision)."""
    if q == 0.0:
        return 0.0
    u = np.unique(allsv)
    i = min(max(int(q * len(u)), 1), len(u) - 1)
    return float(0.5 * (u[i - 1] + u[i]))


@pytest.mark.parametrize("shape", [(32, 32, 16), (33, 17, 7), (17, 33, 8), (40, 24, 1),
                                   (5, 64, 2), (1, 9, 5), (9, 1, 4), (64, 48, 13), (3, 130, 6),
                                   (150, 20, 9), (144, 176, 4), (200, 190, 3),
                                   # long tubes: tube-tile row groups of 2, 4 and 8 rows, padding
                                   (5, 4, 33), (3, 4, 64), (8, 6, 100), (6, 5, 130), (4, 3, 255)])
def test_tsvt_parity_3d(gpu_ctx, shape):
    Y = synth.normal(11, 0, int(np.prod(shape))).reshape(shape, order="F")
    sv = slice_singular_values(Y.astype(np.float32))
    allsv = np.sort(np.concatenate([s for s in sv.values()]))
    for q in (0.0, 0.3, 0.7):
        check_tsvt(gpu_ctx, Y, gap_threshold(allsv, q))
    # above the largest singular value everything is thresholded away
    Zg, rk, _ = gpu_tsvt(gpu_ctx, Y.astype(np.float32), float(allsv[-1]) * 1.01)
    assert np.abs(Zg).max() == 0.0 and rk.max() == 0


@pytest.mark.parametrize("shape", [(9, 7, 3, 6), (16, 12, 3, 5), (8, 8, 4, 4), (6, 10, 5, 1),
                                   (7, 5, 1, 6), (4, 3, 5, 40), (3, 3, 2, 130)])
def test_tsvt_parity_4d(gpu_ctx, shape):
    Y = synth.normal(12, 0, int(np.prod(shape))).reshape(shape, order="F")
    sv = slice_singular_values(Y.astype(np.float32))
    allsv = np.sort(np.concatenate([s for s in sv.values()]))
    for q in (0.0, 0.5):
        check_tsvt(gpu_ctx, Y, gap_threshold(allsv, q))


def test_tsvt_lowrank_input(gpu_ctx):
    X = synth.lowrank_tensor(48, 40, 12, 3, seed=3)
    for tau in (0.0, 1.0, 30.0):
        check_tsvt(gpu_ctx, X, tau)


def test_tsvt_video_full_size(gpu_ctx):
    """The 144 x 176 x 100 video at the sizes the benchmark runs, one t-SVT per threshold."""
    X, om = synth.workload_video_completion(seed=1)
    Y = (X * om).astype(np.float32)
    for tau in (100.0, 1.0, 1e-3):
        check_tsvt(gpu_ctx, Y, tau)


@pytest.mark.parametrize("shape,ctas", [((40, 50, 5), 2), ((40, 50, 5), 8), ((50, 40, 4), 4),
                                        ((130, 150, 4), 4), ((64, 80, 3), 2),
                                        ((17, 33, 3, 4), 2), ((260, 270, 3), 8)])
def test_tsvt_parity_cluster_split(shape, ctas):
    """One slice spread over a cluster of 2, 4 or 8 CTAs (blocks of vectors traded between
    CTAs), including ragged blocks padded with zero vectors."""
    from paper_1407_1785_gb300 import libtsvd
    torch = _torch()
    with libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream,
                         ctas_per_slice=ctas) as ctx:
        Y = synth.normal(31, 0, int(np.prod(shape))).reshape(shape, order="F")
        sv = slice_singular_values(Y.astype(np.float32))
        allsv = np.sort(np.concatenate([s for s in sv.values()]))
        for q in (0.0, 0.5):
            check_tsvt(ctx, Y, gap_threshold(allsv, q))


@pytest.mark.parametrize("shape,ctas", [((40, 50, 5), 1), ((130, 150, 4), 4),
                                        ((17, 33, 3, 4), 2), ((144, 176, 6), 2),
                                        ((260, 270, 3), 8)])
def test_tsvt_parity_accumulated_v(shape, ctas):
    """The V-form rebuild (V accumulated during the sweeps)."""
    from paper_1407_1785_gb300 import libtsvd
    torch = _torch()
    with libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream,
                         ctas_per_slice=ctas, accumulate_v=1) as ctx:
        Y = synth.normal(41, 0, int(np.prod(shape))).reshape(shape, order="F")
        sv = slice_singular_values(Y.astype(np.float32))
        allsv = np.sort(np.concatenate([s for s in sv.values()]))
        for q in (0.0, 0.5):
            check_tsvt(ctx, Y, gap_threshold(allsv, q))


def test_autotune_cache_round_trip(tmp_path):
    """The first completion on a new slice shape times the candidate plans and appends the
    winner to the cache file; a second context reads it back instead of re-timing."""
    from paper_1407_1785_gb300 import libtsvd
    torch = _torch()
    cache = str(tmp_path / "tune.txt").encode()
    X, om = synth.workload_lowrank_completion(seed=5, n1=70, n2=90, n3=8, rank=3, p=0.5)
    Mobs = (X * om).astype(np.float32)
    m = dev(Mobs)
    o = torch.from_numpy(colmajor(om, np.uint8)).cuda()
    outs, launches = [], []
    for _ in range(2):
        with libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream,
                             autotune=1, autotune_cache=cache) as ctx:
            x = torch.empty_like(m)
            st = ctx.tnn_complete(m, o, Mobs.shape, 5, x, stats=True)
            outs.append(host(x, Mobs.shape))
            launches.append(st["launches"])
    lines = open(cache.decode()).read().split()
    # gpu, key (n1, n2, distinct slices, V form: on, the warm-started ADMM solve tunes that
    # plan), plan (CTAs, lanes, pairs in flight, block form)
    assert len(lines) == 9 and lines[1:5] == ["70", "90", "5", "1"]
    assert lines[8] in ("0", "1")
    assert launches[1] < launches[0]
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("kind", ["complete", "rpca"])
def test_graph_replay_matches_direct_launches(kind, tmp_path):
    """Calls 1 (direct, autotunes), 2 (captured into a CUDA graph) and 3 (graph replay) agree
    bit for bit with a context that never uses graphs; stats survive the replay.  The two
    contexts share an autotune cache, so both run the plan the first one timed (plans with
    another cluster split order the rotations differently and agree only to rounding)."""
    from paper_1407_1785_gb300 import libtsvd
    torch = _torch()
    cache = str(tmp_path / "tune.txt").encode()
    X, om = synth.workload_lowrank_completion(seed=6, n1=40, n2=52, n3=10, rank=3, p=0.5)
    M = (X * om).astype(np.float32) if kind == "complete" else X.astype(np.float32)
    m = dev(M)
    o = torch.from_numpy(colmajor(om, np.uint8)).cuda()
    outs = []
    for graphs in (0, 1):
        with libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream,
                             use_graphs=graphs, timing=1, autotune_cache=cache) as ctx:
            a, b = torch.empty_like(m), torch.empty_like(m)
            for call in range(3):
                if kind == "complete":
                    st = ctx.tnn_complete(m, o, M.shape, 12, a, b, stats=True)
                else:
                    st = ctx.trpca(m, M.shape, 0.05, 12, a, b, stats=True)
                outs.append((host(a, M.shape), host(b, M.shape)))
                assert st["slice_launches"] == 12
                assert st["slice_ms"] > 0 and st["tube_ms"] > 0
    for x, y in outs[1:]:
        assert np.array_equal(x, outs[0][0]) and np.array_equal(y, outs[0][1])


@pytest.mark.parametrize("persistent", [1, 0])
@pytest.mark.parametrize("warm", ["off", "auto", "on"])
def test_batched_uneven_problems_match_oracle(warm, persistent):
    """A batch of uneven tensors (completion and RPCA, 3-way and 4-way) in one call: every
    tensor matches the oracle's solve, with the warm-started Jacobi off, AUTO (the default,
    warm for every tensor) or ON, as one persistent launch per iteration or
    as per-tensor stream branches (the default); a second call replays the captured batch
    graph and gives the same bits."""
    from paper_1407_1785_gb300 import libtsvd
    warm_start = {"off": libtsvd.WARM_OFF, "auto": libtsvd.WARM_AUTO, "on": libtsvd.WARM_ON}[warm]
    torch = _torch()
    specs = [("complete", (30, 41, 8), 3, 0.4), ("rpca", (52, 36, 6), 2, 0.1),
             ("complete", (64, 20, 11), 4, 0.5), ("rpca", (20, 70, 9), 2, 0.08),
             ("complete", (18, 22, 3, 6), 0, 0.5), ("rpca", (96, 80, 5), 3, 0.12)]
    iters = 25
    probs, refs, keep = [], [], []
    for i, (kind, shape, rank, frac) in enumerate(specs):
        if len(shape) == 3:
            L0 = synth.lowrank_tensor(shape[0], shape[1], shape[2], rank, seed=50 + i)
        else:
            L0 = np.empty(shape)
            for ch in range(shape[2]):
                L0[:, :, ch, :] = synth.translating_texture(shape[0], shape[1], shape[3],
                                                            seed=50 + i, channel=ch)
        if kind == "complete":
            om = synth.sampling_mask(shape, frac, seed=50 + i)
            M = (L0 * om).astype(np.float32)
            Xo, Zo = oracle.tnn_complete(M.astype(np.float64), om, iters)
            refs.append((Xo, Zo))
            q = dict(kind=kind, dims=shape, M=dev(M),
                     omega=torch.from_numpy(colmajor(om, np.uint8)).cuda())
        else:
            S0, _ = synth.sparse_corruption(shape, frac, seed=50 + i)
            M = (L0 + S0).astype(np.float32)
            lam = 1.0 / math.sqrt(max(shape[0], shape[1]) * shape[2])
            Lo, So = oracle.trpca(M.astype(np.float64), lam, iters)
            refs.append((Lo, So))
            q = dict(kind=kind, dims=shape, M=dev(M), lam=lam)
        q["out0"] = torch.empty_like(q["M"])
        q["out1"] = torch.empty_like(q["M"])
        probs.append(q)
        keep.append(M)
    with libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream,
                         warm_start=warm_start, batch_persistent=persistent) as ctx:
        first = None
        for call in range(2):
            st = ctx.solve_batched(probs, iters, stats=True)
            got = [(host(q["out0"], q["dims"]), host(q["out1"], q["dims"])) for q in probs]
            if first is None:
                first = got
            else:
                for (a, b), (c, d) in zip(got, first):
                    assert np.array_equal(a, c) and np.array_equal(b, d)
            # one launch per iteration for the whole batch, or one slice SVT per tensor
            assert st["slice_launches"] == (iters if persistent else iters * len(specs))
            assert st["nonconverged"] == 0
    for (a, b), (ra, rb), M in zip(first, refs, keep):
        assert relerr(a, ra, floor=1e-6) <= ADMM_TOL
        assert relerr(b, rb, floor=1e-3 * np.linalg.norm(M)) <= ADMM_TOL


def test_tsvt_rpca_full_size(gpu_ctx):
    """240 x 320 x 60 tubal-rank-10 tensor plus 10% sparse corruption: slices larger than one
    SM's shared memory, spread over CTA clusters."""
    M, L, S, sup, lam = synth.workload_rpca(seed=1)
    Y = M.astype(np.float32)
    check_tsvt(gpu_ctx, Y, 50.0)


@pytest.mark.slow
def test_tsvt_color_video_full_size(gpu_ctx):
    """288 x 352 x 3 x 60 colour video (2-D DFT over modes 3-4, 93 stored / 91 distinct
    Fourier slices of 288 x 352)."""
    X, om = synth.workload_color_video(seed=1)
    Y = (X * om).astype(np.float32)
    check_tsvt(gpu_ctx, Y, 20.0)


def test_tsvt_deterministic_and_host_path(gpu_ctx):
    Y = synth.normal(5, 0, 30 * 20 * 9).reshape((30, 20, 9), order="F").astype(np.float32)
    Z1, _, _ = gpu_tsvt(gpu_ctx, Y, 0.8)
    Z2, _, _ = gpu_tsvt(gpu_ctx, Y, 0.8)
    assert np.array_equal(Z1, Z2)
    yh = colmajor(Y)
    zh = np.zeros_like(yh)
    gpu_ctx.tsvt(yh, zh, Y.shape, 0.8)                    # host buffers, staged by the library
    assert np.array_equal(uncolmajor(zh, Y.shape), Z1)


# ------------------------------------------------------------------------ completion (Sec. 4)

def gpu_complete(ctx, Mobs, om, iters, stats=False):
    torch = _torch()
    m = dev(Mobs)
    o = torch.from_numpy(colmajor(om, np.uint8)).cuda()
    x = torch.empty_like(m)
    z = torch.empty_like(m)
    st = ctx.tnn_complete(m, o, Mobs.shape, iters, x, z, stats=stats)
    return host(x, Mobs.shape), host(z, Mobs.shape), st


def test_completion_lowrank_parity(gpu_ctx):
    X, om = synth.workload_lowrank_completion(seed=1)
    Mobs = (X * om).astype(np.float32)
    Xo, Zo = oracle.tnn_complete(Mobs.astype(np.float64), om, 100)
    Xg, Zg, st = gpu_complete(gpu_ctx, Mobs, om, 100, stats=True)
    assert np.array_equal(Xg[om == 1], Mobs[om == 1])              # observed entries exact
    assert relerr(Xg, Xo) <= ADMM_TOL
    assert relerr(Zg, Zo) <= ADMM_TOL
    e_g = relerr(Xg, X)
    e_o = relerr(Xo, X)
    assert abs(e_g - e_o) <= 0.01 * e_o + 1e-5, (e_g, e_o)
    assert st["iters"] == 100 and st["nonconverged"] == 0
    assert st["slice_svds"] == 100 * 9


@pytest.mark.parametrize("iters", [0, 1, 2, 5])
def test_completion_short_runs_match_oracle(gpu_ctx, iters):
    X, om = synth.workload_lowrank_completion(seed=4, n1=21, n2=35, n3=9, rank=4, p=0.4)
    Mobs = (X * om).astype(np.float32)
    Xo, Zo = oracle.tnn_complete(Mobs.astype(np.float64), om, iters)
    Xg, Zg, _ = gpu_complete(gpu_ctx, Mobs, om, iters)
    assert relerr(Xg, Xo, floor=1e-6) <= ADMM_TOL
    assert relerr(Zg, Zo, floor=1e-3 * np.linalg.norm(Mobs)) <= ADMM_TOL
    assert np.array_equal(Xg[om == 1], Mobs[om == 1])


def test_completion_4d_parity(gpu_ctx):
    shape = (20, 18, 3, 8)
    X = np.empty(shape)
    for c in range(3):
        X[:, :, c, :] = synth.translating_texture(20, 18, 8, seed=2, channel=c)
    om = synth.sampling_mask(shape, 0.3, seed=2)
    Mobs = (X * om).astype(np.float32)
    Xo, Zo = oracle.tnn_complete(Mobs.astype(np.float64), om, 40)
    Xg, Zg, _ = gpu_complete(gpu_ctx, Mobs, om, 40)
    assert relerr(Xg, Xo) <= ADMM_TOL
    assert np.array_equal(Xg[om == 1], Mobs[om == 1])
    e_g, e_o = relerr(Xg, X), relerr(Xo, X)
    assert abs(e_g - e_o) <= 0.01 * e_o + 1e-5


def test_completion_video_full_size_short(gpu_ctx):
    """Full benchmark size, first iterations compared entry by entry with the oracle."""
    X, om = synth.workload_video_completion(seed=1)
    Mobs = (X * om).astype(np.float32)
    Xo, Zo = oracle.tnn_complete(Mobs.astype(np.float64), om, 3)
    Xg, Zg, _ = gpu_complete(gpu_ctx, Mobs, om, 3)
    assert relerr(Xg, Xo) <= ADMM_TOL
    assert relerr(Zg, Zo, floor=1e-3 * np.linalg.norm(Mobs)) <= ADMM_TOL


def test_completion_video_full_run_properties(gpu_ctx):
    """The full 150-iteration benchmark run: properties that hold at any size."""
    X, om = synth.workload_video_completion(seed=1)
    Mobs = (X * om).astype(np.float32)
    Xg, Zg, st = gpu_complete(gpu_ctx, Mobs, om, 150, stats=True)
    assert np.all(np.isfinite(Xg))
    assert np.array_equal(Xg[om == 1], Mobs[om == 1])
    assert st["nonconverged"] == 0
    # the penalty grew as min(1.1^k rho0, rho_max)
    assert st["rho_final"] == pytest.approx(1e-2 * 1.1 ** 150, rel=1e-9)
    # completion beats the zero fill by a wide margin on the unobserved entries
    un = om == 0
    e_fill = np.linalg.norm(X[un])
    e_rec = np.linalg.norm((Xg - X)[un])
    assert e_rec < 0.2 * e_fill
    # X and Z agree at convergence (primal residual)
    assert relerr(Xg, Zg) < 0.05


# ------------------------------------------------------------------------ RPCA (Sec. 5)

def gpu_rpca(ctx, M, lam, iters, stats=False):
    torch = _torch()
    m = dev(M)
    l = torch.empty_like(m)
    s = torch.empty_like(m)
    st = ctx.trpca(m, M.shape, lam, iters, l, s, stats=stats)
    return host(l, M.shape), host(s, M.shape), st


@pytest.mark.parametrize("iters", [0, 1, 3, 60])
def test_rpca_entry_parity(gpu_ctx, iters):
    L0 = synth.lowrank_tensor(24, 20, 8, 2, seed=9)
    S0, _ = synth.sparse_corruption(L0.shape, 0.1, seed=9)
    M = (L0 + S0).astype(np.float32)
    lam = 1.0 / math.sqrt(24 * 8)
    Lo, So = oracle.trpca(M.astype(np.float64), lam, iters)
    Lg, Sg, _ = gpu_rpca(gpu_ctx, M, lam, iters)
    assert relerr(Lg, Lo, floor=1e-6) <= ADMM_TOL
    assert relerr(Sg, So, floor=1e-3 * np.linalg.norm(M)) <= ADMM_TOL
    mism = np.count_nonzero((Sg != 0) != (So != 0))
    assert mism <= 1e-3 * M.size


@pytest.mark.parametrize("iters", [1, 40])
def test_rpca_tube_mode_parity(iters):
    from paper_1407_1785_gb300 import libtsvd
    torch = _torch()
    ctx = libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream,
                          sparse_mode=libtsvd.SPARSE_TUBE)
    try:
        L0 = synth.lowrank_tensor(22, 18, 10, 2, seed=10)
        S0, _ = synth.tube_corruption(L0.shape, 0.08, seed=10, block=5, std=3.0)
        M = (L0 + S0).astype(np.float32)
        lam = 1.0 / math.sqrt(22)
        Lo, So = oracle.trpca(M.astype(np.float64), lam, iters, sparse_mode=oracle.SPARSE_TUBE)
        Lg, Sg, _ = gpu_rpca(ctx, M, lam, iters)
        assert relerr(Lg, Lo) <= ADMM_TOL
        assert relerr(Sg, So, floor=1e-3 * np.linalg.norm(M)) <= ADMM_TOL
        tg = np.linalg.norm(Sg, axis=2) > 0
        to = np.linalg.norm(So, axis=2) > 0
        assert np.count_nonzero(tg != to) <= 2
    finally:
        ctx.close()


def _tube_ctx():
    from paper_1407_1785_gb300 import libtsvd
    torch = _torch()
    return libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream,
                           sparse_mode=libtsvd.SPARSE_TUBE)


def test_rpca_tube_video_full_size_short():
    """The tube-sparse RPCA workload at full size (144 x 256 x 80 panning video, 10% of the
    pixel tubes corrupted in 10-frame blocks, lambda = 1/sqrt(max(n1, n2))): the first
    iterations entry by entry against the oracle, and the same corrupted tubes."""
    M, L0, S0, sup, lam = synth.workload_rpca_tube(seed=1)
    M = M.astype(np.float32)
    Lo, So = oracle.trpca(M.astype(np.float64), lam, 3, sparse_mode=oracle.SPARSE_TUBE)
    with _tube_ctx() as ctx:
        Lg, Sg, _ = gpu_rpca(ctx, M, lam, 3)
    assert relerr(Lg, Lo) <= ADMM_TOL
    assert relerr(Sg, So, floor=1e-3 * np.linalg.norm(M)) <= ADMM_TOL
    tg = np.linalg.norm(Sg, axis=2) > 0
    to = np.linalg.norm(So, axis=2) > 0
    assert np.count_nonzero(tg != to) <= 1e-3 * tg.size


def test_rpca_tube_video_full_run_properties():
    """The full 200-iteration tube-sparse RPCA run: properties that hold at any size (on a
    48 x 64 x 40 instance the oracle reaches -27.7 dB from -2.6 dB and finds every corrupted
    tube)."""
    M, L0, S0, sup, lam = synth.workload_rpca_tube(seed=1)
    M = M.astype(np.float32)
    with _tube_ctx() as ctx:
        Lg, Sg, st = gpu_rpca(ctx, M, lam, 200, stats=True)
    assert np.all(np.isfinite(Lg)) and np.all(np.isfinite(Sg))
    assert st["nonconverged"] == 0
    db = lambda e: 20 * math.log10(e)
    assert db(relerr(Lg, L0)) <= db(relerr(M, L0)) - 20.0
    # every corrupted tube carries sparse energy (the l_{1,1,2} group is the whole tube)
    det = np.linalg.norm(Sg, axis=2) > 0
    assert np.all(det[sup.any(axis=2)])
    # L + S reproduces M (the sparse step's residual is the scaled dual, small at the end)
    assert relerr(Lg + Sg, M) < 1e-4


def test_rpca_4d_parity(gpu_ctx):
    shape = (12, 10, 3, 6)
    L0 = synth.normal(13, 0, int(np.prod(shape))).reshape(shape, order="F")
    L0 = oracle.tsvt(L0, 4.0)                       # a low multi-rank 4-way tensor
    S0, _ = synth.sparse_corruption(shape, 0.1, seed=13)
    M = (L0 + S0).astype(np.float32)
    lam = 1.0 / math.sqrt(12 * 18)
    Lo, So = oracle.trpca(M.astype(np.float64), lam, 30)
    Lg, Sg, _ = gpu_rpca(gpu_ctx, M, lam, 30)
    assert relerr(Lg, Lo) <= ADMM_TOL


@pytest.mark.parametrize("shape,ctas", [((40, 30, 9), 0), ((30, 44, 8), 0), ((70, 60, 6), 4),
                                        ((60, 72, 5), 8)])
@pytest.mark.parametrize("kind", ["complete", "rpca"])
def test_warm_start_matches_oracle_and_cold(shape, ctas, kind):
    """Warm-started slice SVDs (pre-rotation to B V or V^T B, a cold restart every 64
    iterations, U-form rebuild from B, one CTA or a cluster per slice) reach the oracle's
    iterates like the cold solve; 70 iterations include one mid-solve cold restart."""
    iters = 70
    from paper_1407_1785_gb300 import libtsvd
    torch = _torch()
    n1, n2, n3 = shape
    if kind == "complete":
        X, om = synth.workload_lowrank_completion(seed=6, n1=n1, n2=n2, n3=n3, rank=3, p=0.4)
        M = (X * om).astype(np.float32)
        Ro, _ = oracle.tnn_complete(M.astype(np.float64), om, iters)
    else:
        X = synth.lowrank_tensor(n1, n2, n3, 2, seed=6)
        S0, _ = synth.sparse_corruption(X.shape, 0.1, seed=6)
        M = (X + S0).astype(np.float32)
        lam = 1.0 / math.sqrt(max(n1, n2) * n3)
        Ro, _ = oracle.trpca(M.astype(np.float64), lam, iters)
    out = {}
    for warm in (libtsvd.WARM_OFF, libtsvd.WARM_ON):
        ctx = libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream,
                              warm_start=warm, ctas_per_slice=ctas)
        try:
            if kind == "complete":
                R, _, st = gpu_complete(ctx, M, om, iters, stats=True)
            else:
                R, _, st = gpu_rpca(ctx, M, lam, iters, stats=True)
        finally:
            ctx.close()
        out[warm] = (R, st)
        assert relerr(R, Ro) <= ADMM_TOL, (warm, relerr(R, Ro))
        assert st["nonconverged"] == 0
    (Rc, sc), (Rw, sw) = out[libtsvd.WARM_OFF], out[libtsvd.WARM_ON]
    e_c, e_w = relerr(Rc, X), relerr(Rw, X)
    assert e_w <= 1.01 * e_c + 1e-5, (e_w, e_c)
    assert sw["total_sweeps"] < sc["total_sweeps"]


# ------------------------------------------------------------------------ error paths

def test_invalid_arguments(gpu_ctx):
    from paper_1407_1785_gb300 import libtsvd
    torch = _torch()
    m = torch.zeros(4 * 4 * 4, device="cuda")
    om = torch.ones(4 * 4 * 4, dtype=torch.uint8, device="cuda")
    x = torch.empty_like(m)
    assert gpu_ctx.raw_tnn_complete(m, om, 7, (4, 4, 4, 1, 1, 1, 1), 3, x) == libtsvd.TSVD_EINVAL
    assert gpu_ctx.raw_tnn_complete(m, om, 3, (4, 0, 4), 3, x) == libtsvd.TSVD_EINVAL
    assert gpu_ctx.raw_tnn_complete(m, om, 3, (4, 4, 4), -1, x) == libtsvd.TSVD_EINVAL
    m[5] = float("nan")
    assert gpu_ctx.raw_tnn_complete(m, om, 3, (4, 4, 4), 3, x) == libtsvd.TSVD_EINVAL
    assert "not finite" in gpu_ctx.last_error()
    om[5] = 0                                   # a NaN at an unobserved entry is ignored
    assert gpu_ctx.raw_tnn_complete(m, om, 3, (4, 4, 4), 3, x) == libtsvd.TSVD_OK
    with pytest.raises(libtsvd.TsvdError):
        gpu_ctx.tsvt(m, x, (4, 4, 4), -1.0)


def test_unsupported_slice_is_reported(gpu_ctx):
    from paper_1407_1785_gb300 import libtsvd
    torch = _torch()
    shape = (600, 700, 2)
    m = torch.zeros(int(np.prod(shape)), device="cuda")
    z = torch.empty_like(m)
    with pytest.raises(libtsvd.TsvdError) as ei:
        gpu_ctx.tsvt(m, z, shape, 1.0)
    assert ei.value.status == libtsvd.TSVD_EUNSUPPORTED
