"""tsvt_static(): the t-SVT for callers that cannot allocate device memory (a process whose
device memory belongs to its own pool allocator, or a loop that must not pay cudaMalloc's
implicit synchronisation).  Its scratch is a fixed array inside the library; the test checks
it through the C ABI against tsvt(), which allocates its own workspace, and against the FP64
oracle's t-SVT (Lemma of Sec. 4.1 per Fourier slice), and checks that a repeated call takes
no device memory.

This file is collected last on purpose, so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

from helpers import colmajor, relerr, uncolmajor

import oracle
from paper_1407_1785_gb300 import libtsvd, synth

pytestmark = pytest.mark.gpu

TSVT_TOL = 2e-5      # the per-call t-SVT tolerance of the parity tests


def _run_pair(ctx, torch, shape, seed, tau):
    Y = synth.normal(seed, 0, int(np.prod(shape))).reshape(shape, order="F").astype(np.float32)
    stream = torch.cuda.current_stream()
    y = torch.from_numpy(colmajor(Y)).cuda()
    z_ref = torch.empty_like(y)
    ctx.tsvt(y, z_ref, shape, tau)
    z = torch.full_like(y, float("nan"))
    st = libtsvd.tsvt_static(y, z, shape, tau, stream.cuda_stream)
    assert st == libtsvd.TSVD_OK
    torch.cuda.synchronize()
    Zr = uncolmajor(z_ref.cpu().numpy(), shape)
    Zs = uncolmajor(z.cpu().numpy(), shape)
    floor = 1e-3 * np.linalg.norm(Y)
    assert np.all(np.isfinite(Zs))
    assert relerr(Zs, Zr, floor=floor) <= TSVT_TOL
    Zo = oracle.tsvt(Y.astype(np.float64), tau)
    Zo_floor = max(np.linalg.norm(Zo), floor)
    assert relerr(Zs, Zo, floor=Zo_floor) <= TSVT_TOL
    # the same call again: the scratch address is cached and the kernels are loaded, so a
    # call that allocated device memory would show as a drop of the free memory
    free0 = torch.cuda.mem_get_info()[0]
    st = libtsvd.tsvt_static(y, z, shape, tau, stream.cuda_stream)
    torch.cuda.synchronize()
    assert st == libtsvd.TSVD_OK
    assert torch.cuda.mem_get_info()[0] >= free0
    assert np.array_equal(uncolmajor(z.cpu().numpy(), shape), Zs)


def test_static_scratch_tsvt_matches_tsvt():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    with libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream) as ctx:
        # two calls in a row on different shapes: the second must not depend on what the
        # first left in the shared scratch
        _run_pair(ctx, torch, (40, 28, 12), seed=21, tau=2.0)
        _run_pair(ctx, torch, (17, 33, 3, 5), seed=22, tau=1.0)
        _run_pair(ctx, torch, (144, 176, 100), seed=23, tau=5.0)
        # back to the first shape after the large one left its spectra in the array
        _run_pair(ctx, torch, (40, 28, 12), seed=24, tau=2.0)


def test_static_scratch_rejects_oversize_and_host_buffers():
    torch = pytest.importorskip("torch")
    y = torch.zeros(8, device="cuda")
    # 144 x 176 x 400: 2 spectra of 201 slices x 198 KiB = 81.5 MB > 64 MiB (the slices
    # themselves fit the kernels, so only the scratch limit rejects it)
    assert libtsvd.tsvt_static(y, y, (144, 176, 400), 1.0) == libtsvd.TSVD_ENOMEM
    h = np.zeros(4 * 4 * 4, np.float32)
    assert libtsvd.tsvt_static(h, h, (4, 4, 4), 1.0) == libtsvd.TSVD_EINVAL
    assert libtsvd.tsvt_static(y, y, (2, 2, 2), -1.0) == libtsvd.TSVD_EINVAL


def test_static_scratch_tsvt_is_capturable():
    """After a first call outside capture (the scratch address lookup), tsvt_static can be
    captured into a CUDA graph: its tables are written on the device from launch arguments,
    so a replay reads no host memory; replays follow new contents of the input buffer."""
    torch = pytest.importorskip("torch")
    shape, tau = (40, 28, 12), 2.0
    Y = synth.normal(25, 0, int(np.prod(shape))).reshape(shape, order="F").astype(np.float32)
    y = torch.from_numpy(colmajor(Y)).cuda()
    z = torch.empty_like(y)
    assert libtsvd.tsvt_static(y, z, shape, tau, torch.cuda.current_stream().cuda_stream) == \
        libtsvd.TSVD_OK
    torch.cuda.synchronize()
    Z1 = uncolmajor(z.cpu().numpy(), shape)
    zg = torch.full_like(y, float("nan"))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="thread_local"):
        st = libtsvd.tsvt_static(y, zg, shape, tau, torch.cuda.current_stream().cuda_stream)
    assert st == libtsvd.TSVD_OK
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(uncolmajor(zg.cpu().numpy(), shape), Z1)
    y.mul_(3.0)
    g.replay()
    torch.cuda.synchronize()
    Zo = oracle.tsvt(3.0 * Y.astype(np.float64), tau)
    Zg = uncolmajor(zg.cpu().numpy(), shape)
    assert relerr(Zg, Zo, floor=max(np.linalg.norm(Zo), 3e-3 * np.linalg.norm(Y))) <= TSVT_TOL
