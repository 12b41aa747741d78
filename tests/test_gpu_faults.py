"""Failure paths driven without a GPU fault: host-side fault injection of a device allocation
(TSVD_ENOMEM, the context usable afterwards) and the persistent kernel's bounded wait run on a
counter nothing raises (TSVD_ETIMEOUT, the device usable afterwards)."""
import numpy as np
import pytest

from helpers import colmajor, relerr, uncolmajor

import oracle
from paper_1407_1785_gb300 import libtsvd, synth

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def test_injected_allocation_failure_reports_enomem_and_recovers():
    torch = _torch()
    Y = synth.normal(41, 0, 30 * 20 * 6).reshape((30, 20, 6), order="F").astype(np.float32)
    y = torch.from_numpy(colmajor(Y)).cuda()
    z = torch.empty_like(y)
    try:
        # the next device allocation of the library fails
        assert libtsvd.fault_injection_reset("alloc:1") == 1
        with libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream) as ctx:
            with pytest.raises(libtsvd.TsvdError) as ei:
                ctx.tsvt(y, z, Y.shape, 1.0)
            assert ei.value.status == libtsvd.TSVD_ENOMEM
            assert "cudaMalloc" in ctx.last_error()
            # the same context then allocates and computes normally
            ctx.tsvt(y, z, Y.shape, 1.0)
            torch.cuda.synchronize()
            Zg = uncolmajor(z.cpu().numpy(), Y.shape)
    finally:
        libtsvd.fault_injection_reset("")
    Zo = oracle.tsvt(Y.astype(np.float64), 1.0)
    assert relerr(Zg, Zo, floor=1e-3 * np.linalg.norm(Y)) <= 2e-5


def test_bounded_wait_gives_up_and_device_stays_usable():
    torch = _torch()
    assert libtsvd.selftest_bounded_wait(0, 50) == libtsvd.TSVD_ETIMEOUT
    assert libtsvd.selftest_bounded_wait(0, 0) == libtsvd.TSVD_ETIMEOUT
    # the device still runs work
    a = torch.arange(1000, device="cuda", dtype=torch.float32)
    assert float(a.sum().item()) == 499500.0
    with libtsvd.Context(device=0, stream=torch.cuda.current_stream().cuda_stream) as ctx:
        Y = synth.normal(42, 0, 16 * 12 * 4).reshape((16, 12, 4), order="F").astype(np.float32)
        y = torch.from_numpy(colmajor(Y)).cuda()
        z = torch.empty_like(y)
        ctx.tsvt(y, z, Y.shape, 0.5)
    assert libtsvd.selftest_bounded_wait(0, -1) == libtsvd.TSVD_EINVAL
