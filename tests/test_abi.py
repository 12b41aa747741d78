"""The C-ABI library loads and exports every symbol include/tsvd.h declares (CPU only: no
compute call is made here)."""
import ctypes
import os
import re

import pytest

from paper_1407_1785_gb300 import libtsvd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(inc, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b([A-Za-z_]\w*)\s*\([^;{]*\)\s*;", text,
                             flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_expected_api():
    names = declared_functions()
    assert {"tsvd_create", "tsvd_destroy", "tsvd_last_error", "tsvt", "tnn_complete",
            "trpca", "tsvd_default_opts"} <= names
    assert names == set(libtsvd.EXPORTED_SYMBOLS)


def test_library_exports_every_declared_symbol():
    L = libtsvd.load()
    for name in declared_functions():
        assert hasattr(L, name), name
        assert getattr(L, name) is not None


def test_default_opts():
    o = libtsvd.default_opts()
    assert o.precision == libtsvd.PRECISION_FP32
    assert o.sparse_mode == libtsvd.SPARSE_ENTRY
    assert o.tnn_scale == libtsvd.SCALE_AVG
    assert o.rho0 == pytest.approx(1e-2)
    assert o.mu == pytest.approx(1.1)
    assert o.rho_max == pytest.approx(1e10)
    assert o.max_sweeps == 40
    assert o.jacobi_tol == pytest.approx(1e-6)
    assert (o.rsvt_oversample, o.rsvt_kmax, o.rsvt_power) == (10, 0, 2)
    assert o.warm_start == libtsvd.WARM_AUTO


def test_null_arguments_are_rejected_without_touching_a_device():
    L = libtsvd.load()
    assert L.tsvd_create(None, 0, None, None) == libtsvd.TSVD_EINVAL
    assert L.tsvd_destroy(None) == libtsvd.TSVD_OK
    assert L.tsvd_last_error(None) == b"no context"
    dims = (ctypes.c_int64 * 3)(4, 4, 4)
    assert L.tsvt(None, None, None, 3, dims, 1.0, None, None) == libtsvd.TSVD_EINVAL
    assert L.tsvd_factor(None, None, 3, dims, 0, None, None, None) == libtsvd.TSVD_EINVAL
    assert L.tsvd_compress(None, None, 3, dims, 1, 1, None, None, None) == libtsvd.TSVD_EINVAL
    assert L.tsvd_tproduct(None, None, None, None, 3, dims, 4) == libtsvd.TSVD_EINVAL
    assert L.tnn_complete(None, None, None, 3, dims, 1, None, None, None) == libtsvd.TSVD_EINVAL
    assert L.trpca(None, None, 3, dims, 1.0, 1, None, None, None) == libtsvd.TSVD_EINVAL


def test_bad_options_rejected():
    L = libtsvd.load()
    o = libtsvd.default_opts()
    o.mu = 0.5
    h = ctypes.c_void_p()
    assert L.tsvd_create(ctypes.byref(h), 0, None, ctypes.byref(o)) == libtsvd.TSVD_EINVAL
    for field, bad in (("precision", 5), ("precision", -1), ("rsvt_oversample", -1),
                       ("rsvt_oversample", 65), ("rsvt_kmax", -3), ("rsvt_power", 9),
                       ("warm_start", 3), ("warm_start", -1), ("ctas_per_slice", 3),
                       ("ctas_per_slice", -2), ("jacobi_stop", 2), ("jacobi_stop", -1)):
        o = libtsvd.default_opts()
        setattr(o, field, bad)
        assert L.tsvd_create(ctypes.byref(h), 0, None, ctypes.byref(o)) == libtsvd.TSVD_EINVAL
    assert not h.value


def test_create_without_gpu_reports_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = libtsvd.load()
    h = ctypes.c_void_p()
    assert L.tsvd_create(ctypes.byref(h), 0, None, None) == libtsvd.TSVD_ECUDA
    assert not h.value
    # valid non-default values pass the option checks and fail only at the device
    for field, val in (("ctas_per_slice", libtsvd.CTAS_FEWEST), ("ctas_per_slice", 8),
                       ("jacobi_stop", libtsvd.STOP_RELATIVE), ("warm_start", libtsvd.WARM_OFF)):
        o = libtsvd.default_opts()
        setattr(o, field, val)
        assert L.tsvd_create(ctypes.byref(h), 0, None, ctypes.byref(o)) == libtsvd.TSVD_ECUDA
        assert not h.value


def test_library_is_the_in_tree_build():
    assert os.path.commonpath([libtsvd.library_path(), ROOT]) == ROOT
    assert os.path.exists(libtsvd.library_path())


def test_fault_injection_spec_parsing():
    """TSVD_FAULT specs: "alloc:N" with N >= 1 turns the N-th device allocation into a failure;
    anything else is off (0).  Needs no GPU."""
    from paper_1407_1785_gb300 import libtsvd
    try:
        assert libtsvd.fault_injection_reset("alloc:3") == 3
        assert libtsvd.fault_injection_reset("alloc:1") == 1
        for bad in ("alloc:0", "alloc:-2", "alloc:", "alloc:3x", "free:1", ""):
            assert libtsvd.fault_injection_reset(bad) == 0, bad
    finally:
        libtsvd.fault_injection_reset("")
