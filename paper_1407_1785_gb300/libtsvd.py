"""Thin ctypes binding of libtsvd (include/tsvd.h).

Only argument marshalling lives here: every step of the t-SVT and of the ADMM solvers runs
in the CUDA kernels of ``libtsvd.so``.  There is no CPU fallback; if the shared library is
missing or fails to load, importing this module raises.

Tensors are passed as 1-D contiguous buffers in MATLAB column-major order (see
``synth.to_colmajor``): CUDA tensors (torch) are used in place on the context's stream,
host tensors (numpy arrays or CPU torch tensors, pinned or not) are staged by the library.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

TSVD_OK, TSVD_EINVAL, TSVD_ENOMEM, TSVD_ECUDA, TSVD_ENOTCONV = 0, 1, 2, 3, 4
TSVD_ETIMEOUT, TSVD_EUNSUPPORTED = 5, 6
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOTCONV", 5: "ETIMEOUT",
                6: "EUNSUPPORTED"}
PRECISION_FP32, PRECISION_TF32, PRECISION_BF16, PRECISION_3XTF32 = 0, 1, 2, 3
PRECISION_RAND_FP32 = 4
SPARSE_ENTRY, SPARSE_TUBE = 0, 1
SCALE_AVG, SCALE_SUM = 0, 1

# Every symbol include/tsvd.h declares.
EXPORTED_SYMBOLS = ("tsvd_default_opts", "tsvd_create", "tsvd_destroy", "tsvd_last_error",
                    "tsvt", "tsvd_factor", "tsvd_compress", "tsvd_tproduct", "tnn_complete",
                    "trpca",
                    "tsvd_solve_batched", "tnn_complete_batched", "trpca_batched",
                    "tsvt_static", "tsvd_cgemm", "tsvd_measure_fp32_peak",
                    "tsvd_fault_injection_reset", "tsvd_selftest_bounded_wait",
                    "tnn_complete_resume", "trpca_resume")
OP_N, OP_T, OP_C = 0, 1, 2
WARM_OFF, WARM_ON, WARM_AUTO = 0, 1, 2
SLICE_AUTO, SLICE_PAIRWISE, SLICE_BLOCK = 0, 1, 2
STOP_SVT, STOP_RELATIVE = 0, 1
CTAS_FEWEST = -1
COMPRESS_GLOBAL, COMPRESS_TUBAL = 1, 2
PROBLEM_COMPLETE, PROBLEM_RPCA = 1, 2


class Problem(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("order", ctypes.c_int),
                ("dims", ctypes.c_int64 * 4), ("M", ctypes.c_void_p),
                ("omega", ctypes.c_void_p), ("lam", ctypes.c_float),
                ("out0", ctypes.c_void_p), ("out1", ctypes.c_void_p)]


class AdmmState(ctypes.Structure):
    _fields_ = [("Z", ctypes.c_void_p), ("Q", ctypes.c_void_p), ("S", ctypes.c_void_p),
                ("W", ctypes.c_void_p), ("rho", ctypes.c_double)]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("sparse_mode", ctypes.c_int),
                ("tnn_scale", ctypes.c_int), ("rho0", ctypes.c_double),
                ("mu", ctypes.c_double), ("rho_max", ctypes.c_double),
                ("max_sweeps", ctypes.c_int), ("jacobi_tol", ctypes.c_float),
                ("timing", ctypes.c_int), ("ctas_per_slice", ctypes.c_int),
                ("accumulate_v", ctypes.c_int), ("lanes_per_pair", ctypes.c_int),
                ("autotune", ctypes.c_int), ("autotune_cache", ctypes.c_char_p),
                ("use_graphs", ctypes.c_int), ("rsvt_oversample", ctypes.c_int),
                ("rsvt_kmax", ctypes.c_int), ("rsvt_power", ctypes.c_int),
                ("warm_start", ctypes.c_int), ("batch_persistent", ctypes.c_int),
                ("slice_form", ctypes.c_int), ("rsvt_small_fp64", ctypes.c_int),
                ("jacobi_stop", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("max_sweeps_used", ctypes.c_int),
                ("total_sweeps", ctypes.c_int64), ("nonconverged", ctypes.c_int64),
                ("slice_svds", ctypes.c_int64), ("rho_final", ctypes.c_double),
                ("tnn_last", ctypes.c_double), ("rank_last_max", ctypes.c_int),
                ("launches", ctypes.c_int64), ("slice_launches", ctypes.c_int64),
                ("slice_ms", ctypes.c_double), ("tube_ms", ctypes.c_double),
                ("slice_ctas", ctypes.c_int), ("slice_lanes", ctypes.c_int),
                ("slice_pairs_in_flight", ctypes.c_int), ("rsvt_k_last", ctypes.c_int),
                ("rsvt_saturated", ctypes.c_int64), ("rsvt_drops", ctypes.c_int64),
                ("rsvt_gemm_ms", ctypes.c_double), ("rsvt_orth_ms", ctypes.c_double),
                ("rsvt_svd_ms", ctypes.c_double), ("rsvt_gemm_gflop", ctypes.c_double),
                ("rsvt_svd_gflop", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class TsvdError(RuntimeError):
    def __init__(self, fn: str, status: int, msg: str):
        super().__init__(f"{fn} failed: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libtsvd.so (building it first if it is missing and nvcc is available)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB_PATH):
        if not build_if_missing:
            raise ImportError(f"libtsvd.so not found at {_build.LIB_PATH}")
        _build.build()
    L = ctypes.CDLL(_build.LIB_PATH)
    P = ctypes.c_void_p
    i64p = ctypes.POINTER(ctypes.c_int64)
    L.tsvd_default_opts.argtypes = [ctypes.POINTER(Opts)]
    L.tsvd_default_opts.restype = None
    L.tsvd_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, P, ctypes.POINTER(Opts)]
    L.tsvd_create.restype = ctypes.c_int
    L.tsvd_destroy.argtypes = [P]
    L.tsvd_destroy.restype = ctypes.c_int
    L.tsvd_last_error.argtypes = [P]
    L.tsvd_last_error.restype = ctypes.c_char_p
    L.tsvt.argtypes = [P, P, P, ctypes.c_int, i64p, ctypes.c_float, P, P]
    L.tsvt.restype = ctypes.c_int
    L.tsvd_factor.argtypes = [P, P, ctypes.c_int, i64p, ctypes.c_int, P, P, P]
    L.tsvd_factor.restype = ctypes.c_int
    L.tsvd_compress.argtypes = [P, P, ctypes.c_int, i64p, ctypes.c_int, ctypes.c_int64, P,
                                ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]
    L.tsvd_compress.restype = ctypes.c_int
    L.tsvd_tproduct.argtypes = [P, P, P, P, ctypes.c_int, i64p, ctypes.c_int64]
    L.tsvd_tproduct.restype = ctypes.c_int
    L.tnn_complete.argtypes = [P, P, P, ctypes.c_int, i64p, ctypes.c_int, P, P,
                               ctypes.POINTER(Stats)]
    L.tnn_complete.restype = ctypes.c_int
    L.trpca.argtypes = [P, P, ctypes.c_int, i64p, ctypes.c_float, ctypes.c_int, P, P,
                        ctypes.POINTER(Stats)]
    L.trpca.restype = ctypes.c_int
    L.tnn_complete_resume.argtypes = [P, P, P, ctypes.c_int, i64p, ctypes.c_int,
                                      ctypes.POINTER(AdmmState), P, P, P, ctypes.POINTER(Stats)]
    L.tnn_complete_resume.restype = ctypes.c_int
    L.trpca_resume.argtypes = [P, P, ctypes.c_int, i64p, ctypes.c_float, ctypes.c_int,
                               ctypes.POINTER(AdmmState), P, P, P, ctypes.POINTER(Stats)]
    L.trpca_resume.restype = ctypes.c_int
    L.tsvt_static.argtypes = [P, P, ctypes.c_int, i64p, ctypes.c_float, P]
    L.tsvt_static.restype = ctypes.c_int
    L.tsvd_solve_batched.argtypes = [P, ctypes.c_int, ctypes.POINTER(Problem), ctypes.c_int,
                                     ctypes.POINTER(Stats)]
    L.tsvd_solve_batched.restype = ctypes.c_int
    for name in ("tnn_complete_batched", "trpca_batched"):
        getattr(L, name).argtypes = L.tsvd_solve_batched.argtypes
        getattr(L, name).restype = ctypes.c_int
    L.tsvd_measure_fp32_peak.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double)]
    L.tsvd_measure_fp32_peak.restype = ctypes.c_int
    L.tsvd_fault_injection_reset.argtypes = [ctypes.c_char_p]
    L.tsvd_fault_injection_reset.restype = ctypes.c_longlong
    L.tsvd_selftest_bounded_wait.argtypes = [ctypes.c_int, ctypes.c_int]
    L.tsvd_selftest_bounded_wait.restype = ctypes.c_int
    i64 = ctypes.c_int64
    L.tsvd_cgemm.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                             ctypes.c_int, P, i64, i64, P, i64, i64, P, i64, i64, ctypes.c_int]
    L.tsvd_cgemm.restype = ctypes.c_int
    _lib = L
    return L


def tsvt_static(Y, Z, dims: Sequence[int], tau: float, stream: Optional[int] = None) -> int:
    """t-SVT with the library's fixed device scratch (no device allocation).  Y and Z are
    device buffers on the current device; returns the tsvd_status code."""
    return load().tsvt_static(_ptr(Y), _ptr(Z), len(dims), _dims(dims), float(tau),
                              ctypes.c_void_p(stream or 0))


def measure_fp32_peak(device: int = 0):
    """Measured FP32 CUDA-core throughput (TFLOP/s) of the device: (scalar FMA loop, packed
    FP32x2 FMA loop).  Raises on failure."""
    a, b = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = load().tsvd_measure_fp32_peak(int(device), ctypes.byref(a), ctypes.byref(b))
    if st != TSVD_OK:
        raise TsvdError("tsvd_measure_fp32_peak", st, "measurement failed")
    return a.value, b.value


def fault_injection_reset(spec: Optional[str] = None) -> int:
    """Host-side fault injection ("alloc:N": the N-th device allocation of the library fails);
    None re-reads the TSVD_FAULT environment variable.  Returns N (0 = off)."""
    return int(load().tsvd_fault_injection_reset(spec.encode() if spec is not None else None))


def selftest_bounded_wait(device: int = 0, limit_ms: int = 50) -> int:
    """Runs the persistent kernel's bounded wait on a counter nothing raises; returns the
    status (TSVD_ETIMEOUT when the wait gave up, as it must)."""
    return int(load().tsvd_selftest_bounded_wait(int(device), int(limit_ms)))


def default_opts() -> Opts:
    o = Opts()
    load().tsvd_default_opts(ctypes.byref(o))
    return o


def _ptr(x) -> Optional[int]:
    """Raw address of a tensor / array buffer (None stays None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):          # torch.Tensor
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported buffer type {type(x)}")


def _dims(dims: Sequence[int]):
    return (ctypes.c_int64 * len(dims))(*[int(d) for d in dims])


class Context:
    """A libtsvd context bound to one device and one CUDA stream."""

    def __init__(self, device: int = 0, stream: Optional[int] = None, **opts):
        L = load()
        o = default_opts()
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            if isinstance(v, str):   # autotune_cache: a path
                v = os.fsencode(v)
            setattr(o, k, v)
        h = ctypes.c_void_p()
        st = L.tsvd_create(ctypes.byref(h), int(device), ctypes.c_void_p(stream or 0),
                           ctypes.byref(o))
        if st != TSVD_OK:
            raise TsvdError("tsvd_create", st, "cannot create context")
        self._h = h
        self._L = L
        self.opts = o

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.tsvd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def last_error(self) -> str:
        return self._L.tsvd_last_error(self._h).decode()

    def _check(self, fn: str, st: int, allow=(TSVD_OK,)) -> int:
        if st not in allow:
            raise TsvdError(fn, st, self.last_error())
        return st

    def tsvt(self, Y, Z, dims: Sequence[int], tau: float, multirank=None, with_tnn=False,
             allow_notconv: bool = False):
        """t-SVT of Y into Z.  Returns (status, tnn or None)."""
        tnn = ctypes.c_double(0.0)
        st = self._L.tsvt(self._h, _ptr(Y), _ptr(Z), len(dims), _dims(dims), float(tau),
                          _ptr(multirank), ctypes.byref(tnn) if with_tnn else None)
        allow = (TSVD_OK, TSVD_ENOTCONV) if allow_notconv else (TSVD_OK,)
        self._check("tsvt", st, allow)
        return st, (tnn.value if with_tnn else None)

    def factor(self, Y, dims: Sequence[int], k: int, U, S, V):
        """Truncated t-SVD of Y: U (n1, k, ...), S (k, k, ...), V (n2, k, ...); k = 0 keeps
        min(n1, n2) singular tubes."""
        st = self._L.tsvd_factor(self._h, _ptr(Y), len(dims), _dims(dims), int(k), _ptr(U),
                                 _ptr(S), _ptr(V))
        self._check("tsvd_factor", st)
        return st

    def compress(self, Y, dims: Sequence[int], method: int, k: int, Z):
        """t-SVD compression (Method 1: COMPRESS_GLOBAL, Method 2: COMPRESS_TUBAL) of Y into Z.
        Returns (entries kept, compression ratio)."""
        kept = ctypes.c_int64(0)
        ratio = ctypes.c_double(0.0)
        st = self._L.tsvd_compress(self._h, _ptr(Y), len(dims), _dims(dims), int(method), int(k),
                                   _ptr(Z), ctypes.byref(kept), ctypes.byref(ratio))
        self._check("tsvd_compress", st)
        return kept.value, ratio.value

    def raw_compress(self, Y, dims: Sequence[int], method: int, k: int, Z) -> int:
        return self._L.tsvd_compress(self._h, _ptr(Y), len(dims), _dims(dims), int(method),
                                     int(k), _ptr(Z), None, None)

    def raw_factor(self, Y, dims: Sequence[int], k: int, U, S, V) -> int:
        """tsvd_factor status without raising (argument checks in the tests)."""
        return self._L.tsvd_factor(self._h, _ptr(Y), len(dims), _dims(dims), int(k), _ptr(U),
                                   _ptr(S), _ptr(V))

    def tproduct(self, A, B, C, dims: Sequence[int], n4: int):
        """t-product C = A * B: A dims (n1, n2, ...), B (n2, n4, ...), C (n1, n4, ...)."""
        st = self._L.tsvd_tproduct(self._h, _ptr(A), _ptr(B), _ptr(C), len(dims), _dims(dims),
                                   int(n4))
        self._check("tsvd_tproduct", st)
        return st

    def raw_tproduct(self, A, B, C, dims: Sequence[int], n4: int) -> int:
        return self._L.tsvd_tproduct(self._h, _ptr(A), _ptr(B), _ptr(C), len(dims),
                                     _dims(dims), int(n4))

    def tnn_complete(self, M_obs, omega, dims: Sequence[int], iters: int, X_out, Z_out=None,
                     stats: bool = False):
        s = Stats()
        st = self._L.tnn_complete(self._h, _ptr(M_obs), _ptr(omega), len(dims), _dims(dims),
                                  int(iters), _ptr(X_out), _ptr(Z_out),
                                  ctypes.byref(s) if stats else None)
        self._check("tnn_complete", st)
        return s.as_dict() if stats else None

    def trpca(self, M, dims: Sequence[int], lam: float, iters: int, L_out, S_out,
              stats: bool = False):
        s = Stats()
        st = self._L.trpca(self._h, _ptr(M), len(dims), _dims(dims), float(lam), int(iters),
                           _ptr(L_out), _ptr(S_out), ctypes.byref(s) if stats else None)
        self._check("trpca", st)
        return s.as_dict() if stats else None

    def tnn_complete_resume(self, M_obs, omega, dims: Sequence[int], iters: int, X_out,
                            Z_out=None, Q_out=None, Z0=None, Q0=None, rho=0.0,
                            stats: bool = False):
        """tnn_complete continued from (Z0, Q0, rho) (device buffers or None); Q_out receives
        the final scaled dual."""
        st0 = AdmmState(_ptr(Z0), _ptr(Q0), None, None, float(rho))
        s = Stats()
        st = self._L.tnn_complete_resume(self._h, _ptr(M_obs), _ptr(omega), len(dims),
                                         _dims(dims), int(iters), ctypes.byref(st0),
                                         _ptr(X_out), _ptr(Z_out), _ptr(Q_out),
                                         ctypes.byref(s) if stats else None)
        self._check("tnn_complete_resume", st)
        return s.as_dict() if stats else None

    def trpca_resume(self, M, dims: Sequence[int], lam: float, iters: int, L_out, S_out,
                     W_out=None, S0=None, W0=None, rho=0.0, stats: bool = False):
        """trpca continued from (S0, W0, rho); W_out receives the final scaled dual."""
        st0 = AdmmState(None, None, _ptr(S0), _ptr(W0), float(rho))
        s = Stats()
        st = self._L.trpca_resume(self._h, _ptr(M), len(dims), _dims(dims), float(lam),
                                  int(iters), ctypes.byref(st0), _ptr(L_out), _ptr(S_out),
                                  _ptr(W_out), ctypes.byref(s) if stats else None)
        self._check("trpca_resume", st)
        return s.as_dict() if stats else None

    def solve_batched(self, problems, iters: int, stats: bool = False,
                      entry: str = "tsvd_solve_batched"):
        """problems: sequence of dicts with keys kind ('complete' | 'rpca'), dims, M,
        omega (completion), lam (RPCA), out0, out1 (device buffers).  `entry` picks the C
        entry point: tsvd_solve_batched (any mix), tnn_complete_batched or trpca_batched."""
        st = self.raw_solve_batched(problems, iters, stats, entry)
        self._check(entry, st[0])
        return st[1]

    def tnn_complete_batched(self, problems, iters: int, stats: bool = False):
        return self.solve_batched(problems, iters, stats, "tnn_complete_batched")

    def trpca_batched(self, problems, iters: int, stats: bool = False):
        return self.solve_batched(problems, iters, stats, "trpca_batched")

    def raw_solve_batched(self, problems, iters: int, stats: bool = False,
                          entry: str = "tsvd_solve_batched"):
        """(status, stats dict or None) without raising."""
        if entry not in ("tsvd_solve_batched", "tnn_complete_batched", "trpca_batched"):
            raise ValueError(f"unknown batched entry point {entry}")
        arr = (Problem * len(problems))()
        for i, q in enumerate(problems):
            if len(q["dims"]) not in (3, 4):
                raise ValueError(f"problem {i}: batched tensors are 3-way or 4-way")
            d = list(q["dims"]) + [1] * (4 - len(q["dims"]))
            arr[i].kind = PROBLEM_COMPLETE if q["kind"] == "complete" else PROBLEM_RPCA
            arr[i].order = len(q["dims"])
            arr[i].dims = (ctypes.c_int64 * 4)(*[int(x) for x in d])
            arr[i].M = _ptr(q["M"])
            arr[i].omega = _ptr(q.get("omega"))
            arr[i].lam = float(q.get("lam", 0.0))
            arr[i].out0 = _ptr(q["out0"])
            arr[i].out1 = _ptr(q.get("out1"))
        s = Stats()
        st = getattr(self._L, entry)(self._h, len(problems), arr, int(iters),
                                     ctypes.byref(s) if stats else None)
        return st, (s.as_dict() if stats and st == TSVD_OK else None)

    def cgemm(self, transa, transb, m, n, k, A, lda, stride_a, B, ldb, stride_b, C, ldc,
              stride_c, batch):
        """C_b = op(A_b) op(B_b) on complex64 column-major device buffers (see tsvd_cgemm)."""
        st = self._L.tsvd_cgemm(self._h, int(transa), int(transb), int(m), int(n), int(k),
                                _ptr(A), int(lda), int(stride_a), _ptr(B), int(ldb),
                                int(stride_b), _ptr(C), int(ldc), int(stride_c), int(batch))
        self._check("tsvd_cgemm", st)

    # raw status variants (for error-path tests)
    def raw_tnn_complete(self, M_obs, omega, order, dims, iters, X_out, Z_out=None) -> int:
        return self._L.tnn_complete(self._h, _ptr(M_obs), _ptr(omega), int(order),
                                    _dims(dims) if dims is not None else None, int(iters),
                                    _ptr(X_out), _ptr(Z_out), None)
