"""FP64 CPU oracle for the t-SVT ADMM path (test infrastructure).

This package is the plain, slow reference that the CUDA library is checked against.  It is
loaded only by the test suite, by ``__graft_entry__.smoke()`` and by the CPU-baseline leg of
``bench.py``; the library (``paper_1407_1785_gb300``) never imports it, and the two share no
code.  The arithmetic lives in ``tsvd_oracle.c`` (plain C99, FP64, OpenMP over independent
slices); this module only marshals numpy arrays through ctypes.

Array convention: a tensor of shape (n1, n2, n3[, n4]) is passed in MATLAB column-major
order, i.e. ``np.asfortranarray(x)`` flattened with ``order="F"``.  The helpers below take
and return ordinary numpy arrays of shape (n1, n2, ...) and do that conversion.

Functions (each cites the passage of arXiv:1407.1785 it follows):
  dft / idft          DFT along modes 3..N, naive sum (Sec. 2.1, Algorithm 1)
  svd                 full complex SVD by one-sided Jacobi (Algorithm 1's per-slice SVD)
  tsvt                t-SVT, the TNN proximal map (eq. shrink, eq. shrink2, Lemma of Sec. 4.1)
  tnn_complete        TNN completion ADMM (eq. proj, eq. shrink, dual ascent; Sec. 4)
  trpca               tensor robust PCA ADMM (eq. low_rank, eq. sparse, eq. sparse2, eq. dual)
  shrink              entrywise / tube-wise shrink (eq. sparse2)
  tproduct            t-product by the FFT route (Def. 2.1.1, Sec. 2.1)
  ttranspose          tensor transpose (Def. 2.1.2)
  tsvd                full t-SVD (Theorem 2.2.1, Algorithm 1)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tsvd_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")

OK, EINVAL, ENOMEM, ENOTCONV, EIMAG = 0, 1, 2, 4, 7
SCALE_AVG, SCALE_SUM = 0, 1
SPARSE_ENTRY, SPARSE_TUBE = 0, 1
COMPRESS_GLOBAL, COMPRESS_TUBAL = 1, 2


def build(force: bool = False) -> str:
    """Compile tsvd_oracle.c into oracle/_build/liboracle.so with gcc (plain C99 + OpenMP)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu99", "-O2", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i64p = ctypes.POINTER(ctypes.c_int64)
        c_int, c_i64, c_dbl = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        L.orc_num_threads.restype = c_int
        L.orc_set_num_threads.argtypes = [c_int]
        L.orc_dft.argtypes = [c_int, i64p, P, c_int]
        L.orc_svd.argtypes = [c_i64, c_i64, P, P, P, P]
        L.orc_tsvt.argtypes = [c_int, i64p, P, c_dbl, P, P, P]
        L.orc_tnn_complete.argtypes = [c_int, i64p, P, P, c_int, c_dbl, c_dbl, c_dbl, c_int,
                                       P, P, P, P]
        L.orc_trpca.argtypes = [c_int, i64p, P, c_dbl, c_int, c_dbl, c_dbl, c_dbl, c_int,
                                c_int, P, P, P, P]
        L.orc_shrink.argtypes = [c_int, i64p, P, c_dbl, c_int, P]
        L.orc_tproduct.argtypes = [c_i64, c_i64, c_i64, c_i64, P, P, P]
        L.orc_ttranspose.argtypes = [c_i64, c_i64, c_i64, P, P]
        L.orc_tsvd.argtypes = [c_i64, c_i64, c_i64, P, P, P, P]
        L.orc_tproduct_nd.argtypes = [c_int, i64p, c_i64, P, P, P]
        L.orc_ttranspose_nd.argtypes = [c_int, i64p, P, P]
        L.orc_tsvd_nd.argtypes = [c_int, i64p, P, P, P, P]
        L.orc_compress.argtypes = [c_int, i64p, P, c_int, c_i64, P, i64p]
        for name in ("orc_dft", "orc_svd", "orc_tsvt", "orc_tnn_complete", "orc_trpca",
                     "orc_shrink", "orc_tproduct", "orc_ttranspose", "orc_tsvd",
                     "orc_tproduct_nd", "orc_ttranspose_nd", "orc_tsvd_nd", "orc_compress"):
            getattr(L, name).restype = c_int
        _lib = L
    return _lib


class OracleError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"oracle {fn} returned status {code}")
        self.code = code


def _check(fn: str, code: int, allow=(OK,)):
    if code not in allow:
        raise OracleError(fn, code)
    return code


def _dims(shape) -> ctypes.Array:
    return (ctypes.c_int64 * len(shape))(*[int(s) for s in shape])


def _f64(x) -> np.ndarray:
    """Column-major float64 copy, flattened in MATLAB order."""
    return np.asfortranarray(np.asarray(x, dtype=np.float64)).ravel(order="F").copy()


def _c128(x) -> np.ndarray:
    return np.asfortranarray(np.asarray(x, dtype=np.complex128)).ravel(order="F").copy()


def _unflat(v: np.ndarray, shape) -> np.ndarray:
    return np.reshape(v, shape, order="F")


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    lib().orc_set_num_threads(int(n))


def dft(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """DFT (or inverse DFT, 1/n normalised) along modes 3..N of an (n1, n2, ...) array."""
    x = np.asarray(x)
    v = _c128(x)
    _check("dft", lib().orc_dft(x.ndim, _dims(x.shape), _ptr(v), int(bool(inverse))))
    return _unflat(v, x.shape)


def idft(x: np.ndarray) -> np.ndarray:
    return dft(x, inverse=True)


def svd(A: np.ndarray):
    """Full SVD A = U diag(s) V^H by one-sided Jacobi; returns (U, s, V)."""
    A = np.asarray(A, dtype=np.complex128)
    m, n = A.shape
    a = _c128(A)
    U = np.zeros(m * m, np.complex128)
    V = np.zeros(n * n, np.complex128)
    s = np.zeros(min(m, n), np.float64)
    _check("svd", lib().orc_svd(m, n, _ptr(a), _ptr(U), _ptr(s), _ptr(V)))
    return _unflat(U, (m, m)), s, _unflat(V, (n, n))


def tsvt(Y: np.ndarray, tau: float, with_info: bool = False):
    """t-SVT of a real (n1, n2, n3[, n4]) tensor.  With with_info also returns the
    per-Fourier-slice ranks (shape dims[2:], column-major) and the TNN (sum form)."""
    Y = np.asarray(Y, dtype=np.float64)
    y = _f64(Y)
    z = np.zeros_like(y)
    ns = int(np.prod(Y.shape[2:]))
    rk = np.zeros(ns, np.int32)
    tnn = ctypes.c_double(0.0)
    _check("tsvt", lib().orc_tsvt(Y.ndim, _dims(Y.shape), _ptr(y), float(tau), _ptr(z),
                                  _ptr(rk), ctypes.byref(tnn)))
    Z = _unflat(z, Y.shape)
    if with_info:
        return Z, _unflat(rk, Y.shape[2:]), tnn.value
    return Z


def tnn_complete(M: np.ndarray, omega: np.ndarray, iters: int, rho0: float = 1e-2,
                 mu: float = 1.1, rho_max: float = 1e10, tnn_scale: int = SCALE_AVG,
                 with_dual: bool = False):
    """TNN completion ADMM; returns (X, Z) after `iters` iterations, plus (Q, rho) with
    with_dual."""
    M = np.asarray(M, dtype=np.float64)
    m = _f64(M)
    om = np.asfortranarray(np.asarray(omega, dtype=np.uint8)).ravel(order="F").copy()
    assert om.size == m.size
    X = np.zeros_like(m)
    Z = np.zeros_like(m)
    Q = np.zeros_like(m)
    rho = ctypes.c_double(0.0)
    _check("tnn_complete", lib().orc_tnn_complete(M.ndim, _dims(M.shape), _ptr(m), _ptr(om),
                                                  int(iters), rho0, mu, rho_max, tnn_scale,
                                                  _ptr(X), _ptr(Z), _ptr(Q), ctypes.byref(rho)))
    out = (_unflat(X, M.shape), _unflat(Z, M.shape))
    if with_dual:
        return out + (_unflat(Q, M.shape), rho.value)
    return out


def trpca(M: np.ndarray, lam: float, iters: int, rho0: float = 1e-2, mu: float = 1.1,
          rho_max: float = 1e10, tnn_scale: int = SCALE_AVG, sparse_mode: int = SPARSE_ENTRY,
          with_dual: bool = False):
    """Tensor robust PCA ADMM; returns (L, S) after `iters` iterations, plus (W, rho) with
    with_dual."""
    M = np.asarray(M, dtype=np.float64)
    m = _f64(M)
    L = np.zeros_like(m)
    S = np.zeros_like(m)
    W = np.zeros_like(m)
    rho = ctypes.c_double(0.0)
    _check("trpca", lib().orc_trpca(M.ndim, _dims(M.shape), _ptr(m), float(lam), int(iters),
                                    rho0, mu, rho_max, tnn_scale, sparse_mode, _ptr(L),
                                    _ptr(S), _ptr(W), ctypes.byref(rho)))
    out = (_unflat(L, M.shape), _unflat(S, M.shape))
    if with_dual:
        return out + (_unflat(W, M.shape), rho.value)
    return out


def shrink(D: np.ndarray, kappa: float, mode: int = SPARSE_ENTRY) -> np.ndarray:
    D = np.asarray(D, dtype=np.float64)
    d = _f64(D)
    s = np.zeros_like(d)
    _check("shrink", lib().orc_shrink(D.ndim, _dims(D.shape), _ptr(d), float(kappa), mode,
                                      _ptr(s)))
    return _unflat(s, D.shape)


def tproduct(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """t-product A * B (Def. 2.1.1; for order > 3 through the DFT along every mode from 3 on):
    A (n1, n2, ...), B (n2, n4, ...) -> (n1, n4, ...)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    assert A.ndim >= 3 and B.ndim == A.ndim
    assert A.shape[1] == B.shape[0] and A.shape[2:] == B.shape[2:]
    n1, n2, n4, rest = A.shape[0], A.shape[1], B.shape[1], A.shape[2:]
    a, b = _f64(A), _f64(B)
    c = np.zeros(n1 * n4 * int(np.prod(rest)), np.float64)
    if A.ndim == 3:
        _check("tproduct", lib().orc_tproduct(n1, n2, n4, rest[0], _ptr(a), _ptr(b), _ptr(c)))
    else:
        _check("tproduct", lib().orc_tproduct_nd(A.ndim, _dims(A.shape), n4, _ptr(a), _ptr(b),
                                                 _ptr(c)))
    return _unflat(c, (n1, n4) + rest)


def ttranspose(A: np.ndarray) -> np.ndarray:
    """Tensor transpose (Def. 2.1.2): (n1, n2, ...) -> (n2, n1, ...)."""
    A = np.asarray(A, dtype=np.float64)
    assert A.ndim >= 3
    n1, n2, rest = A.shape[0], A.shape[1], A.shape[2:]
    a = _f64(A)
    t = np.zeros_like(a)
    if A.ndim == 3:
        _check("ttranspose", lib().orc_ttranspose(n1, n2, rest[0], _ptr(a), _ptr(t)))
    else:
        _check("ttranspose", lib().orc_ttranspose_nd(A.ndim, _dims(A.shape), _ptr(a), _ptr(t)))
    return _unflat(t, (n2, n1) + rest)


def tsvd(M: np.ndarray):
    """Full t-SVD M = U * S * V^T (order 3 to 6); returns real (U, S, V)."""
    M = np.asarray(M, dtype=np.float64)
    assert M.ndim >= 3
    n1, n2, rest = M.shape[0], M.shape[1], M.shape[2:]
    ns = int(np.prod(rest))
    m = _f64(M)
    U = np.zeros(n1 * n1 * ns)
    S = np.zeros(n1 * n2 * ns)
    V = np.zeros(n2 * n2 * ns)
    if M.ndim == 3:
        _check("tsvd", lib().orc_tsvd(n1, n2, rest[0], _ptr(m), _ptr(U), _ptr(S), _ptr(V)))
    else:
        _check("tsvd", lib().orc_tsvd_nd(M.ndim, _dims(M.shape), _ptr(m), _ptr(U), _ptr(S),
                                         _ptr(V)))
    return (_unflat(U, (n1, n1) + rest), _unflat(S, (n1, n2) + rest), _unflat(V, (n2, n2) + rest))


def compress(M: np.ndarray, method: int, k: int):
    """t-SVD compression of Sec. 3 (Method 1: COMPRESS_GLOBAL, the k largest Fourier singular
    values over all slices, ties at the cut kept; Method 2: COMPRESS_TUBAL, the first k
    singular tubes).  Returns (Z, entries kept)."""
    M = np.asarray(M, dtype=np.float64)
    m = _f64(M)
    z = np.zeros_like(m)
    kept = ctypes.c_int64(0)
    _check("compress", lib().orc_compress(M.ndim, _dims(M.shape), _ptr(m), int(method), int(k),
                                          _ptr(z), ctypes.byref(kept)))
    return _unflat(z, M.shape), kept.value
