"""Small helpers shared by the tests (layout conversion and error measures)."""
import numpy as np


def colmajor(x, dtype=np.float32):
    return np.asfortranarray(np.asarray(x, dtype=dtype)).ravel(order="F").copy()


def uncolmajor(v, shape):
    return np.reshape(np.asarray(v), tuple(shape), order="F")


def relerr(a, b, floor=0.0):
    """||a - b||_F / max(||b||_F, floor)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = max(np.linalg.norm(b.ravel()), floor)
    if den == 0:
        return float(np.linalg.norm(a.ravel()))
    return float(np.linalg.norm((a - b).ravel()) / den)


def rse_db(x_rec, x_true):
    """Relative square error in dB, 20 log10(||X_rec - X|| / ||X||) (Sec. 3)."""
    return 20.0 * np.log10(np.linalg.norm((x_rec - x_true).ravel())
                           / np.linalg.norm(np.asarray(x_true).ravel()))


def bcirc(A):
    """Block-circulant matrix of an n1 x n2 x n3 tensor: block (i, j) is A(:, :, (i-j) mod n3)."""
    n1, n2, n3 = A.shape
    B = np.zeros((n1 * n3, n2 * n3), dtype=A.dtype)
    for i in range(n3):
        for j in range(n3):
            B[i * n1:(i + 1) * n1, j * n2:(j + 1) * n2] = A[:, :, (i - j) % n3]
    return B


def svt_matrix(Y, tau):
    """Textbook singular value thresholding of a matrix via numpy's SVD."""
    U, s, Vh = np.linalg.svd(Y, full_matrices=False)
    return (U * np.maximum(s - tau, 0.0)) @ Vh


def lowrank_fourier(shape, rank, seed):
    """A real tensor of tubal rank <= rank of any order >= 3: A * B with A (n1 x r x ...),
    B (r x n2 x ...) seeded N(0, 1), the t-product taken slice by slice after numpy's FFT over
    every mode from 3 on (Def. 2.1.1 extended to order p by the DFT along each such mode)."""
    from paper_1407_1785_gb300 import synth
    n1, n2, rest = shape[0], shape[1], tuple(shape[2:])
    nr = int(np.prod(rest))
    A = synth.normal(seed, 1, n1 * rank * nr).reshape((n1, rank) + rest, order="F")
    B = synth.normal(seed, 2, rank * n2 * nr).reshape((rank, n2) + rest, order="F")
    axes = tuple(range(2, len(shape)))
    Ch = np.einsum("ik...,kj...->ij...", np.fft.fftn(A, axes=axes), np.fft.fftn(B, axes=axes))
    return np.real(np.fft.ifftn(Ch, axes=axes))
