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
