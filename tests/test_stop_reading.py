"""The reading behind the SVT stopping test of the slice Jacobi (the Lemma of Sec. 4.1 computed
by an FP32 one-sided Jacobi that stops at a tolerance), checked on the CPU with a plain FP64
one-sided Jacobi written here: a pair also stops once |x^H y| <= tol min(||x||, ||y||)
||B||_F / nv.  On nearly low-rank complex slices (the late iterations of an ADMM solve) that
test never rotates more than the relative one, and the U-form rebuild
D = sum_{sigma > tau} (1 - tau / sigma) u u^H B then differs from the exact D_tau(B) by no
more than a small multiple of tol ||B||_F -- the scale the relative test already leaves --
whether the noise directions are thresholded away or kept."""
import numpy as np
import pytest

TOL = 1e-6


def _jacobi(B, svt_stop, max_sweeps=60):
    """Cyclic one-sided Jacobi on the columns of B; returns (W = B V, rotations applied)."""
    W = B.copy()
    nv = W.shape[1]
    floor2 = TOL * TOL * np.linalg.norm(B) ** 2 / (nv * nv)
    rots = 0
    for _ in range(max_sweeps):
        rotated = False
        for p in range(nv - 1):
            for q in range(p + 1, nv):
                x, y = W[:, p], W[:, q]
                al, be = np.vdot(x, x).real, np.vdot(y, y).real
                g = np.vdot(x, y)
                c2 = abs(g) ** 2
                if c2 <= TOL * TOL * al * be:
                    continue
                if svt_stop and c2 <= floor2 * min(al, be):
                    continue
                zeta = (be - al) / (2 * abs(g))
                t = (1.0 if zeta >= 0 else -1.0) / (abs(zeta) + np.sqrt(1 + zeta * zeta))
                cs = 1 / np.sqrt(1 + t * t)
                sn = t * cs
                ph = g / abs(g)
                W[:, p], W[:, q] = cs * x - sn * np.conj(ph) * y, sn * ph * x + cs * y
                rotated = True
                rots += 1
        if not rotated:
            break
    return W, rots


def _svt_u_form(W, B, tau):
    sig = np.linalg.norm(W, axis=0)
    keep = sig > tau
    U = W[:, keep] / sig[keep]
    return (U * ((sig[keep] - tau) / sig[keep])) @ (U.conj().T @ B)


def _svt_exact(B, tau):
    U, s, Vh = np.linalg.svd(B, full_matrices=False)
    return (U * np.maximum(s - tau, 0)) @ Vh


@pytest.mark.parametrize("noise", [1e-5, 1e-3])
@pytest.mark.parametrize("tau_frac", [1e-2, 1e-9])
def test_svt_stopping_test_error_and_work(noise, tau_frac):
    rng = np.random.default_rng(7)
    m, n, r = 48, 36, 4
    A = (rng.standard_normal((m, r)) + 1j * rng.standard_normal((m, r))) @ \
        (rng.standard_normal((r, n)) + 1j * rng.standard_normal((r, n)))
    E = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
    B = A + noise * np.linalg.norm(A) / np.sqrt(A.size) * E
    s = np.linalg.svd(B, compute_uv=False)
    tau = tau_frac * s[0]   # 1e-2: the noise thresholded away; 1e-9: every direction kept
    exact = _svt_exact(B, tau)
    nb = np.linalg.norm(B)
    W_rel, rot_rel = _jacobi(B, svt_stop=False)
    W_svt, rot_svt = _jacobi(B, svt_stop=True)
    err_rel = np.linalg.norm(_svt_u_form(W_rel, B, tau) - exact) / nb
    err_svt = np.linalg.norm(_svt_u_form(W_svt, B, tau) - exact) / nb
    assert rot_svt <= rot_rel
    assert err_rel <= 10 * TOL and err_svt <= 10 * TOL, (err_rel, err_svt)
    if noise == 1e-5:
        # the noise tail is far below the RMS column norm: the SVT test skips its pairs
        assert rot_svt < rot_rel
