/*
 * tsvd_oracle.c -- FP64 CPU oracle for the t-SVD completion / tensor robust PCA path of
 * Zhang, Ely, Aeron, Hao and Kilmer, "Novel methods for multilinear data completion and
 * de-noising based on tensor-SVD" (arXiv:1407.1785).
 *
 * TEST INFRASTRUCTURE.  This is the plain, slow, obviously-correct reference that the CUDA
 * library is checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it; the library itself never does.  It shares no code, header,
 * table or helper with the CUDA sources.
 *
 * Every routine writes out the paper's definition or algorithm in its own order:
 *   - DFT along a mode: a naive O(n^2) sum per fiber (the FFT route of Sec. 2.1 and the
 *     fft(.,[],i) loop of Algorithm 1);
 *   - matrix SVD: cyclic one-sided (Hestenes) Jacobi in complex FP64, no LAPACK;
 *   - singular value thresholding D_tau: the Lemma of Sec. 4.1 (eq. "operator");
 *   - t-SVT: Algorithm 1's per-slice SVDs + the Lemma on every Fourier slice (eq. shrink2);
 *   - TNN completion ADMM: eq. proj, eq. shrink and the dual ascent of Sec. 4;
 *   - tensor RPCA ADMM: eq. low_rank, eq. sparse (closed form eq. sparse2) and eq. dual of
 *     Sec. 5;
 *   - t-product (Def. 2.1.1 via the FFT route of Sec. 2.1), tensor transpose (Def. 2.1.2),
 *     full t-SVD (Theorem 2.2.1 / Algorithm 1), for order 3 and, through Algorithm 1's loop
 *     over modes 3..N, for orders up to 6;
 *   - t-SVD compression, Methods 1 and 2 of Sec. 3.
 *
 * Layout: every tensor is MATLAB column-major; entry (i1,i2,i3[,i4]) lives at
 * i1 + n1*(i2 + n2*(i3 + n3*i4)).  Complex values are C99 double complex.
 *
 * Readings of points the paper leaves open (each one is listed in the design notes):
 *   - Algorithm 1 SVDs every slice independently, which would make the inverse-transformed
 *     factors complex.  Here slice k and its conjugate partner (-k mod n along each
 *     transformed mode) share one SVD (the partner gets the complex conjugate), and a
 *     self-conjugate slice (its own partner) is made exactly real before its SVD, so U, S, V
 *     and every thresholded result are real after the inverse DFT.
 *   - The threshold of eq. shrink is applied to the singular values of the unnormalised DFT
 *     slices, tau = 1/rho ("avg" scaling, the default) or tau = P/rho with P the number of
 *     Fourier slices ("sum" scaling, the prox of the TNN exactly as defined in Thm 2.4.1).
 *   - rho grows as rho <- min(mu*rho, rho_max) after each iteration and the scaled dual is
 *     rescaled by rho_k/rho_{k+1} so that it keeps meaning (multiplier / rho).
 *   - In D_tau the "(1 - tau/sigma)_+" form of Sec. 4.1 is taken as max(sigma - tau, 0) and
 *     the tube shrink factor of eq. sparse2 is 0 when the tube norm is 0.
 *   - For a 4-way tensor the tube group of the l_{1,1,2} norm is every entry with the same
 *     (i,j), i.e. S(i,j,:,:).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_ENOTCONV = 4, ORC_EIMAG = 7 };
enum { ORC_SCALE_AVG = 0, ORC_SCALE_SUM = 1 };
enum { ORC_SPARSE_ENTRY = 0, ORC_SPARSE_TUBE = 1 };

#define ORC_MAX_ORDER 6
#define ORC_JACOBI_MAX_SWEEPS 80

/* Number of threads the oracle runs with (OpenMP over independent slices / fibers). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

static int64_t prod_dims(const int64_t* dims, int from, int to)
{
    int64_t p = 1;
    for (int d = from; d < to; ++d) p *= dims[d];
    return p;
}

static int check_dims(int order, const int64_t* dims)
{
    if (order < 2 || order > ORC_MAX_ORDER || !dims) return 0;
    for (int d = 0; d < order; ++d)
        if (dims[d] < 1) return 0;
    return 1;
}

/* ------------------------------------------------------------------------------------------
 * DFT along one mode (Sec. 2.1 computes the t-product and the t-SVD with FFTs along the tubes;
 * Algorithm 1 transforms along each mode i = 3..N in turn).  A naive sum per fiber:
 *     forward  y[k] = sum_t x[t] exp(-2 pi i t k / n)
 *     inverse  y[t] = (1/n) sum_k x[k] exp(+2 pi i t k / n)
 * The phase index t*k is reduced modulo n before the angle is formed.
 * ---------------------------------------------------------------------------------------- */
static void dft_mode(cplx* x, int order, const int64_t* dims, int mode, int inverse)
{
    const int64_t n = dims[mode];
    const int64_t inner = prod_dims(dims, 0, mode);          /* stride of this mode */
    const int64_t outer = prod_dims(dims, mode + 1, order);
    const double sgn = inverse ? 1.0 : -1.0;
    cplx* w = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    for (int64_t m = 0; m < n; ++m) {
        double a = 2.0 * M_PI * (double)m / (double)n;
        w[m] = cos(a) + sgn * sin(a) * I;
    }
    #pragma omp parallel
    {
        cplx* in = (cplx*)malloc(sizeof(cplx) * (size_t)n);
        #pragma omp for schedule(static)
        for (int64_t f = 0; f < inner * outer; ++f) {
            const int64_t a = f % inner, b = f / inner;
            cplx* base = x + a + b * inner * n;
            for (int64_t t = 0; t < n; ++t) in[t] = base[t * inner];
            for (int64_t k = 0; k < n; ++k) {
                cplx s = 0;
                for (int64_t t = 0; t < n; ++t) s += in[t] * w[(t * k) % n];
                base[k * inner] = inverse ? s / (double)n : s;
            }
        }
        free(in);
    }
    free(w);
}

/* DFT along modes 3..N (0-based 2..order-1), the loop of Algorithm 1. */
static void dft_tubes(cplx* x, int order, const int64_t* dims, int inverse)
{
    for (int mode = 2; mode < order; ++mode) dft_mode(x, order, dims, mode, inverse);
}

/* Exported for tests: complex in-place DFT along modes 3..N of a column-major tensor. */
int orc_dft(int order, const int64_t* dims, double* xz /* interleaved complex */, int inverse)
{
    if (!check_dims(order, dims) || !xz) return ORC_EINVAL;
    dft_tubes((cplx*)xz, order, dims, inverse);
    return ORC_OK;
}

/* Linear index of the Fourier slice that is the complex conjugate partner of slice s.
 * Slice s = (k3,...,kN) in column-major order over dims[2..]; partner = (-k3 mod n3, ...). */
static int64_t conj_partner(int order, const int64_t* dims, int64_t s)
{
    int64_t p = 0, stride = 1, rem = s;
    for (int d = 2; d < order; ++d) {
        const int64_t n = dims[d];
        const int64_t k = rem % n;
        rem /= n;
        p += ((n - k) % n) * stride;
        stride *= n;
    }
    return p;
}

/* ------------------------------------------------------------------------------------------
 * Matrix SVD by cyclic one-sided (Hestenes) Jacobi, complex FP64.
 * G is m-by-n column-major with m >= n; on return its columns are U*Sigma (unnormalised),
 * V (n-by-n) accumulates the rotations, so that A = G V^H at every step.
 * A pair (p,q) is rotated when |g_p^H g_q| > tol * ||g_p|| ||g_q||; the plane rotation
 * diagonalises the 2x2 Gram matrix [[a, c], [c*, b]] of the pair:
 *     c = |c| e^{i phi}, zeta = (b - a) / (2|c|), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
 *     cs = 1/sqrt(1+t^2), sn = cs*t,
 *     g_p <- cs g_p - sn e^{-i phi} g_q,   g_q <- sn e^{i phi} g_p + cs g_q.
 * Returns the number of sweeps used, or -1 if it hit the sweep cap.
 * ---------------------------------------------------------------------------------------- */
static int jacobi_onesided(int64_t m, int64_t n, cplx* G, cplx* V)
{
    const double tol = sqrt((double)m) * DBL_EPSILON;
    for (int64_t i = 0; i < n * n; ++i) V[i] = 0;
    for (int64_t i = 0; i < n; ++i) V[i + i * n] = 1;
    for (int sweep = 1; sweep <= ORC_JACOBI_MAX_SWEEPS; ++sweep) {
        int rotated = 0;
        for (int64_t p = 0; p < n - 1; ++p) {
            for (int64_t q = p + 1; q < n; ++q) {
                cplx* gp = G + p * m;
                cplx* gq = G + q * m;
                double a = 0, b = 0;
                cplx c = 0;
                for (int64_t r = 0; r < m; ++r) {
                    a += creal(gp[r]) * creal(gp[r]) + cimag(gp[r]) * cimag(gp[r]);
                    b += creal(gq[r]) * creal(gq[r]) + cimag(gq[r]) * cimag(gq[r]);
                    c += conj(gp[r]) * gq[r];
                }
                const double ac = cabs(c);
                if (ac == 0.0 || !(ac > tol * sqrt(a) * sqrt(b))) continue;
                rotated = 1;
                const cplx e = c / ac; /* e^{i phi} */
                const double zeta = (b - a) / (2.0 * ac);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double cs = 1.0 / sqrt(1.0 + t * t);
                const double sn = cs * t;
                for (int64_t r = 0; r < m; ++r) {
                    const cplx x = gp[r], y = gq[r];
                    gp[r] = cs * x - sn * conj(e) * y;
                    gq[r] = sn * e * x + cs * y;
                }
                cplx* vp = V + p * n;
                cplx* vq = V + q * n;
                for (int64_t r = 0; r < n; ++r) {
                    const cplx x = vp[r], y = vq[r];
                    vp[r] = cs * x - sn * conj(e) * y;
                    vq[r] = sn * e * x + cs * y;
                }
            }
        }
        if (!rotated) return sweep;
    }
    return -1;
}

/* Extend the orthonormal columns U(:, 0..k-1) (m-by-m array, column-major) to a full unitary
 * basis by Gram-Schmidt (applied twice) on the standard basis vectors. */
static void complete_basis(int64_t m, int64_t k, cplx* U)
{
    cplx* v = (cplx*)malloc(sizeof(cplx) * (size_t)m);
    int64_t have = k;
    for (int64_t e = 0; e < m && have < m; ++e) {
        for (int64_t r = 0; r < m; ++r) v[r] = (r == e) ? 1.0 : 0.0;
        for (int pass = 0; pass < 2; ++pass) {
            for (int64_t j = 0; j < have; ++j) {
                cplx d = 0;
                for (int64_t r = 0; r < m; ++r) d += conj(U[r + j * m]) * v[r];
                for (int64_t r = 0; r < m; ++r) v[r] -= d * U[r + j * m];
            }
        }
        double nv = 0;
        for (int64_t r = 0; r < m; ++r) nv += creal(v[r] * conj(v[r]));
        nv = sqrt(nv);
        if (nv < 0.5) continue;
        for (int64_t r = 0; r < m; ++r) U[r + have * m] = v[r] / nv;
        ++have;
    }
    free(v);
}

/* Full SVD A = U diag(sigma) V^H of an m-by-n complex matrix (column-major).
 * U is m-by-m, V is n-by-n (both unitary), sigma has min(m,n) entries, descending.
 * Singular vectors whose singular value is zero are completed to an orthonormal basis.
 * Returns sweeps used (>0) or -1 on non-convergence. */
static int svd_full(int64_t m, int64_t n, const cplx* A, cplx* U, double* sigma, cplx* V)
{
    const int tr = m < n;                 /* work on A^H when A is wide */
    const int64_t mm = tr ? n : m, nn = tr ? m : n;
    cplx* G = (cplx*)malloc(sizeof(cplx) * (size_t)(mm * nn));
    cplx* W = (cplx*)malloc(sizeof(cplx) * (size_t)(nn * nn));
    for (int64_t j = 0; j < nn; ++j)
        for (int64_t i = 0; i < mm; ++i)
            G[i + j * mm] = tr ? conj(A[j + i * m]) : A[i + j * m];
    const int sweeps = jacobi_onesided(mm, nn, G, W);
    /* sigma_j = ||g_j||; order descending (selection by index, stable on ties) */
    double* s = (double*)malloc(sizeof(double) * (size_t)nn);
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)nn);
    for (int64_t j = 0; j < nn; ++j) {
        double acc = 0;
        for (int64_t i = 0; i < mm; ++i) acc += creal(G[i + j * mm] * conj(G[i + j * mm]));
        s[j] = sqrt(acc);
        idx[j] = j;
    }
    for (int64_t a = 0; a < nn; ++a)
        for (int64_t b = a + 1; b < nn; ++b)
            if (s[idx[b]] > s[idx[a]]) { int64_t t = idx[a]; idx[a] = idx[b]; idx[b] = t; }
    /* left vectors of the worked matrix (mm-by-mm) and right vectors (nn-by-nn) */
    cplx* UL = (cplx*)calloc((size_t)(mm * mm), sizeof(cplx));
    cplx* VR = (cplx*)malloc(sizeof(cplx) * (size_t)(nn * nn));
    int64_t nonzero = 0;
    for (int64_t a = 0; a < nn; ++a) {
        const int64_t j = idx[a];
        sigma[a] = s[j];
        for (int64_t i = 0; i < nn; ++i) VR[i + a * nn] = W[i + j * nn];
        if (s[j] > 0 && nonzero == a) {
            for (int64_t i = 0; i < mm; ++i) UL[i + a * mm] = G[i + j * mm] / s[j];
            ++nonzero;
        }
    }
    complete_basis(mm, nonzero, UL);
    if (!tr) {
        memcpy(U, UL, sizeof(cplx) * (size_t)(m * m));
        memcpy(V, VR, sizeof(cplx) * (size_t)(n * n));
    } else {
        /* A^H = UL S VR^H  =>  A = VR S UL^H */
        memcpy(U, VR, sizeof(cplx) * (size_t)(m * m));
        memcpy(V, UL, sizeof(cplx) * (size_t)(n * n));
    }
    free(G); free(W); free(s); free(idx); free(UL); free(VR);
    return sweeps;
}

/* Exported for tests: full complex SVD (A, U, V interleaved complex, column-major). */
int orc_svd(int64_t m, int64_t n, const double* A, double* U, double* sigma, double* V)
{
    if (m < 1 || n < 1 || !A || !U || !sigma || !V) return ORC_EINVAL;
    return svd_full(m, n, (const cplx*)A, (cplx*)U, sigma, (cplx*)V) < 0 ? ORC_ENOTCONV : ORC_OK;
}

/* Singular value thresholding of one m-by-n slice (Lemma of Sec. 4.1, eq. "operator"):
 *     D_tau(A) = U diag((sigma_i - tau)_+) V^H.
 * Writes the result into Z (m-by-n), the count of sigma_i > tau into *rank and
 * sum sigma_i into *nuc.  Returns the SVD status. */
static int svt_slice(int64_t m, int64_t n, const cplx* A, double tau, cplx* Z, int32_t* rank,
                     double* nuc)
{
    const int64_t k = m < n ? m : n;
    cplx* U = (cplx*)malloc(sizeof(cplx) * (size_t)(m * m));
    cplx* V = (cplx*)malloc(sizeof(cplx) * (size_t)(n * n));
    double* s = (double*)malloc(sizeof(double) * (size_t)k);
    const int sweeps = svd_full(m, n, A, U, s, V);
    int32_t r = 0;
    double sum = 0;
    for (int64_t i = 0; i < k; ++i) {
        sum += s[i];
        if (s[i] > tau) ++r;
    }
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) {
            cplx acc = 0;
            for (int64_t l = 0; l < k; ++l) {
                const double d = s[l] - tau;
                if (d > 0) acc += U[i + l * m] * d * conj(V[j + l * n]);
            }
            Z[i + j * m] = acc;
        }
    *rank = r;
    *nuc = sum;
    free(U); free(V); free(s);
    return sweeps < 0 ? ORC_ENOTCONV : ORC_OK;
}

/* ------------------------------------------------------------------------------------------
 * t-SVT: the proximal map of the tensor nuclear norm (eq. shrink / eq. shrink2 with the Lemma
 * on each Fourier slice), for a real tensor of order 3 or more:
 *   1. Yhat = DFT of Y along modes 3..N (Algorithm 1);
 *   2. for every Fourier slice that is not the conjugate partner of an earlier one:
 *      D_tau of the slice (made exactly real first when it is self-conjugate);
 *   3. the partner slice takes the complex conjugate;
 *   4. inverse DFT; the imaginary part must vanish (relative 1e-12) and is dropped.
 * multirank (nullable) receives the rank of every thresholded Fourier slice (Def. 2.4.1 of
 * the result); tnn (nullable) receives sum over ALL Fourier slices of the singular values of
 * Yhat (the TNN of Thm 2.4.1, unnormalised DFT).
 * ---------------------------------------------------------------------------------------- */
int orc_tsvt(int order, const int64_t* dims, const double* Y, double tau, double* Z,
             int32_t* multirank, double* tnn)
{
    if (order < 3 || !check_dims(order, dims) || !Y || !Z || !(tau >= 0)) return ORC_EINVAL;
    const int64_t n1 = dims[0], n2 = dims[1];
    const int64_t ns = prod_dims(dims, 2, order);
    const int64_t sl = n1 * n2, N = sl * ns;
    cplx* X = (cplx*)malloc(sizeof(cplx) * (size_t)N);
    cplx* R = (cplx*)malloc(sizeof(cplx) * (size_t)N);
    double* nuc = (double*)calloc((size_t)ns, sizeof(double));
    int32_t* rk = (int32_t*)calloc((size_t)ns, sizeof(int32_t));
    if (!X || !R || !nuc || !rk) { free(X); free(R); free(nuc); free(rk); return ORC_ENOMEM; }
    for (int64_t i = 0; i < N; ++i) X[i] = Y[i];
    dft_tubes(X, order, dims, 0);
    int status = ORC_OK;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < ns; ++s) {
        const int64_t p = conj_partner(order, dims, s);
        if (p < s) continue;                              /* filled from its partner below */
        cplx* A = X + s * sl;
        if (p == s)
            for (int64_t i = 0; i < sl; ++i) A[i] = creal(A[i]);   /* self-conjugate: real */
        const int st = svt_slice(n1, n2, A, tau, R + s * sl, &rk[s], &nuc[s]);
        if (st != ORC_OK) {
            #pragma omp critical
            status = st;
        }
    }
    for (int64_t s = 0; s < ns; ++s) {
        const int64_t p = conj_partner(order, dims, s);
        if (p < s) {
            for (int64_t i = 0; i < sl; ++i) R[s * sl + i] = conj(R[p * sl + i]);
            rk[s] = rk[p];
            nuc[s] = nuc[p];
        }
    }
    dft_tubes(R, order, dims, 1);
    double nre = 0, nim = 0;
    for (int64_t i = 0; i < N; ++i) {
        nre += creal(R[i]) * creal(R[i]);
        nim += cimag(R[i]) * cimag(R[i]);
        Z[i] = creal(R[i]);
    }
    if (sqrt(nim) > 1e-12 * (sqrt(nre) + 1e-300) && nim > 0) status = ORC_EIMAG;
    double t = 0;
    for (int64_t s = 0; s < ns; ++s) t += nuc[s];
    if (tnn) *tnn = t;
    if (multirank) for (int64_t s = 0; s < ns; ++s) multirank[s] = rk[s];
    free(X); free(R); free(nuc); free(rk);
    return status;
}

/* Threshold used by the ADMM Z-step for penalty rho (see the reading in the file header). */
static double tnn_tau(int order, const int64_t* dims, double rho, int tnn_scale)
{
    return (tnn_scale == ORC_SCALE_SUM ? (double)prod_dims(dims, 2, order) : 1.0) / rho;
}

/* ------------------------------------------------------------------------------------------
 * TNN tensor completion by ADMM (Sec. 4, eq. proj, eq. shrink, dual ascent), scaled dual Q:
 *   init  X = Y = P_Omega(M), Z = 0, Q = 0, rho = rho0
 *   for k = 0..iters-1:
 *     X = P_Omega(M) + P_Omega^c(Z - Q)                  (eq. proj)
 *     Z = tSVT(X + Q, tau(rho))                          (eq. shrink, per slice eq. shrink2)
 *     Q = Q + X - Z                                      (dual ascent)
 *     rho' = min(mu rho, rho_max);  Q = Q rho / rho';  rho = rho'
 * Returns X (feasible) and Z of the last iteration; optionally the scaled dual Q and the
 * penalty rho after the last iteration.
 * ---------------------------------------------------------------------------------------- */
int orc_tnn_complete(int order, const int64_t* dims, const double* M, const uint8_t* omega,
                     int iters, double rho0, double mu, double rho_max, int tnn_scale,
                     double* X_out, double* Z_out, double* Q_out, double* rho_out)
{
    if (order < 3 || !check_dims(order, dims) || !M || !omega || iters < 0 || !(rho0 > 0) ||
        !(mu >= 1) || !(rho_max >= rho0) || !X_out)
        return ORC_EINVAL;
    const int64_t N = prod_dims(dims, 0, order);
    double* X = X_out;
    double* Z = (double*)calloc((size_t)N, sizeof(double));
    double* Q = (double*)calloc((size_t)N, sizeof(double));
    double* V = (double*)malloc(sizeof(double) * (size_t)N);
    if (!Z || !Q || !V) { free(Z); free(Q); free(V); return ORC_ENOMEM; }
    for (int64_t i = 0; i < N; ++i) X[i] = omega[i] ? M[i] : 0.0;
    double rho = rho0;
    int status = ORC_OK;
    for (int k = 0; k < iters; ++k) {
        for (int64_t i = 0; i < N; ++i) X[i] = omega[i] ? M[i] : Z[i] - Q[i];
        for (int64_t i = 0; i < N; ++i) V[i] = X[i] + Q[i];
        const int st = orc_tsvt(order, dims, V, tnn_tau(order, dims, rho, tnn_scale), Z, NULL, NULL);
        if (st != ORC_OK) status = st;
        for (int64_t i = 0; i < N; ++i) Q[i] = Q[i] + X[i] - Z[i];
        const double rho_next = fmin(mu * rho, rho_max);
        for (int64_t i = 0; i < N; ++i) Q[i] *= rho / rho_next;
        rho = rho_next;
    }
    if (Z_out) memcpy(Z_out, Z, sizeof(double) * (size_t)N);
    if (Q_out) memcpy(Q_out, Q, sizeof(double) * (size_t)N);
    if (rho_out) *rho_out = rho;
    free(Z); free(Q); free(V);
    return status;
}

/* Entrywise soft threshold: the prox of kappa*||.||_1 (the shrink of eq. sparse with an
 * entrywise l1 penalty). */
static void shrink_entry(int64_t N, const double* D, double kappa, double* S)
{
    for (int64_t i = 0; i < N; ++i) {
        const double a = fabs(D[i]) - kappa;
        S[i] = a > 0 ? (D[i] > 0 ? a : -a) : 0.0;
    }
}

/* Tube-wise group shrink, eq. sparse2: S(i,j,:) = (1 - kappa/||D(i,j,:)||_F)_+ D(i,j,:),
 * for every tube (i,j); the factor is 0 when the tube norm is 0. */
static void shrink_tube(int order, const int64_t* dims, const double* D, double kappa, double* S)
{
    const int64_t sl = dims[0] * dims[1], len = prod_dims(dims, 2, order);
    for (int64_t t = 0; t < sl; ++t) {
        double nrm = 0;
        for (int64_t k = 0; k < len; ++k) nrm += D[t + k * sl] * D[t + k * sl];
        nrm = sqrt(nrm);
        const double f = nrm > 0 ? fmax(1.0 - kappa / nrm, 0.0) : 0.0;
        for (int64_t k = 0; k < len; ++k) S[t + k * sl] = f * D[t + k * sl];
    }
}

/* Exported for tests: the two shrink operators. */
int orc_shrink(int order, const int64_t* dims, const double* D, double kappa, int mode, double* S)
{
    if (!check_dims(order, dims) || !D || !S || !(kappa >= 0)) return ORC_EINVAL;
    if (mode == ORC_SPARSE_TUBE) {
        if (order < 3) return ORC_EINVAL;
        shrink_tube(order, dims, D, kappa, S);
    } else {
        shrink_entry(prod_dims(dims, 0, order), D, kappa, S);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------
 * Tensor robust PCA by ADMM (Sec. 5, eq. low_rank, eq. sparse, eq. dual), scaled dual W:
 *   init  L = S = W = 0, rho = rho0
 *   for k = 0..iters-1:
 *     L = tSVT(M - S - W, tau(rho))                      (eq. low_rank)
 *     D = M - W - L;  S = shrink(D, lambda/rho)          (eq. sparse, closed form eq. sparse2
 *                                                          in tube mode; soft threshold in
 *                                                          entry mode)
 *     W = W + L + S - M                                  (eq. dual)
 *     rho' = min(mu rho, rho_max);  W = W rho / rho';  rho = rho'
 * Returns L and S of the last iteration; optionally the scaled dual W and the final rho.
 * ---------------------------------------------------------------------------------------- */
int orc_trpca(int order, const int64_t* dims, const double* M, double lambda, int iters,
              double rho0, double mu, double rho_max, int tnn_scale, int sparse_mode,
              double* L_out, double* S_out, double* W_out, double* rho_out)
{
    if (order < 3 || !check_dims(order, dims) || !M || !(lambda > 0) || iters < 0 ||
        !(rho0 > 0) || !(mu >= 1) || !(rho_max >= rho0) || !L_out || !S_out)
        return ORC_EINVAL;
    const int64_t N = prod_dims(dims, 0, order);
    double* L = L_out;
    double* S = S_out;
    double* W = (double*)calloc((size_t)N, sizeof(double));
    double* V = (double*)malloc(sizeof(double) * (size_t)N);
    double* D = (double*)malloc(sizeof(double) * (size_t)N);
    if (!W || !V || !D) { free(W); free(V); free(D); return ORC_ENOMEM; }
    memset(L, 0, sizeof(double) * (size_t)N);
    memset(S, 0, sizeof(double) * (size_t)N);
    double rho = rho0;
    int status = ORC_OK;
    for (int k = 0; k < iters; ++k) {
        for (int64_t i = 0; i < N; ++i) V[i] = M[i] - S[i] - W[i];
        const int st = orc_tsvt(order, dims, V, tnn_tau(order, dims, rho, tnn_scale), L, NULL, NULL);
        if (st != ORC_OK) status = st;
        for (int64_t i = 0; i < N; ++i) D[i] = M[i] - W[i] - L[i];
        if (sparse_mode == ORC_SPARSE_TUBE) shrink_tube(order, dims, D, lambda / rho, S);
        else shrink_entry(N, D, lambda / rho, S);
        for (int64_t i = 0; i < N; ++i) W[i] = W[i] + L[i] + S[i] - M[i];
        const double rho_next = fmin(mu * rho, rho_max);
        for (int64_t i = 0; i < N; ++i) W[i] *= rho / rho_next;
        rho = rho_next;
    }
    if (W_out) memcpy(W_out, W, sizeof(double) * (size_t)N);
    if (rho_out) *rho_out = rho;
    free(W); free(V); free(D);
    return status;
}

/* ------------------------------------------------------------------------------------------
 * Tensor algebra used by the tests and the data generator checks.
 * ---------------------------------------------------------------------------------------- */

/* t-product C = A * B (Def. 2.1.1), computed by the FFT route of Sec. 2.1: DFT both along
 * modes 3..N (for N = 3 the mode-3 DFT of the definition; for N > 3 the loop of Algorithm 1
 * over every mode from 3 on, so that the product is the multi-dimensional circular
 * convolution of the tubes), multiply matching Fourier slices, inverse DFT.  A has dims
 * (n1, n2, n3, ...), B (n2, n4, n3, ...), C (n1, n4, n3, ...). */
int orc_tproduct_nd(int order, const int64_t* dims, int64_t n4, const double* A, const double* B,
                    double* C)
{
    if (order < 3 || !check_dims(order, dims) || n4 < 1 || !A || !B || !C) return ORC_EINVAL;
    const int64_t n1 = dims[0], n2 = dims[1], ns = prod_dims(dims, 2, order);
    int64_t db[ORC_MAX_ORDER], dc[ORC_MAX_ORDER];
    for (int d = 0; d < order; ++d) db[d] = dc[d] = dims[d];
    db[0] = n2;
    db[1] = n4;
    dc[1] = n4;
    cplx* Ah = (cplx*)malloc(sizeof(cplx) * (size_t)(n1 * n2 * ns));
    cplx* Bh = (cplx*)malloc(sizeof(cplx) * (size_t)(n2 * n4 * ns));
    cplx* Ch = (cplx*)calloc((size_t)(n1 * n4 * ns), sizeof(cplx));
    if (!Ah || !Bh || !Ch) { free(Ah); free(Bh); free(Ch); return ORC_ENOMEM; }
    for (int64_t i = 0; i < n1 * n2 * ns; ++i) Ah[i] = A[i];
    for (int64_t i = 0; i < n2 * n4 * ns; ++i) Bh[i] = B[i];
    dft_tubes(Ah, order, dims, 0);
    dft_tubes(Bh, order, db, 0);
    for (int64_t k = 0; k < ns; ++k)
        for (int64_t j = 0; j < n4; ++j)
            for (int64_t l = 0; l < n2; ++l) {
                const cplx b = Bh[l + j * n2 + k * n2 * n4];
                for (int64_t i = 0; i < n1; ++i)
                    Ch[i + j * n1 + k * n1 * n4] += Ah[i + l * n1 + k * n1 * n2] * b;
            }
    dft_tubes(Ch, order, dc, 1);
    for (int64_t i = 0; i < n1 * n4 * ns; ++i) C[i] = creal(Ch[i]);
    free(Ah); free(Bh); free(Ch);
    return ORC_OK;
}

int orc_tproduct(int64_t n1, int64_t n2, int64_t n4, int64_t n3, const double* A, const double* B,
                 double* C)
{
    const int64_t da[3] = {n1, n2, n3};
    return orc_tproduct_nd(3, da, n4, A, B, C);
}

/* Tensor transpose (Def. 2.1.2): transpose every frontal slice, then reverse the order of
 * slices 2..n3; for order N > 3 the slice at (k3, ..., kN) takes the transposed slice at
 * (-k3 mod n3, ..., -kN mod nN), the conjugate partner, so that the transpose is the
 * conjugate transpose of every Fourier slice for any order.  A has dims (n1, n2, ...), AT
 * (n2, n1, ...). */
int orc_ttranspose_nd(int order, const int64_t* dims, const double* A, double* AT)
{
    if (order < 3 || !check_dims(order, dims) || !A || !AT) return ORC_EINVAL;
    const int64_t n1 = dims[0], n2 = dims[1], ns = prod_dims(dims, 2, order);
    for (int64_t k = 0; k < ns; ++k) {
        const int64_t src = conj_partner(order, dims, k);
        for (int64_t j = 0; j < n2; ++j)
            for (int64_t i = 0; i < n1; ++i)
                AT[j + i * n2 + k * n2 * n1] = A[i + j * n1 + src * n1 * n2];
    }
    return ORC_OK;
}

int orc_ttranspose(int64_t n1, int64_t n2, int64_t n3, const double* A, double* AT)
{
    const int64_t da[3] = {n1, n2, n3};
    return orc_ttranspose_nd(3, da, A, AT);
}

/* Full t-SVD M = U * S * V^T (Theorem 2.2.1) by Algorithm 1: DFT along modes 3..N, full SVD
 * of each Fourier slice (shared by conjugate partners, real on self-conjugate slices),
 * inverse DFT of the three factor tensors.  M has dims (n1, n2, n3, ...); U (n1, n1, ...),
 * S (n1, n2, ...), V (n2, n2, ...), all real.  Returns ORC_EIMAG if an inverse-transformed
 * factor is not real. */
int orc_tsvd_nd(int order, const int64_t* dims, const double* M, double* U, double* S, double* V)
{
    if (order < 3 || !check_dims(order, dims) || !M || !U || !S || !V) return ORC_EINVAL;
    const int64_t n1 = dims[0], n2 = dims[1], ns = prod_dims(dims, 2, order);
    const int64_t k0 = n1 < n2 ? n1 : n2;
    int64_t du[ORC_MAX_ORDER], dv[ORC_MAX_ORDER];
    for (int d = 0; d < order; ++d) du[d] = dv[d] = dims[d];
    du[1] = n1;
    dv[0] = n2;
    cplx* Mh = (cplx*)malloc(sizeof(cplx) * (size_t)(n1 * n2 * ns));
    cplx* Uh = (cplx*)malloc(sizeof(cplx) * (size_t)(n1 * n1 * ns));
    cplx* Sh = (cplx*)calloc((size_t)(n1 * n2 * ns), sizeof(cplx));
    cplx* Vh = (cplx*)malloc(sizeof(cplx) * (size_t)(n2 * n2 * ns));
    double* sg = (double*)malloc(sizeof(double) * (size_t)k0);
    if (!Mh || !Uh || !Sh || !Vh || !sg) {
        free(Mh); free(Uh); free(Sh); free(Vh); free(sg);
        return ORC_ENOMEM;
    }
    for (int64_t i = 0; i < n1 * n2 * ns; ++i) Mh[i] = M[i];
    dft_tubes(Mh, order, dims, 0);
    int status = ORC_OK;
    for (int64_t k = 0; k < ns; ++k) {
        const int64_t p = conj_partner(order, dims, k);
        cplx* Uk = Uh + k * n1 * n1;
        cplx* Vk = Vh + k * n2 * n2;
        cplx* Sk = Sh + k * n1 * n2;
        if (p < k) {
            const cplx* Up = Uh + p * n1 * n1;
            const cplx* Vp = Vh + p * n2 * n2;
            const cplx* Sp = Sh + p * n1 * n2;
            for (int64_t i = 0; i < n1 * n1; ++i) Uk[i] = conj(Up[i]);
            for (int64_t i = 0; i < n2 * n2; ++i) Vk[i] = conj(Vp[i]);
            for (int64_t i = 0; i < n1 * n2; ++i) Sk[i] = Sp[i];
            continue;
        }
        cplx* A = Mh + k * n1 * n2;
        if (p == k)
            for (int64_t i = 0; i < n1 * n2; ++i) A[i] = creal(A[i]);
        if (svd_full(n1, n2, A, Uk, sg, Vk) < 0) status = ORC_ENOTCONV;
        for (int64_t i = 0; i < k0; ++i) Sk[i + i * n1] = sg[i];
    }
    dft_tubes(Uh, order, du, 1);
    dft_tubes(Sh, order, dims, 1);
    dft_tubes(Vh, order, dv, 1);
    double im = 0, re = 0;
    for (int64_t i = 0; i < n1 * n1 * ns; ++i) { U[i] = creal(Uh[i]); re += creal(Uh[i]) * creal(Uh[i]); im += cimag(Uh[i]) * cimag(Uh[i]); }
    for (int64_t i = 0; i < n1 * n2 * ns; ++i) { S[i] = creal(Sh[i]); re += creal(Sh[i]) * creal(Sh[i]); im += cimag(Sh[i]) * cimag(Sh[i]); }
    for (int64_t i = 0; i < n2 * n2 * ns; ++i) { V[i] = creal(Vh[i]); re += creal(Vh[i]) * creal(Vh[i]); im += cimag(Vh[i]) * cimag(Vh[i]); }
    if (sqrt(im) > 1e-12 * sqrt(re) && status == ORC_OK) status = ORC_EIMAG;
    free(Mh); free(Uh); free(Sh); free(Vh); free(sg);
    return status;
}

int orc_tsvd(int64_t n1, int64_t n2, int64_t n3, const double* M, double* U, double* S, double* V)
{
    const int64_t dm[3] = {n1, n2, n3};
    return orc_tsvd_nd(3, dm, M, U, S, V);
}

/* ------------------------------------------------------------------------------------------
 * t-SVD compression (Sec. 3).  The t-SVD of Algorithm 1 gives, in every Fourier slice, the
 * f-diagonal entries of S-hat (the slice's singular values).  Method 1 (t-SVD compression)
 * keeps the k largest of those entries over all slices; an entry equal to the k-th largest is
 * kept too, so that a slice and its conjugate partner, which have equal singular values, keep
 * the same terms and the result stays real.  Method 2 (t-SVD-tubal compression) keeps the
 * first k of every slice, i.e. the first k singular tubes.  Z is the inverse DFT of
 * Z-hat = sum over the kept terms of sigma u v^H; *kept receives the number of entries kept.
 * ---------------------------------------------------------------------------------------- */
enum { ORC_COMPRESS_GLOBAL = 1, ORC_COMPRESS_TUBAL = 2 };

static int cmp_desc(const void* a, const void* b)
{
    const double x = *(const double*)a, y = *(const double*)b;
    return (x < y) - (x > y);
}

int orc_compress(int order, const int64_t* dims, const double* M, int method, int64_t k,
                 double* Z, int64_t* kept)
{
    if (order < 3 || !check_dims(order, dims) || !M || !Z) return ORC_EINVAL;
    const int64_t n1 = dims[0], n2 = dims[1], ns = prod_dims(dims, 2, order);
    const int64_t k0 = n1 < n2 ? n1 : n2;
    if (method == ORC_COMPRESS_TUBAL ? (k < 1 || k > k0)
        : method == ORC_COMPRESS_GLOBAL ? (k < 1 || k > k0 * ns) : 1)
        return ORC_EINVAL;
    cplx* Mh = (cplx*)malloc(sizeof(cplx) * (size_t)(n1 * n2 * ns));
    cplx* Uh = (cplx*)malloc(sizeof(cplx) * (size_t)(n1 * n1 * ns));
    cplx* Vh = (cplx*)malloc(sizeof(cplx) * (size_t)(n2 * n2 * ns));
    cplx* Zh = (cplx*)calloc((size_t)(n1 * n2 * ns), sizeof(cplx));
    double* sg = (double*)malloc(sizeof(double) * (size_t)(k0 * ns));
    double* sorted = (double*)malloc(sizeof(double) * (size_t)(k0 * ns));
    if (!Mh || !Uh || !Vh || !Zh || !sg || !sorted) {
        free(Mh); free(Uh); free(Vh); free(Zh); free(sg); free(sorted);
        return ORC_ENOMEM;
    }
    for (int64_t i = 0; i < n1 * n2 * ns; ++i) Mh[i] = M[i];
    dft_tubes(Mh, order, dims, 0);
    int status = ORC_OK;
    /* the SVD of every Fourier slice, shared by conjugate partners as in the t-SVD */
    for (int64_t s = 0; s < ns; ++s) {
        const int64_t p = conj_partner(order, dims, s);
        cplx* Us = Uh + s * n1 * n1;
        cplx* Vs = Vh + s * n2 * n2;
        if (p < s) {
            for (int64_t i = 0; i < n1 * n1; ++i) Us[i] = conj(Uh[p * n1 * n1 + i]);
            for (int64_t i = 0; i < n2 * n2; ++i) Vs[i] = conj(Vh[p * n2 * n2 + i]);
            for (int64_t i = 0; i < k0; ++i) sg[s * k0 + i] = sg[p * k0 + i];
            continue;
        }
        cplx* A = Mh + s * n1 * n2;
        if (p == s)
            for (int64_t i = 0; i < n1 * n2; ++i) A[i] = creal(A[i]);
        if (svd_full(n1, n2, A, Us, sg + s * k0, Vs) < 0) status = ORC_ENOTCONV;
    }
    /* the kept entries: a threshold at the k-th largest (Method 1) or the first k (Method 2) */
    double thr = 0.0;
    if (method == ORC_COMPRESS_GLOBAL) {
        memcpy(sorted, sg, sizeof(double) * (size_t)(k0 * ns));
        qsort(sorted, (size_t)(k0 * ns), sizeof(double), cmp_desc);
        thr = sorted[k - 1];
    }
    int64_t count = 0;
    for (int64_t s = 0; s < ns; ++s) {
        const cplx* Us = Uh + s * n1 * n1;
        const cplx* Vs = Vh + s * n2 * n2;
        cplx* Zs = Zh + s * n1 * n2;
        for (int64_t g = 0; g < k0; ++g) {
            const double sv = sg[s * k0 + g];
            const int keep = method == ORC_COMPRESS_TUBAL ? (g < k) : (sv >= thr);
            if (!keep) continue;
            ++count;
            for (int64_t j = 0; j < n2; ++j) {
                const cplx v = conj(Vs[j + g * n2]) * sv;
                for (int64_t i = 0; i < n1; ++i) Zs[i + j * n1] += Us[i + g * n1] * v;
            }
        }
    }
    dft_tubes(Zh, order, dims, 1);
    double im = 0, re = 0;
    for (int64_t i = 0; i < n1 * n2 * ns; ++i) {
        Z[i] = creal(Zh[i]);
        re += creal(Zh[i]) * creal(Zh[i]);
        im += cimag(Zh[i]) * cimag(Zh[i]);
    }
    if (sqrt(im) > 1e-12 * (sqrt(re) + 1e-300) && im > 0 && status == ORC_OK) status = ORC_EIMAG;
    if (kept) *kept = count;
    free(Mh); free(Uh); free(Vh); free(Zh); free(sg); free(sorted);
    return status;
}
