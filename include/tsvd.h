/*
 * tsvd.h -- C ABI of libtsvd: tensor singular value thresholding (t-SVT) and the two ADMM
 * solvers built on it, from Zhang, Ely, Aeron, Hao and Kilmer, "Novel methods for
 * multilinear data completion and de-noising based on tensor-SVD" (arXiv:1407.1785).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Tensors.  A real tensor of order N = 3..6 (n1 x n2 x n3 x ... x nN) is a dense FP32 array in
 *   MATLAB column-major order: entry (i1, i2, i3, ...) (0-based) lives at
 *   i1 + n1*(i2 + n2*(i3 + n3*(...))).  `order` is N and `dims` points to N int64 extents,
 *   each >= 1.  The transformed modes are 3..N: the Fourier slices of Sec. 2 are taken along
 *   them (Algorithm 1, "fft along modes 3..N"); for N >= 5 the product n3 * ... * n(N-1) is at
 *   most 64.  tsvd_solve_batched and tsvt_static take N = 3 or 4.
 * Memory.  Every tensor pointer may be either a device pointer (on the context's device) or
 *   host memory (pinned or pageable); the library asks the CUDA runtime which it is.  Device
 *   tensors are used in place and the call returns as soon as the work is queued on the
 *   context's stream (results are ready when that stream reaches them).  Host tensors are
 *   copied to and from library-owned device buffers on the stream and the call returns after
 *   the stream has finished.  The caller owns all tensors; the library keeps no pointer
 *   after a call returns.  Small outputs (`multirank`, `tnn`, `stats`) are host pointers; a
 *   call that fills one of them waits for its stream.
 * Errors.  Every call returns a tsvd_status and never aborts; tsvd_last_error() holds a
 *   one-line reason for the last failure on that context.  TSVD_EINVAL: a null required
 *   pointer, order outside 3..6, an extent < 1, a non-finite observed entry or a bad scalar.
 *   TSVD_EUNSUPPORTED: a shape the kernels do not handle (reported before any work).
 *   TSVD_ECUDA: a CUDA runtime error.  TSVD_ENOTCONV: a tsvt() call whose Jacobi SVD of some
 *   Fourier slice reached max_sweeps (the result is still written); inside the ADMM solvers
 *   such slices are only counted in tsvd_stats.
 * Threads.  A context is not thread-safe; calls on one context run in order on its stream.
 *   Distinct contexts are independent.
 */
#ifndef TSVD_H
#define TSVD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tsvd_ctx tsvd_ctx;

typedef enum tsvd_status {
  TSVD_OK = 0,
  TSVD_EINVAL = 1,
  TSVD_ENOMEM = 2,
  TSVD_ECUDA = 3,
  TSVD_ENOTCONV = 4,
  TSVD_ETIMEOUT = 5,
  TSVD_EUNSUPPORTED = 6
} tsvd_status;

/* Arithmetic of the slice SVTs.
 *   FP32       the plain form: one-sided Jacobi SVD of every Fourier slice in FP32.
 *   TF32, BF16, 3XTF32, RAND_FP32
 *              the mixed form: a rank-adaptive randomized subspace-iteration SVT.  Per slice
 *              A: Y = A P (P warm-started from the previous call's right singular vectors),
 *              Q = CholeskyQR2(Y), D = D_tau(Q^H A) by one-sided Jacobi on the k x n matrix,
 *              Z = Q D.  The three products with A and Z run as 3M complex products on the
 *              tensor cores with TF32 operands, BF16 operands or split TF32 operands
 *              (hi*hi + hi*lo + lo*hi: FP32-level accuracy), all with FP32 accumulation;
 *              RAND_FP32 runs them in FP32 on the CUDA cores.  The result equals
 *              D_tau(Q Q^H A); it is the t-SVT when the sketch width k covers every singular
 *              value above tau (k adapts to the ranks seen, see rsvt_* options). */
enum { TSVD_PRECISION_FP32 = 0, TSVD_PRECISION_TF32 = 1, TSVD_PRECISION_BF16 = 2,
       TSVD_PRECISION_3XTF32 = 3, TSVD_PRECISION_RAND_FP32 = 4 };

/* Sparse penalty of tensor RPCA: entrywise l1 (soft threshold at lambda/rho) or the
 * tube-wise l_{1,1,2} norm of Sec. 5 (eq. sparse2; for order >= 4 the group is every entry
 * sharing (i, j), S(i,j,:,...,:)). */
enum { TSVD_SPARSE_ENTRY = 0, TSVD_SPARSE_TUBE = 1 };

/* Threshold of the ADMM low-rank step for penalty rho.  AVG: tau = 1/rho applied to the
 * singular values of the unnormalised DFT slices, i.e. eq. shrink as printed (the prox of
 * TNN/P in the original domain, P = number of Fourier slices).  SUM: tau = P/rho, the prox
 * of the TNN exactly as defined in Thm 2.4.1 (sum over all Fourier slices). */
enum { TSVD_SCALE_AVG = 0, TSVD_SCALE_SUM = 1 };

/* Warm start of the plain-form slice SVDs inside ADMM solves (tsvd_opts.warm_start). */
enum { TSVD_WARM_OFF = 0, TSVD_WARM_ON = 1, TSVD_WARM_AUTO = 2 };

typedef struct tsvd_opts {
  int precision;      /* TSVD_PRECISION_*; default FP32 */
  int sparse_mode;    /* TSVD_SPARSE_*; default ENTRY */
  int tnn_scale;      /* TSVD_SCALE_*; default AVG */
  double rho0;        /* initial ADMM penalty; default 1e-2 */
  double mu;          /* penalty growth per iteration, rho <- min(mu*rho, rho_max); 1.1 */
  double rho_max;     /* penalty cap; default 1e10 */
  int max_sweeps;     /* Jacobi sweep cap per slice SVD; default 40 */
  float jacobi_tol;   /* rotate a pair while |x^H y| > tol ||x|| ||y||; default 1e-6 */
  int timing;         /* 1: time every kernel launch with CUDA events on the context's stream
                         and report the totals in tsvd_stats; default 0 */
  int ctas_per_slice; /* CTAs (one thread-block cluster) per Fourier slice SVD: 1, 2, 4 or 8;
                         TSVD_CTAS_FEWEST (-1): the fewest that hold the slice (for launches
                         that share the GPU, e.g. many tensors at once); 0 (default) = chosen
                         from the slice shape and count as if the launch had the GPU alone */
  int accumulate_v;   /* 1: also rotate V during the Jacobi sweeps and rebuild each slice as
                         W diag((s - tau)/s) V^H instead of U diag((s - tau)/s) U^H A;
                         default 0 */
  int lanes_per_pair; /* lanes that share one vector pair: 4, 8, 16 or 32; 0 (default) = chosen */
  int autotune;       /* 1 (default): the first slice-SVT launch of each new slice shape in a
                         context times the valid (ctas_per_slice, lanes_per_pair) plans on the
                         real input (sweeps capped at 4) and keeps the fastest; choices fixed
                         by nonzero ctas_per_slice / lanes_per_pair are kept */
  const char* autotune_cache; /* nullable: text file of tuned plans keyed by GPU name and
                         slice shape, read at the first tuning and appended to after it */
  int use_graphs;     /* 1 (default): tnn_complete / trpca capture their whole launch sequence
                         (all iterations) into a CUDA graph on a private stream the first time
                         a given (buffers, shape, iterations, options) combination runs with a
                         settled plan, and replay it on the context's stream afterwards
                         (the mixed precisions choose the sketch width on the host during a
                         solve and are not captured) */
  int rsvt_oversample; /* mixed form: sketch width = (singular values above the threshold and
                         the products' noise floor) + this margin, rounded up to 8; the
                         width only grows during a solve; default 10 */
  int rsvt_kmax;      /* mixed form: largest sketch width (<= 128 and <= min(n1, n2));
                         0 (default) = min(128, n1, n2) */
  int rsvt_power;     /* mixed form, tsvt() only: extra power steps from a random start
                         (ADMM solves start each iteration from the previous basis);
                         default 2 */
  int warm_start;     /* plain form, tnn_complete / trpca: a warm start begins each slice's
                         Jacobi SVD from the previous iteration's right singular vectors V
                         (the slice is pre-rotated to B V and the rotations accumulate into V,
                         the V form), with a cold start every 64 iterations; the rebuild
                         still projects B itself (U form), so the result is the same SVT,
                         reached in fewer sweeps.  TSVD_WARM_OFF: every SVD starts from B.
                         TSVD_WARM_ON / TSVD_WARM_AUTO (default): warm wherever the slice
                         shape has a V-form plan (AUTO is ON; it stays a separate value so
                         that a later policy can refine it).  Measured on the completion and
                         RPCA workloads, warm solves take 2.5-3x fewer sweeps than cold ones,
                         which more than pays for the V form's nv extra entries per vector:
                         with the SVT stopping test (jacobi_stop) the directions of the
                         FP32-noise tail, which change at every iteration of an RPCA solve,
                         no longer cost rotations. */
  int batch_persistent; /* plain form, batched solves: 1 runs each ADMM iteration of the whole
                         batch as one persistent kernel launch that takes the slice SVTs of all
                         tensors (largest first) and then their tube passes from device work
                         queues, a tube pass starting once its tensor's slices are done; the
                         cluster size and which tensors run one CTA per slice are autotuned per
                         batch shape (timed on the first iteration) and kept in the context.
                         0 (default): one chain of kernels per tensor on parallel stream
                         branches, which lets every tensor advance at its own pace (faster on
                         uneven batches, where the persistent form waits each iteration for
                         its slowest slice). */
  int slice_form;     /* plain-form Jacobi: TSVD_SLICE_AUTO (default: the autotuner compares
                         both forms), TSVD_SLICE_PAIRWISE (each local round rotates its vector
                         pairs directly) or TSVD_SLICE_BLOCK (each round of vector blocks runs
                         its rotations on the Gram matrix of the CTA's vectors, then applies
                         their product to the vectors: the same rotations, fewer passes over
                         the vectors) */
  int rsvt_small_fp64; /* mixed form: 1 runs the k x k CholeskyQR2 factorisations (k <= 112)
                         and the Rayleigh-Ritz eigen-solve of the projected Gram (k <= 80) in
                         FP64; 0 (default) in FP32 with the Cholesky pivots in double-single
                         arithmetic (FP32 pairs).  The Grams themselves are FP32-level
                         products either way. */
  int jacobi_stop;    /* plain-form Jacobi stopping test of the slice SVTs (tsvt, the ADMM
                         solves; tsvd_factor / tsvd_compress always use RELATIVE).
                         TSVD_STOP_RELATIVE: a vector pair (x, y) is orthogonal once
                         |x^H y| <= tol ||x|| ||y||, which orders even the tiniest singular
                         directions to full relative accuracy.  TSVD_STOP_SVT (default): also
                         once |x^H y| <= tol min(||x||, ||y||) ||B||_F / nv, i.e. once what
                         the pair still moves in the rebuilt slice D_tau(B) (about
                         |x^H y| / min(||x||, ||y||)) is below tol ||B||_F / nv (B the slice,
                         nv = min(n1, n2)), so that all pairs stopped this way together move
                         D_tau(B) by about tol ||B||_F at most.  This never rotates more than
                         RELATIVE, stays within its worst-case error per pair, and stops
                         rotating pairs of directions far below the slice's energy -- the
                         FP32-noise tail of a nearly low-rank slice, which RELATIVE would
                         orthogonalise to 1e-6 for nothing. */
} tsvd_opts;

enum { TSVD_SLICE_AUTO = 0, TSVD_SLICE_PAIRWISE = 1, TSVD_SLICE_BLOCK = 2 };
enum { TSVD_STOP_SVT = 0, TSVD_STOP_RELATIVE = 1 };
enum { TSVD_CTAS_FEWEST = -1 };

/* Counters of one ADMM solve (host struct). */
typedef struct tsvd_stats {
  int iters;                    /* ADMM iterations run */
  int max_sweeps_used;          /* most Jacobi sweeps taken by any slice SVD */
  int64_t total_sweeps;         /* Jacobi sweeps summed over all slice SVDs */
  int64_t nonconverged;         /* slice SVDs stopped by max_sweeps */
  int64_t slice_svds;           /* slice SVDs run */
  double rho_final;             /* penalty after the last iteration */
  double tnn_last;              /* TNN (sum form) of the last t-SVT input */
  int rank_last_max;            /* largest Fourier-slice rank of the last t-SVT result */
  int64_t launches;             /* kernels launched by the call */
  int64_t slice_launches;       /* of which slice-SVT launches */
  double slice_ms;              /* summed device time of the slice-SVT launches (timing=1) */
  double tube_ms;               /* summed device time of the tube-pass launches (timing=1) */
  int slice_ctas;               /* CTAs per slice of the slice-SVT plan used */
  int slice_lanes;              /* lanes per vector pair of that plan (0 = planner default) */
  int slice_pairs_in_flight;    /* vector pairs a lane group interleaves (0/1 = one) */
  int rsvt_k_last;              /* mixed form: sketch width of the last slice SVT */
  int64_t rsvt_saturated;       /* mixed form: slice SVTs whose whole sketch lay above the
                                   threshold (the result may miss directions) */
  int64_t rsvt_drops;           /* mixed form: sketch columns dropped as dependent by the
                                   CholeskyQR factorisations (refilled at random) */
  double rsvt_gemm_ms;          /* mixed form, timing=1: device time of the three slice
                                   products (sketch, projection, rebuild) */
  double rsvt_orth_ms;          /* ... of the CholeskyQR2 orthonormalisations */
  double rsvt_svd_ms;           /* ... of the small Jacobi SVTs */
  double rsvt_gemm_gflop;       /* algorithmic GFLOP of those products: 8 m n k per complex
                                   m x k times k x n product */
  double rsvt_svd_gflop;        /* Golub-Van Loan count of the small SVDs: 4 (4 n k^2 + 8 k^3)
                                   per n x k matrix */
} tsvd_stats;

/* Fill *opts with the defaults listed above. */
void tsvd_default_opts(tsvd_opts* opts);

/* Create a context on CUDA device `device`, issuing all work on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream).  `opts` may be NULL for the defaults and
 * is copied.  On success *out owns device workspaces that grow on demand; free it with
 * tsvd_destroy().  Errors: EINVAL (out == NULL, bad opts), ECUDA (device unusable). */
tsvd_status tsvd_create(tsvd_ctx** out, int device, void* cuda_stream, const tsvd_opts* opts);

/* Wait for the context's stream, release every buffer the context owns and free it.
 * NULL is accepted. */
tsvd_status tsvd_destroy(tsvd_ctx* ctx);

/* One-line description of the last failure on ctx (static string for ctx == NULL). */
const char* tsvd_last_error(const tsvd_ctx* ctx);

/* t-SVT: Z = prox of tau*TNN-per-slice, i.e. for every Fourier slice Yhat^(k) (DFT along
 * modes 3..order) Zhat^(k) = D_tau(Yhat^(k)) = U diag((sigma_i - tau)_+) V^H, then the
 * inverse DFT (Lemma and eq. shrink2 of Sec. 4.1, Algorithm 1).  tau applies to the singular
 * values of the unnormalised DFT slices.  Y and Z: dims-shaped tensors (may alias).  Unlike
 * the solvers, tsvt() always waits for its stream before returning (it reports ENOTCONV).
 * multirank (nullable, host): receives the rank of every Fourier slice of Z, prod(dims[2..])
 * int32 in column-major (k3, k4, ...) order.  tnn (nullable, host): receives the TNN of Y, the
 * sum of the singular values of all Fourier slices (Thm 2.4.1).  Errors: EINVAL (tau < 0 or
 * not finite), EUNSUPPORTED, ENOTCONV. */
tsvd_status tsvt(tsvd_ctx* ctx, const float* Y, float* Z, int order, const int64_t* dims,
                 float tau, int32_t* multirank, double* tnn);

/* Truncated t-SVD (Algorithm 1; Theorem 2.3.1): Y = U * S * V^T with the first k singular
 * tubes, where * is the t-product (Def. 2.1.1) and V^T the tensor transpose.  Per Fourier
 * slice the singular values are taken in decreasing order and the first k kept, so for
 * k = min(n1, n2) U * S * V^T reproduces Y (the economy t-SVD: U^T * U = I), and for smaller k
 * it is M_k, the best approximation of Theorem 2.3.1.  k = 0 means min(n1, n2).
 * Outputs (real, column-major, device or host, not aliasing Y): U dims (n1, k, n3, ...),
 * S dims (k, k, n3, ...) f-diagonal, V dims (n2, k, n3, ...).  The factors are unique up
 * to a phase per (slice, column) in the Fourier domain; U * S * V^T is unique when the k-th
 * and (k+1)-th singular values of every slice differ.  A column whose singular value is 0 is
 * returned as zeros in U (n1 >= n2) or V (n1 < n2).  Plain form (one-sided Jacobi, FP32)
 * whatever the context's precision; waits for its stream.  Errors: EINVAL (k < 0 or
 * k > min(n1, n2), NULL or aliasing buffers), EUNSUPPORTED, ENOTCONV, ENOMEM. */
tsvd_status tsvd_factor(tsvd_ctx* ctx, const float* Y, int order, const int64_t* dims, int k,
                        float* U, float* S, float* V);

/* t-SVD compression (Sec. 3).  Z = the tensor rebuilt from the kept Fourier-domain singular
 * terms: method TSVD_COMPRESS_GLOBAL (Method 1, t-SVD compression) keeps the k largest
 * f-diagonal entries of S-hat over all min(n1, n2) * prod(dims[2..]) of them -- every entry
 * equal to the k-th largest is kept too, so conjugate Fourier slices keep the same terms and Z
 * is real (*kept_total may exceed k); TSVD_COMPRESS_TUBAL (Method 2, t-SVD-tubal compression)
 * keeps the first k singular tubes (Z = M_k of Theorem 2.3.1, as tsvd_factor with k).
 * 1 <= k <= min(n1, n2) * prod(dims[2..]) (GLOBAL) or min(n1, n2) (TUBAL).  Z (dims-shaped,
 * may alias Y); kept_total (nullable, host): the entries kept (GLOBAL) or k (TUBAL); ratio
 * (nullable, host): the compression ratio of Sec. 3, n1 n2 prod(dims[2..]) / (kept (n1 + n2 + 1))
 * or n1 n2 / (k (n1 + n2 + 1)).  Plain form; waits for its stream.  Errors as tsvd_factor. */
enum { TSVD_COMPRESS_GLOBAL = 1, TSVD_COMPRESS_TUBAL = 2 };
tsvd_status tsvd_compress(tsvd_ctx* ctx, const float* Y, int order, const int64_t* dims,
                          int method, int64_t k, float* Z, int64_t* kept_total, double* ratio);

/* t-product C = A * B (Def. 2.1.1): tube (i, j) of C is the sum over l of the circular
 * convolutions of the tubes A(i, l, :) and B(l, j, :); for order > 3 the convolution runs over
 * every mode from 3 on, i.e. C-hat = A-hat B-hat in every slice of the DFT along modes 3..N
 * (Sec. 2.1).  A: dims (n1, n2, n3, ...), order 3 to 6 with the limits of tsvt(); B: (n2, n4,
 * n3, ...); C: (n1, n4, n3, ...); real FP32, column-major, device or host memory; C must not
 * alias A or B.  The slice products follow the context's precision (FP32 on CUDA cores for
 * TSVD_PRECISION_FP32 and RAND_FP32; 3M tensor-core products for TF32, BF16, 3XTF32).
 * Asynchronous on the context's stream for device buffers; with any buffer in host memory the
 * call returns after C is written.  Errors: EINVAL (NULL or aliasing buffers, bad order or
 * dims, n4 < 1), EUNSUPPORTED, ENOMEM. */
tsvd_status tsvd_tproduct(tsvd_ctx* ctx, const float* A, const float* B, float* C, int order,
                          const int64_t* dims, int64_t n4);

/* TNN tensor completion (Sec. 4: min ||X||_TNN s.t. P_Omega(X) = P_Omega(M), eq.
 * originalTNN) by the ADMM of eq. proj / eq. shrink / dual ascent with scaled dual Q and
 * penalty schedule rho_{k+1} = min(mu rho_k, rho_max) from opts:
 *   X = P_Omega(M) + P_Omega^c(Z - Q);  Z = tSVT(X + Q, tau(rho));  Q = (Q + X - Z) rho_k/rho_{k+1}.
 * M_obs: dims-shaped tensor whose entries are read only where omega is nonzero (they must be
 * finite there).  omega: uint8 per entry (nonzero = observed).  iters >= 0 ADMM iterations.
 * X_out: receives X of the last iteration (it agrees with M_obs on Omega).  Z_out
 * (nullable): receives Z of the last iteration.  stats (nullable, host).  Errors: EINVAL,
 * EUNSUPPORTED. */
tsvd_status tnn_complete(tsvd_ctx* ctx, const float* M_obs, const uint8_t* omega, int order,
                         const int64_t* dims, int iters, float* X_out, float* Z_out,
                         tsvd_stats* stats);

/* Tensor robust PCA (Sec. 5: min ||L||_TNN + lambda ||S||, s.t. M = L + S, eq. tensor_PCA)
 * by the ADMM of eq. low_rank / eq. sparse / eq. dual with scaled dual W:
 *   L = tSVT(M - S - W, tau(rho));  S = shrink(M - W - L, lambda/rho);
 *   W = (W + L + S - M) rho_k/rho_{k+1}.
 * The shrink is opts.sparse_mode (entrywise, or tube-wise eq. sparse2).  M: dims-shaped,
 * finite.  lambda > 0.  L_out, S_out: receive L and S of the last iteration.  stats
 * (nullable, host).  Errors: EINVAL, EUNSUPPORTED. */
tsvd_status trpca(tsvd_ctx* ctx, const float* M, int order, const int64_t* dims, float lambda,
                  int iters, float* L_out, float* S_out, tsvd_stats* stats);

/* The ADMM state a solve continues from (tnn_complete_resume, trpca_resume): the state after
 * some iterations of the same method, as returned by an earlier call.  Every pointer is a
 * device pointer on the context's device, dims-shaped, or NULL for a zero tensor. */
typedef struct tsvd_admm_state {
  const float* Z;       /* completion: Z of the last iteration */
  const float* Q;       /* completion: scaled dual Q after the last iteration */
  const float* S;       /* RPCA: S of the last iteration */
  const float* W;       /* RPCA: scaled dual W after the last iteration */
  double rho;           /* penalty to continue with (> 0), e.g. tsvd_stats.rho_final of the
                           earlier call; <= 0: opts.rho0 */
} tsvd_admm_state;

/* tnn_complete continued from a state: `iters` (>= 1) more iterations of the same ADMM from
 * (Z, Q, rho) instead of Z = Q = 0, rho = rho0, so that k1 iterations followed by a resumed
 * call of k2 iterations (fed the first call's Z_out, Q_out and rho_final) compute what one
 * call of k1 + k2 iterations computes.  init may be NULL (a fresh start).  Q_out (nullable,
 * device): receives the scaled dual after the last iteration, rescaled to the final rho
 * (stats->rho_final).  Other arguments, memory and errors as tnn_complete, plus EINVAL for
 * host state pointers or iters < 1 with init. */
tsvd_status tnn_complete_resume(tsvd_ctx* ctx, const float* M_obs, const uint8_t* omega,
                                int order, const int64_t* dims, int iters,
                                const tsvd_admm_state* init, float* X_out, float* Z_out,
                                float* Q_out, tsvd_stats* stats);

/* trpca continued from a state: `iters` (>= 1) more iterations from (S, W, rho); W_out
 * (nullable, device) receives the scaled dual after the last iteration.  Otherwise as trpca
 * and tnn_complete_resume. */
tsvd_status trpca_resume(tsvd_ctx* ctx, const float* M, int order, const int64_t* dims,
                         float lambda, int iters, const tsvd_admm_state* init, float* L_out,
                         float* S_out, float* W_out, tsvd_stats* stats);

/* One tensor of a batched solve (tsvd_solve_batched). */
enum { TSVD_PROBLEM_COMPLETE = 1, TSVD_PROBLEM_RPCA = 2 };
typedef struct tsvd_problem {
  int kind;             /* TSVD_PROBLEM_COMPLETE or TSVD_PROBLEM_RPCA */
  int order;            /* 3 or 4 */
  int64_t dims[4];      /* n1, n2, n3[, n4] */
  const float* M;       /* completion: observed tensor (read on omega); RPCA: M */
  const uint8_t* omega; /* completion: uint8 mask; RPCA: unused (NULL) */
  float lambda;         /* RPCA: sparse weight (> 0); completion: unused */
  float* out0;          /* completion: X; RPCA: L */
  float* out1;          /* completion: Z (nullable); RPCA: S */
} tsvd_problem;

/* Batched solve: runs `iters` ADMM iterations of every problem -- TNN completion (as
 * tnn_complete) or tensor RPCA (as trpca) -- for `count` tensors of any shapes, with the
 * context's options (one rho schedule for all).  With a mixed precision each tensor's sketch
 * width is chosen on the device after every iteration (same rule as the single-tensor
 * solvers, widths up to 112), so the whole batch is still captured into one graph.  In the
 * plain form each tensor follows warm_start as the single-tensor solvers do.  All pointers
 * must be device memory on the context's device.  Each tensor's iterations form an
 * independent chain of kernels (its own slice-SVT plan); the chains of all tensors are issued
 * on parallel stream branches and, with
 * use_graphs, captured once into one CUDA graph that later calls with the same problems
 * replay, so the tensors overlap on the GPU.  Plans come from the context's autotune cache
 * for shapes tuned earlier, else from the planner (no tuning inside a batch).  stats
 * (nullable, host) sums the counters over the batch.  Errors as tnn_complete / trpca, per
 * problem; nothing is launched if any problem is invalid. */
tsvd_status tsvd_solve_batched(tsvd_ctx* ctx, int count, const tsvd_problem* problems, int iters,
                               tsvd_stats* stats);

/* The batched solve restricted to one method: TNN completion of `count` tensors (Sec. 4, as
 * tnn_complete; every problem of kind TSVD_PROBLEM_COMPLETE) or tensor RPCA of `count`
 * tensors (Sec. 5, as trpca; every problem of kind TSVD_PROBLEM_RPCA).  Same arguments,
 * memory rules, scheduling and errors as tsvd_solve_batched, plus EINVAL when a problem is of
 * the other kind. */
tsvd_status tnn_complete_batched(tsvd_ctx* ctx, int count, const tsvd_problem* problems,
                                 int iters, tsvd_stats* stats);
tsvd_status trpca_batched(tsvd_ctx* ctx, int count, const tsvd_problem* problems, int iters,
                          tsvd_stats* stats);

/* Operand forms of tsvd_cgemm: as stored, transposed, conjugate-transposed. */
enum { TSVD_OP_N = 0, TSVD_OP_T = 1, TSVD_OP_C = 2 };

/* Batched complex product of Fourier slices, C_b = op(A_b) op(B_b) for b < batch: the
 * slice-wise product by which the t-product is computed in the Fourier domain (Sec. 2.1),
 * and the engine of the mixed form's slice products.  Complex single precision, interleaved
 * (re, im), column-major: entry (i, j) of a matrix with leading dimension ld at float offset
 * 2 (i + j ld); matrix b of A starts stride_a complex entries after matrix b - 1 (likewise
 * for B and C).  op(A) is m x k, op(B) is k x n, C is m x n (lda, ldb, ldc >= the stored
 * row counts).  Arithmetic follows the context's precision: FP32 and RAND_FP32 on CUDA cores
 * in FP32; TF32, BF16 and 3XTF32 as 3M products on the tensor cores (see
 * TSVD_PRECISION_*).  A, B and C are device pointers on the context's device (C must not
 * overlap A or B); asynchronous on the context's stream.  Errors: EINVAL (bad sizes, strides
 * or pointers). */
tsvd_status tsvd_cgemm(tsvd_ctx* ctx, int transa, int transb, int m, int n, int k,
                       const float* A, int64_t lda, int64_t stride_a, const float* B,
                       int64_t ldb, int64_t stride_b, float* C, int64_t ldc, int64_t stride_c,
                       int batch);

/* Testing aid (not a step of the paper's method): host-side fault injection.  With the spec
 * "alloc:N" (from the TSVD_FAULT environment variable, read at the library's first device
 * allocation, or given here) the N-th device allocation the library makes in this process,
 * counting from 1, fails as if the device had no memory left, so the call that makes it
 * returns TSVD_ENOMEM; the allocations before and after it are unaffected.  This call re-reads
 * the spec (spec = NULL: the environment variable again), restarts the count and returns N (0:
 * off, also for a spec it cannot parse).  Needs no device. */
long long tsvd_fault_injection_reset(const char* spec);

/* Testing aid (not a step of the paper's method): runs, on device `device`, the bounded wait
 * the persistent batched kernel uses for its dependencies, on a device counter that nothing
 * raises, with a limit of limit_ms milliseconds (0..10000).  The wait must give up: the call
 * returns TSVD_ETIMEOUT, the way a batched solve reports a dependency that never arrived, and
 * leaves the device usable.  TSVD_OK would mean the wait did not end by its limit.  Errors:
 * EINVAL (limit out of range), ENOMEM, ECUDA. */
tsvd_status tsvd_selftest_bounded_wait(int device, int limit_ms);

/* Measurement aid (not a step of the paper's method): the FP32 CUDA-core throughput of device
 * `device` in TFLOP/s (2 flops per fused multiply-add), measured with a loop of independent
 * scalar FMAs (*tflops_fma) and of packed FP32x2 FMAs (*tflops_fma2, the instruction form of
 * the Jacobi kernels), each the best of 5 launches of 16 blocks of 1024 threads per SM timed
 * with CUDA events.  This is the denominator of the FP32 ("alu") rooflines of the slice SVT.
 * Allocates 4 bytes of device memory and a stream for the duration of the call and waits for
 * them.  Errors: EINVAL (NULL outputs), ECUDA. */
tsvd_status tsvd_measure_fp32_peak(int device, double* tflops_fma, double* tflops_fma2);

/* The paper has no counterpart to this entry point; it exists for callers that cannot
 * allocate device memory.  Some callers cannot call cudaMalloc: a process that has handed the
 * whole device memory budget to its own pool allocator (a later cudaMalloc fails or fragments
 * the pool), or a latency-critical loop that must not pay the implicit device-wide
 * synchronisation of cudaMalloc / cudaFree.  tsvt() allocates its workspace on first use, so
 * tsvt_static() computes the same t-SVT (same kernels, default opts) with every byte of its
 * scratch taken from one fixed 64 MiB array in the library's device memory, and calls no
 * cudaMalloc, cudaFree or allocating library routine.
 * Y, Z: device pointers on the current device (host memory is rejected), dims-shaped as for
 * tsvt(); Y and Z may alias.  The work is queued on `cuda_stream` (a cudaStream_t, NULL =
 * legacy default stream) and the call returns without waiting; no multi-rank, TNN or
 * convergence report: TSVD_OK means the work was queued, not that every slice SVD converged
 * within the default 40 sweeps (tsvt() reports that case as TSVD_ENOTCONV).  Each call's
 * tables (twiddles, distinct-slice list) are written into the array by its first kernel from
 * the launch arguments; no host buffer is read on the GPU.
 * Limit: 2 * 8 * n1*n2*P_half bytes of spectra plus small tables must fit in 64 MiB, where
 * P_half = floor(n3/2)+1 (order 3) or n3*(floor(n4/2)+1) (order 4); larger problems return
 * TSVD_ENOMEM before any work.  Every GPU that loads the library holds the 64 MiB until the
 * process exits.  The first call on a device (with that device current) looks up the array's
 * device address once; make it before any stream capture.  That address is cached for the
 * process: resetting the device (cudaDeviceReset) while the library is loaded is not
 * supported.  All calls on a device share the array: calls that overlap on the GPU race and
 * corrupt each other, so order them (one stream, or events).  Errors: EINVAL (null or host
 * pointer, bad order/dims/tau), EUNSUPPORTED, ENOMEM (over the limit), ECUDA. */
tsvd_status tsvt_static(const float* Y, float* Z, int order, const int64_t* dims, float tau,
                        void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* TSVD_H */
