// tsvd_internal.h -- declarations shared by the CUDA translation units of libtsvd.
// Not part of the public C ABI (that is include/tsvd.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace tsvd {

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount, cached per
// device); the planners size grids and waves with it.
int device_sm_count();

// Geometry of the tube passes.  A real tensor of order 3 to 6 is stored MATLAB column-major;
// the "tube" of pixel t = i + n1*j is the set of entries t + N12*(jf + nf*jh).  The last
// mode (length nh) is transformed real-to-complex and only its first hh = nh/2+1 frequencies
// are kept; modes 3..N-1 (flat index jf, mode 3 fastest, nf entries in all) take a full
// complex DFT.  A 3-way tensor has nf = 1, nh = n3.
// Fourier slice (kf, kh) is stored at slice index kf + nf*kh, as an n1 x n2 complex matrix
// (float2, column-major), i.e. spectrum entry (t, kf, kh) at t + N12*(kf + nf*kh).
struct TubeGeom {
  int64_t N12;   // number of tubes (n1*n2)
  int nf;        // full-DFT index length: the product of modes 3..N-1 (1 for 3-way)
  int nh;        // half-spectrum mode length (mode N)
  int hh;        // nh/2 + 1
  int nstore;    // nf*hh stored Fourier slices
  int nfm = 0;                  // number of full-DFT modes (N - 3)
  int fdim[4] = {0, 0, 0, 0};   // their sizes, mode 3 first (its index varies fastest in kf)
};

// (cos, sin)(2 pi m / n) computed in FP64 and rounded once to FP32, exact at the quarter
// points: the twiddle factor of every DFT table of the library (host and device).
__host__ __device__ inline float2 twiddle_value(int m, int n) {
  double c, s;
  if (m == 0) {
    c = 1.0;
    s = 0.0;
  } else if (2 * m == n) {
    c = -1.0;
    s = 0.0;
  } else if (4 * m == n) {
    c = 0.0;
    s = 1.0;
  } else if (4 * m == 3 * n) {
    c = 0.0;
    s = -1.0;
  } else {
    const double a = 2.0 * 3.14159265358979323846 * (double)m / (double)n;
    c = cos(a);
    s = sin(a);
  }
  return make_float2((float)c, (float)s);
}

// Flat full index of the conjugate partner of full index kf: (-k3 mod n3, -k4 mod n4, ...).
__host__ __device__ inline int full_partner(const TubeGeom& g, int kf) {
  if (g.nfm <= 1) return (g.nf - kf) % g.nf;
  int r = 0, mul = 1, rem = kf;
  for (int d = 0; d < g.nfm; ++d) {
    const int n = g.fdim[d], k = rem % n;
    rem /= n;
    r += ((n - k) % n) * mul;
    mul *= n;
  }
  return r;
}

// Stored slice (kf, kh) is computed by the t-SVT unless it is the conjugate partner of an
// earlier stored slice: only possible on the self-conjugate columns kh = 0, nh/2, where a
// slice and its partner are conjugates and the one with the smaller full index is computed.
__host__ __device__ inline bool slice_is_distinct(const TubeGeom& g, int kf, int kh) {
  const bool selfcol = (kh == 0) || (2 * kh == g.nh);
  return !(selfcol && full_partner(g, kf) < kf);
}

// Work modes of the tube pass.
enum TubeMode : int {
  TUBE_FWD = 0,        // V = input; Vhat = R2C(V)                    (t-SVT input / first pass)
  TUBE_INV = 1,        // out = C2R(spec)                              (t-SVT output / last pass)
  TUBE_COMPLETE = 2,   // fused completion pass, see tube_pass.cu
  TUBE_RPCA = 3,       // fused RPCA pass, see tube_pass.cu
};

struct TubeArgs {
  TubeGeom g;
  int mode;
  const float2* spec_in;  // Zhat / Lhat (nullable in the first pass)
  float2* spec_out;       // Vhat (nullable in the last pass)
  const float2* twid_h;   // nh entries (cos, sin)(2 pi m / nh)
  const float2* twid_f;   // nf entries
  // more than one full-DFT mode (order >= 5): the nf x nf matrix of the multi-dimensional
  // DFT, fmat[o * nf + f] = exp(+2 pi i sum_d o_d f_d / n_d), and the conjugate partner of
  // every full index (the flat index of (-k3 mod n3, ...)); nullptr for order <= 4, where the
  // kernels use twid_f and the partner nf - kf
  const float2* fmat = nullptr;
  const int* fpart = nullptr;
  const float* in;        // TUBE_FWD: input tensor; COMPLETE: Yn (NaN = unobserved); RPCA: M
  float* state;           // COMPLETE: V = X + Q;  RPCA: W (scaled dual)
  float* out0;            // INV: output; COMPLETE: X (when write_out); RPCA: L (when last)
  float* out1;            // RPCA: S (when last)
  float ratio;            // rho_k / rho_{k+1}
  float kappa;            // RPCA: lambda / rho_k
  int first;              // COMPLETE: no Zhat / V yet;  RPCA: W == 0
  int last;               // RPCA: final pass (write L, S; no Vhat, no W update)
  int write_out;          // COMPLETE: also write X
  int tube_sparse;        // RPCA: 1 = tube-wise group shrink (eq. sparse2), 0 = entrywise
};

cudaError_t launch_tube_pass(const TubeArgs& a, cudaStream_t st);
// Whether the tube pass handles tubes of nf*nh entries (shared-memory limit).
bool tube_pass_supported(const TubeGeom& g);

// Encode observed entries: Yn[e] = omega[e] ? M[e] : NaN; counts non-finite observed
// entries into *bad.
cudaError_t launch_encode_observed(const float* M, const uint8_t* omega, float* Yn,
                                   int64_t N, int* bad, cudaStream_t st);
// Counts non-finite entries of x into *bad.
cudaError_t launch_count_nonfinite(const float* x, int64_t N, int* bad, cudaStream_t st);
// out = (a x + b y + c z + d w) * scale elementwise (nullptr inputs count as zero; out may
// alias an input).
cudaError_t launch_combine4(float* out, const float* x, float a, const float* y, float b,
                           const float* z, float c, const float* w, float d, float scale,
                           int64_t N, cudaStream_t st);
// X = omega ? M : 0, Z = 0 (the zero-iteration completion result).
cudaError_t launch_project_observed(const float* M, const uint8_t* omega, float* X, int64_t N,
                                    cudaStream_t st);

// Per-slice results of the Jacobi t-SVT kernel.
struct SliceStat {
  int rank;       // singular values above tau
  int sweeps;     // Jacobi sweeps used
  int converged;  // 1 if the last sweep made no rotation
  int pad;
  double nuc;     // sum of singular values
};

// Accumulators over many launches (ADMM loops).
struct SweepAccum {
  unsigned long long total_sweeps;
  unsigned long long nonconverged;
  int max_sweeps;
  int pad;
};

// Tunable launch choices of the slice SVT (0 = let the planner choose).
struct SliceKnobs {
  int ctas;    // CTAs per slice (1, 2, 4 or 8)
  int lanes;   // lanes per vector pair (4, 8 or 16)
  int ppg;     // vector pairs each lane group keeps in flight (1 or 2)
  int vform;   // 1: accumulate V and rebuild as W diag(d) V^H
  int block;   // 1: block form (each block round on the Gram of the CTA's vectors)
};

struct SliceArgs {
  const float2* ahat;     // input spectrum, nstore slices of n1 x n2
  float2* zhat;           // output spectrum
  const int* slices;      // list of slice indices to process (length nslices)
  int nslices;
  int n1, n2;
  int64_t N12;
  float tau;
  float tol;
  int max_sweeps;
  SliceStat* stat;        // indexed by slice index (nullable)
  SweepAccum* acc;        // nullable
  void* scratch;          // global scratch of jacobi_svt_scratch_bytes() (block exchange and
                          // partial rebuilds of multi-CTA slices); nullable = one CTA per slice
  size_t scratch_bytes;
  SliceKnobs knobs;
  // Optional outputs of the converged vectors W = B V = U diag(sigma) (vectors = columns,
  // n1 >= n2) or W = B^T V (vectors = rows): entry e < len = max(n1, n2) of vector v of slice s
  // (the index the slice list gives) is written, conjugated when wout_conj, to
  // wout[s * wout_stride + e + len * v], and sigma_v to sigout[s * sig_stride + v].
  float2* wout = nullptr;
  int64_t wout_stride = 0;
  int wout_conj = 0;
  float* sigout = nullptr;
  int64_t sig_stride = 0;
  // V form only (nullable): the accumulated rotations start from vin instead of the identity
  // and end in vout (may equal vin); slice s at v*[s * vstride], nv x nv complex, column-major
  // (column g belongs to vector g).  With vin = V0 the input slice must be B V0 (columns
  // orientation) or V0^T B (rows orientation): the SVT is then D_tau(B) exactly.
  const float2* vin = nullptr;
  float2* vout = nullptr;
  int64_t vstride = 0;
  // Nullable: the original slices B (same layout as ahat).  When set, the rebuild is the
  // U form over these slices even while V is accumulated, so a pre-rotated input (vin) or a
  // V that is only unitary to rounding does not enter D_tau(B): the kept u_i span range(W)
  // and u_i^H B is taken from B itself.
  const float2* brb = nullptr;
  // V form with vin: the kernel forms the pre-rotated vectors B V (columns) or V^T B (rows)
  // from ahat = B and vin itself while loading them (no separate pre-rotated input)
  int prerot = 0;
  // 1: the SVT stopping test -- a pair also counts as orthogonal once
  // |x^H y|^2 <= tol^2 (||B||_F^2 / nv^2) min(||x||^2, ||y||^2); 0: the relative test alone
  int abs_stop = 0;
};

// Returns cudaErrorInvalidValue when a slice does not fit the kernel's shared memory.
cudaError_t launch_jacobi_svt(const SliceArgs& a, cudaStream_t st);

// ---- persistent batched launch (plain form): one kernel launch per ADMM iteration runs the
// slice SVTs of every tensor of a batch, then the tube passes that follow them, from device
// work queues (slice_svt.cu).
// One tensor of the batch, as the host describes it.
struct BatchTensor {
  TubeGeom g;
  int kind;                 // TSVD_PROBLEM_COMPLETE (1) or TSVD_PROBLEM_RPCA (2)
  int n1, n2;
  int nslices;              // distinct stored slices (the `slices` list)
  int warm;                 // plain V-form warm start
  double scale;             // threshold scale: tau = scale / rho
  float lambda;             // RPCA
  int tube_sparse;          // RPCA: eq. sparse2 shrink
  float2* spec_a;           // V-hat (slice SVT input) and B of the U-form rebuild
  float2* spec_b;           // Z-hat (slice SVT output)
  float* state;             // completion V = X + Q; RPCA W
  const float* in;          // completion Yn (NaN = unobserved); RPCA M
  const float2* twid_h;
  const float2* twid_f;
  const int* slices;
  SliceStat* stat;
  SweepAccum* acc;
  float2* vwarm;            // warm: nstore x nv x nv accumulated right rotations
  float* out0;              // completion X; RPCA L
  float* out1;              // completion Z (nullable: not written); RPCA S
};

// Schedule of a persistent batched launch (filled by batch_plan).
struct BatchPlan {
  int C = 1;                // CTAs of a thread-block cluster (1, 2, 4 or 8)
  int small_nv = 0;         // tensors with min(n1, n2) below this run their slices as
                            // single-CTA items (if they fit one CTA), the others as cluster items
  int cmax = 0;             // kernel instance: largest chunks per lane of any tensor's plan
  int threads = 0;
  size_t smem = 0;          // dynamic shared memory per CTA
  int grid = 0;             // CTAs (a multiple of C)
  int nbig = 0, nsmall = 0, ntiles = 0, ntensors = 0;
  size_t xbuf_floats = 0;   // exchange buffer per cluster
  size_t table_bytes = 0;   // device table: descriptors, item lists, tile prefix
  size_t scratch_bytes = 0; // exchange buffers of all clusters
  // byte offsets of the table's sections
  size_t off_desc = 0, off_big = 0, off_small = 0, off_tstart = 0, off_ttensor = 0;
};

// Per-launch arguments of the persistent batched kernel.
struct BatchIter {
  int k;                    // ADMM iteration (the init launch: -1)
  int iters;
  double r, r_next;         // rho_k and rho_{k+1}
  float tol;
  int max_sweeps;
  int* ctr;                 // 3 work-queue counters of this launch, zero before it
  unsigned* done;           // per tensor: slice SVTs finished (monotonic over the solve)
  int* err;                 // set to 1 when a bounded wait gave up
  int slices_only = 0;      // skip the tube passes (plan timing)
  int abs_stop = 1;         // SliceArgs::abs_stop of the slice SVTs
};

// Iterations between cold starts of the warm-started plain Jacobi (V reset to I).
constexpr int kWarmColdEvery = 64;

// Plans the persistent launch for the tensors (C = 0: choose; small_nv < 0: choose) and
// writes the device table (to be copied to the device verbatim) into `table`.
bool batch_plan(const BatchTensor* ts, int n, int C, int small_nv, BatchPlan& plan,
                std::vector<unsigned char>& table);
// One launch: iteration it.k's slice SVTs of every tensor (it.k >= 0) and the tube passes
// that follow them (the init launch, it.k = -1: the first tube passes only).
cudaError_t launch_batch_iteration(const BatchPlan& plan, const void* table_dev, void* scratch,
                                   const BatchIter& it, cudaStream_t st);
// The persistent kernel's bounded wait on `counter` (>= 1) with the given limit; *err = 1 when
// it gave up.
cudaError_t launch_wait_selftest(const unsigned* counter, unsigned long long limit_ns, int* err,
                                 cudaStream_t st);

// Fourier-domain factors of the truncated t-SVD from the converged Jacobi of every distinct
// slice (factor.cu): W (len x nv per stored slice, as SliceArgs::wout writes it), sigma (nv per
// slice) and the accumulated rotations J (nv x nv, as SliceArgs::vout writes it from V = I).
struct FactorArgs {
  const float2* W;
  const float* sig;
  const float2* J;
  const int* slices;    // distinct stored slices
  int nslices;
  int n1, n2, k;        // k <= min(n1, n2) factors kept
  float2* Uh;           // n1 x k per stored slice
  float2* Sh;           // k x k per stored slice (f-diagonal)
  float2* Vh;           // n2 x k per stored slice
};
cudaError_t launch_factor_assemble(const FactorArgs& a, cudaStream_t st);
// Z-hat of every distinct slice from its kept[s] (per stored slice) largest singular terms
// (uses W, sig, J, slices, nslices, n1, n2 of `a`); Zh laid out like the stored spectrum.
cudaError_t launch_compress_rebuild(const FactorArgs& a, const int* kept, float2* Zh,
                                    cudaStream_t st);
// Whether launch_jacobi_svt supports an n1 x n2 slice (with scratch available).
bool jacobi_svt_supported(int n1, int n2);
// Whether the knobs give a valid plan for `nslices` n1 x n2 slices.
bool jacobi_svt_plan_ok(int n1, int n2, int nslices, const SliceKnobs& k);
// Global scratch the launch of `nslices` n1 x n2 slices needs (0 for one CTA per slice).
size_t jacobi_svt_scratch_bytes(int n1, int n2, int nslices, const SliceKnobs& k);
// CTAs per slice the launch would use.
int jacobi_svt_ctas_per_slice(int n1, int n2, int nslices, const SliceKnobs& k);

// ---- batched complex GEMM with generic strides (rsvt.cu, tc_gemm.cu)
// One operand or the result: entry (i0, i1) of batch entry b at
// p[(idx ? idx[b] : b) * bs + i0 * s0 + i1 * s1], conjugated when conj.
struct CMat {
  const float2* p;
  const int* idx;
  int64_t bs;
  int64_t s0, s1;
  int conj;
};
// C(i, j) = sum_l A(i, l) B(l, j) for i < M, j < N, l < K, for every batch entry.  With kdev
// set, the dimensions flagged dyn* are read from *kdev on the device (at most the value given,
// which sizes the grid).
struct CGemm {
  int M, N, K, batch;
  CMat a, b, c;
  const int* kdev = nullptr;
  int dynM = 0, dynN = 0, dynK = 0;
};
// Arithmetic of the slice products: FP32 on CUDA cores, or 3M complex products on the tensor
// cores with TF32, BF16 or split (3xTF32) operands and FP32 accumulation.
enum RsvtEngine : int { RSVT_GEMM_FP32 = 0, RSVT_GEMM_TF32 = 1, RSVT_GEMM_BF16 = 2,
                        RSVT_GEMM_3XTF32 = 3 };
cudaError_t launch_cgemm(const CGemm& g, int engine, cudaStream_t st);
cudaError_t launch_cgemm_tc(const CGemm& g, int engine, cudaStream_t st);
// Number of tensor-core product launches whose bounded waits expired since the last call
// (reset to 0); waits for `st`.
cudaError_t tc_gemm_take_timeouts(int* count, cudaStream_t st);

// ---- randomized, rank-adaptive slice SVT (rsvt.cu)
struct RsvtStat {
  int rank_max;    // max over slices of the singular values above max(tau, floor sigma_max)
  int saturated;   // slices whose whole sketch lay above that level
  int drops;       // columns dropped by the Cholesky factorisations
  int k;           // device-chosen sketch width (RsvtArgs::kdev mode)
  double ksum[3];  // kdev mode: sums of k, k^2, k^3 over the iterations run (work accounting)
};

struct RsvtArgs {
  const float2* ahat;     // input spectrum (slices at slices[s] * N12)
  float2* zhat;           // output spectrum
  const int* slices;      // stored slice indices to process
  int nslices;
  int mw, nw;             // working matrix Aw: mw x nw (nw <= mw)
  int64_t wr, wc;         // Aw(i, j) at i * wr + j * wc inside a slice
  int64_t N12;
  int k, kmax;            // sketch width of this call; allocated width
  int kfill;              // columns of P to refill after the call (<= kmax)
  int power;              // extra power steps (0 in warm-started ADMM loops)
  float tau;
  float floor_rel;        // noise floor of the products, relative to sigma_max
  float chol_tol;         // dropped-pivot tolerance of CholeskyQR
  float tol;              // Jacobi rotation tolerance
  int max_sweeps;
  unsigned long long seed;
  int iter;               // counter of the random refills
  int engine;             // RsvtEngine
  SliceStat* stat;        // per stored slice (nullable)
  SweepAccum* acc;        // nullable
  RsvtStat* rstat;        // nullable
  // per stored slice: P nw x kmax, Y and Q mw x kmax, Bt and Dt nw x kmax, G and T kmax x kmax,
  // sig kmax; isreal: 1 for slices whose matrix is real (self-conjugate)
  float2 *P, *Y, *Q, *Bt, *Dt, *G, *T;
  float* sig;
  const unsigned char* isreal;
  void* jscratch;
  size_t jscratch_bytes;
  SliceKnobs jknobs;      // plan of the small Jacobi SVTs (0 = planner's choice)
  // Device-chosen width: when set (= &rstat->k), the kernels read the width from it, k above
  // is its upper bound (grids, shared memory, strides), the small SVD always takes the Gram
  // path (k <= rsvt_eig_max_k()), and the call ends with rsvt_next_k_kernel picking the next
  // width from the ranks it saw: no host decision, so the sequence can be captured.
  const int* kdev = nullptr;
  int oversample = 10;
  // nullable: 7 events recorded at the stage boundaries of a call without power steps:
  // [0] sketch product [1] CholeskyQR2 [2] projection product [3] small SVT [4] rebuild
  // product [5] refill [6]
  cudaEvent_t* stage_ev = nullptr;
  // 1: the k x k CholeskyQR2 factorisations and (for k <= 80) the Rayleigh-Ritz eigen-solve
  // in FP64 instead of FP32 with double-single pivots
  int small_fp64 = 0;
  // 1: the small SVTs use the SVT stopping test (SliceArgs::abs_stop)
  int abs_stop = 0;
};

int rsvt_max_k();
// Widest sketch whose small SVD runs as the two-sided Jacobi of its Gram (wider: one-sided).
int rsvt_eig_max_k();
size_t rsvt_jacobi_scratch_bytes(int nw, int kmax, int nslices, const SliceKnobs& kn);
cudaError_t launch_rsvt(const RsvtArgs& a, cudaStream_t st);
// Refill columns c < kfill of P that carry no direction (all of them when k = 0).
cudaError_t launch_rsvt_refill(const RsvtArgs& a, int k, int kfill, cudaStream_t st);
// Device-chosen width mode: counters zero, width k0.
cudaError_t launch_rsvt_state_init(RsvtStat* st_dev, int k0, cudaStream_t st);

}  // namespace tsvd
