// tsvd_internal.h -- declarations shared by the CUDA translation units of libtsvd.
// Not part of the public C ABI (that is include/tsvd.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tsvd {

// Geometry of the tube passes.  A real tensor of order 3 or 4 is stored MATLAB column-major;
// the "tube" of pixel t = i + n1*j is the set of entries t + N12*(jf + nf*jh).  The last
// transformed mode (length nh) is transformed real-to-complex and only its first
// hh = nh/2+1 frequencies are kept; the other transformed mode (4-way case, length nf) is a
// full complex DFT.  A 3-way tensor has nf = 1, nh = n3.
// Fourier slice (kf, kh) is stored at slice index kf + nf*kh, as an n1 x n2 complex matrix
// (float2, column-major), i.e. spectrum entry (t, kf, kh) at t + N12*(kf + nf*kh).
struct TubeGeom {
  int64_t N12;   // number of tubes (n1*n2)
  int nf;        // full-DFT mode length (1 for 3-way)
  int nh;        // half-spectrum mode length
  int hh;        // nh/2 + 1
  int nstore;    // nf*hh stored Fourier slices
};

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
};

// Returns cudaErrorInvalidValue when a slice does not fit the kernel's shared memory.
cudaError_t launch_jacobi_svt(const SliceArgs& a, cudaStream_t st);
// Whether launch_jacobi_svt supports an n1 x n2 slice (with scratch available).
bool jacobi_svt_supported(int n1, int n2);
// Whether the knobs give a valid plan for `nslices` n1 x n2 slices.
bool jacobi_svt_plan_ok(int n1, int n2, int nslices, const SliceKnobs& k);
// Global scratch the launch of `nslices` n1 x n2 slices needs (0 for one CTA per slice).
size_t jacobi_svt_scratch_bytes(int n1, int n2, int nslices, const SliceKnobs& k);
// CTAs per slice the launch would use.
int jacobi_svt_ctas_per_slice(int n1, int n2, int nslices, const SliceKnobs& k);

}  // namespace tsvd
