// factor.cu -- Fourier-domain factors of the truncated t-SVD (Algorithm 1, Theorem 2.3.1).
//
// After the one-sided Jacobi of every distinct Fourier slice B (vectors = columns when
// n1 >= n2, else rows), with the accumulated rotations J (nv x nv) and the converged vectors
// W = B J (columns) or W = B^T J (rows), len x nv, and sigma_g = ||w_g||:
//   columns:  B = (W diag(1/sigma)) diag(sigma) J^H      U-hat = W / sigma,  V-hat = J;
//   rows:     B^T = W J^H, so B = conj(J) diag(sigma) (conj(W) / sigma)^H
//             U-hat = conj(J),  V-hat = conj(W) / sigma.
// The t-SVD orders each slice's singular values decreasingly (Algorithm 1 takes the SVD of
// each slice; Theorem 2.3.1 keeps the first k), so the kernel ranks them (ties by index) and
// writes the first k columns of U-hat (n1 x k), V-hat (n2 x k) and the f-diagonal S-hat
// (k x k), column-major, at slice s of buffers laid out like the tensor's stored spectrum.
// A vector whose singular value is 0 has no defined left (columns) or right (rows) partner:
// that column is written as zeros.
//
// The compression of Sec. 3 (Methods 1 and 2) keeps, per slice, a number of the largest terms
// sigma_g u_g v_g^H chosen on the host and rebuilds the slice from W and J directly (W
// already carries sigma).
#include "tsvd_internal.h"

namespace tsvd {
namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) factor_assemble_kernel(FactorArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int s = a.slices[blockIdx.x];
  const int nv = a.n1 < a.n2 ? a.n1 : a.n2;
  const int len = a.n1 < a.n2 ? a.n2 : a.n1;
  const bool rows = a.n1 < a.n2;
  float* sg = reinterpret_cast<float*>(smem_raw);
  int* perm = reinterpret_cast<int*>(sg + nv);
  const float* sig = a.sig + (size_t)s * nv;
  for (int g = threadIdx.x; g < nv; g += blockDim.x) sg[g] = sig[g];
  __syncthreads();
  // rank of g among the singular values, decreasing, ties broken by index
  for (int g = threadIdx.x; g < nv; g += blockDim.x) {
    const float v = sg[g];
    int r = 0;
    for (int h = 0; h < nv; ++h) r += (sg[h] > v || (sg[h] == v && h < g)) ? 1 : 0;
    if (r < a.k) perm[r] = g;
  }
  __syncthreads();
  const float2* W = a.W + (size_t)s * len * nv;
  const float2* J = a.J + (size_t)s * nv * nv;
  float2* Uh = a.Uh + (size_t)s * a.n1 * a.k;
  float2* Vh = a.Vh + (size_t)s * a.n2 * a.k;
  float2* Sh = a.Sh + (size_t)s * a.k * a.k;
  // U-hat: n1 x k
  for (int idx = threadIdx.x; idx < a.n1 * a.k; idx += blockDim.x) {
    const int i = idx % a.n1, r = idx / a.n1;
    const int g = perm[r];
    float2 u;
    if (rows) {
      const float2 j = J[i + (size_t)nv * g];
      u = make_float2(j.x, -j.y);
    } else {
      const float sv = sg[g];
      const float2 w = W[i + (size_t)len * g];
      u = sv > 0.f ? make_float2(w.x / sv, w.y / sv) : make_float2(0.f, 0.f);
    }
    Uh[idx] = u;
  }
  // V-hat: n2 x k
  for (int idx = threadIdx.x; idx < a.n2 * a.k; idx += blockDim.x) {
    const int i = idx % a.n2, r = idx / a.n2;
    const int g = perm[r];
    float2 v;
    if (rows) {
      const float sv = sg[g];
      const float2 w = W[i + (size_t)len * g];
      v = sv > 0.f ? make_float2(w.x / sv, -w.y / sv) : make_float2(0.f, 0.f);
    } else {
      v = J[i + (size_t)nv * g];
    }
    Vh[idx] = v;
  }
  // S-hat: k x k, sigma on the diagonal
  for (int idx = threadIdx.x; idx < a.k * a.k; idx += blockDim.x) {
    const int i = idx % a.k, r = idx / a.k;
    Sh[idx] = make_float2(i == r ? sg[perm[r]] : 0.f, 0.f);
  }
}

// Compression rebuild: Z-hat = sum of the kept[s] largest terms sigma_g u_g v_g^H of the slice,
// from W = U diag(sigma) and J: columns  Z(i, j) = sum_g W(i, g) conj(J(j, g));
//                                rows     Z(i, j) = sum_g conj(J(i, g)) W(j, g).
__global__ void __launch_bounds__(kThreads) compress_rebuild_kernel(FactorArgs a,
                                                                    const int* kept,
                                                                    float2* Zh) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int s = a.slices[blockIdx.x];
  const int nv = a.n1 < a.n2 ? a.n1 : a.n2;
  const int len = a.n1 < a.n2 ? a.n2 : a.n1;
  const bool rows = a.n1 < a.n2;
  float* sg = reinterpret_cast<float*>(smem_raw);
  int* perm = reinterpret_cast<int*>(sg + nv);
  const float* sig = a.sig + (size_t)s * nv;
  const int kk = min(max(kept[s], 0), nv);
  for (int g = threadIdx.x; g < nv; g += blockDim.x) sg[g] = sig[g];
  __syncthreads();
  for (int g = threadIdx.x; g < nv; g += blockDim.x) {
    const float v = sg[g];
    int r = 0;
    for (int h = 0; h < nv; ++h) r += (sg[h] > v || (sg[h] == v && h < g)) ? 1 : 0;
    perm[r] = g;
  }
  __syncthreads();
  const float2* W = a.W + (size_t)s * len * nv;
  const float2* J = a.J + (size_t)s * nv * nv;
  float2* Z = Zh + (size_t)s * a.n1 * a.n2;
  for (int idx = threadIdx.x; idx < a.n1 * a.n2; idx += blockDim.x) {
    const int i = idx % a.n1, j = idx / a.n1;
    float zr = 0.f, zi = 0.f;
    for (int r = 0; r < kk; ++r) {
      const int g = perm[r];
      float2 x, y;   // Z(i, j) += x * y
      if (rows) {
        const float2 jv = J[i + (size_t)nv * g];
        x = make_float2(jv.x, -jv.y);
        y = W[j + (size_t)len * g];
      } else {
        x = W[i + (size_t)len * g];
        const float2 jv = J[j + (size_t)nv * g];
        y = make_float2(jv.x, -jv.y);
      }
      zr += x.x * y.x - x.y * y.y;
      zi += x.x * y.y + x.y * y.x;
    }
    Z[idx] = make_float2(zr, zi);
  }
}

}  // namespace

cudaError_t launch_compress_rebuild(const FactorArgs& a, const int* kept, float2* Zh,
                                    cudaStream_t st) {
  if (a.nslices <= 0) return cudaSuccess;
  const int nv = a.n1 < a.n2 ? a.n1 : a.n2;
  const size_t smem = (size_t)nv * (sizeof(float) + sizeof(int));
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(compress_rebuild_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  compress_rebuild_kernel<<<a.nslices, kThreads, smem, st>>>(a, kept, Zh);
  return cudaGetLastError();
}

cudaError_t launch_factor_assemble(const FactorArgs& a, cudaStream_t st) {
  if (a.nslices <= 0) return cudaSuccess;
  const int nv = a.n1 < a.n2 ? a.n1 : a.n2;
  if (a.k < 1 || a.k > nv) return cudaErrorInvalidValue;
  const size_t smem = (size_t)nv * (sizeof(float) + sizeof(int));
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(factor_assemble_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  factor_assemble_kernel<<<a.nslices, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace tsvd
