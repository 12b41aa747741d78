// slice_svt.cu -- singular value thresholding of every Fourier slice (the Z-step of the
// completion ADMM, eq. shrink split into the per-slice problems of eq. shrink2, and the
// L-step of tensor RPCA, eq. low_rank), solved by the Lemma of Sec. 4.1:
//     D_tau(A) = U diag((sigma_i - tau)_+) V^H.
//
// One CTA owns one complex n1 x n2 slice, held entirely in shared memory.  The SVD is a
// one-sided (Hestenes) Jacobi iteration on the nv = min(n1, n2) "vectors" of the slice
// (its columns when n1 >= n2, otherwise its rows, i.e. the columns of A^T, since
// D_tau(A^T) = D_tau(A)^T).  A sweep visits every vector pair once in the round-robin
// (circle) order: each of the P-1 rounds holds P/2 disjoint pairs (P = nv rounded up to
// even), which the warps process concurrently; one warp rotates one pair, with the three
// inner products reduced by warp shuffles.  The plane rotation of a pair diagonalises its
// 2x2 Gram matrix [[a, c], [c*, b]]:
//     c = |c| e^{i phi},  zeta = (b - a) / (2|c|),  t = sign(zeta) / (|zeta| + sqrt(1+zeta^2)),
//     cs = 1/sqrt(1+t^2), sn = cs t,
//     x <- cs x - sn e^{-i phi} y,   y <- sn e^{i phi} x + cs y.
// A pair is rotated while |c| > tol sqrt(a b); sweeps stop when a whole sweep rotates
// nothing (or at max_sweeps).  The converged vectors are U diag(sigma); with
// u_i = w_i / sigma_i the thresholded slice is rebuilt without V as
//     D_tau(B) = sum_{sigma_i > tau} ((sigma_i - tau)/sigma_i) u_i (u_i^H B),
// re-reading the original slice B from global memory (it is L2 resident) in chunks.
//
// A slice whose matrix is exactly real (the self-conjugate Fourier slices) stays exactly
// real: every inner product then has a zero imaginary part and every rotation is real.
#include "tsvd_internal.h"

namespace tsvd {
namespace {

constexpr int kNC = 8;            // rebuild chunk width (vectors of B per chunk)
constexpr int kMinWarps = 4;
constexpr size_t kStaticSmemReserve = 1024;   // static __shared__ of the kernel, with margin

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Pair (p, q) of slot `slot` in round r of the circle method over P players.
__device__ __forceinline__ void round_robin_pair(int r, int slot, int P, int& p, int& q) {
  if (slot == 0) {
    p = P - 1;
    q = r;
  } else {
    p = (r + slot) % (P - 1);
    q = (r - slot + P - 1) % (P - 1);
  }
}

struct SliceShape {
  int nv;    // number of vectors
  int len;   // vector length
  int ld;    // shared-memory pitch of a vector (odd, in float2)
  int rows;  // 1: vectors are the rows of the slice
  int nc;    // rebuild chunk width
};

__host__ __device__ inline size_t slice_smem_bytes(const SliceShape& sh) {
  return (size_t)sh.nv * sh.ld * sizeof(float2) + (size_t)sh.len * sh.nc * sizeof(float2) +
         (size_t)sh.nv * sh.nc * sizeof(float2) + (size_t)sh.nv * (2 * sizeof(float) + sizeof(int));
}

__global__ void __launch_bounds__(1024) jacobi_svt_kernel(SliceArgs a, SliceShape sh) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nv = sh.nv, len = sh.len, ld = sh.ld, nc = sh.nc;
  float2* W = reinterpret_cast<float2*>(smem_raw);
  float2* Bc = W + (size_t)nv * ld;
  float2* Cc = Bc + (size_t)len * nc;
  float* sig = reinterpret_cast<float*>(Cc + (size_t)nv * nc);
  float* dsc = sig + nv;
  int* keep = reinterpret_cast<int*>(dsc + nv);
  __shared__ int s_rank;

  const int s = a.slices ? a.slices[blockIdx.x] : (int)blockIdx.x;
  const int n1 = a.n1;
  const int64_t N12 = a.N12;
  const float2* __restrict__ A = a.ahat + (size_t)s * N12;
  float2* __restrict__ Z = a.zhat + (size_t)s * N12;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nthr >> 5;

  // ---- load the slice: vector v, element p  <->  A(i, j) at i + n1*j
  for (int64_t idx = tid; idx < N12; idx += nthr) {
    const int i = (int)(idx % n1), j = (int)(idx / n1);
    const int v = sh.rows ? i : j, p = sh.rows ? j : i;
    W[(size_t)v * ld + p] = A[idx];
  }
  __syncthreads();

  // ---- one-sided Jacobi sweeps in round-robin order
  const int P = nv + (nv & 1);
  const int npairs = P / 2;
  const float tol = a.tol;
  int sweeps = 0, converged = 0;
  for (int sw = 0; sw < a.max_sweeps; ++sw) {
    int rotated = 0;
    for (int r = 0; r < P - 1; ++r) {
      for (int slot = warp; slot < npairs; slot += nwarps) {
        int p, q;
        round_robin_pair(r, slot, P, p, q);
        if (p >= nv || q >= nv) continue;
        float2* wp = W + (size_t)p * ld;
        float2* wq = W + (size_t)q * ld;
        float al = 0.f, be = 0.f, cr = 0.f, ci = 0.f;
        for (int e = lane; e < len; e += 32) {
          const float2 x = wp[e], y = wq[e];
          al += x.x * x.x + x.y * x.y;
          be += y.x * y.x + y.y * y.y;
          cr += x.x * y.x + x.y * y.y;   // Re(x^H y)
          ci += x.x * y.y - x.y * y.x;   // Im(x^H y)
        }
        al = warp_sum(al);
        be = warp_sum(be);
        cr = warp_sum(cr);
        ci = warp_sum(ci);
        const float g = hypotf(cr, ci);
        if (!(g > tol * sqrtf(al) * sqrtf(be))) continue;
        const float zeta = (be - al) / (2.f * g);
        float t;
        if (fabsf(zeta) > 1e18f)
          t = 0.5f / zeta;
        else
          t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
        if (t == 0.f) continue;
        rotated = 1;
        // correctly rounded: an approximate reciprocal square root makes every rotation
        // slightly non-unitary and the vector norms drift over thousands of rotations
        const float cs = 1.f / sqrtf(1.f + t * t), sn = cs * t;
        const float er = cr / g, ei = ci / g;       // e^{i phi}
        const float kr = sn * er, ki = sn * ei;     // sn e^{i phi}
        for (int e = lane; e < len; e += 32) {
          const float2 x = wp[e], y = wq[e];
          // x' = cs x - conj(k) y,   y' = k x + cs y
          wp[e] = make_float2(cs * x.x - (kr * y.x + ki * y.y), cs * x.y - (kr * y.y - ki * y.x));
          wq[e] = make_float2(kr * x.x - ki * x.y + cs * y.x, kr * x.y + ki * x.x + cs * y.y);
        }
      }
      __syncthreads();
    }
    ++sweeps;
    if (!__syncthreads_or(rotated)) {
      converged = 1;
      break;
    }
  }

  // ---- singular values: sigma_v = ||w_v||
  for (int v = warp; v < nv; v += nwarps) {
    const float2* wv = W + (size_t)v * ld;
    float acc = 0.f;
    for (int e = lane; e < len; e += 32) acc += wv[e].x * wv[e].x + wv[e].y * wv[e].y;
    acc = warp_sum(acc);
    if (lane == 0) sig[v] = sqrtf(acc);
  }
  __syncthreads();
  const float tau = a.tau;
  if (tid == 0) {
    int r = 0;
    double nuc = 0.0;
    for (int v = 0; v < nv; ++v) {
      nuc += (double)sig[v];
      if (sig[v] > tau) {
        keep[r++] = v;
        dsc[v] = (sig[v] - tau) / sig[v];
      }
    }
    s_rank = r;
    if (a.stat) {
      SliceStat st;
      st.rank = r;
      st.sweeps = sweeps;
      st.converged = converged;
      st.pad = 0;
      st.nuc = nuc;
      a.stat[s] = st;
    }
    if (a.acc) {
      atomicAdd(&a.acc->total_sweeps, (unsigned long long)sweeps);
      if (!converged) atomicAdd(&a.acc->nonconverged, 1ull);
      atomicMax(&a.acc->max_sweeps, sweeps);
    }
  }
  __syncthreads();
  const int rank = s_rank;

  if (rank == 0) {
    for (int64_t idx = tid; idx < N12; idx += nthr) Z[idx] = make_float2(0.f, 0.f);
    return;
  }

  // ---- normalise the kept vectors: u = w / sigma
  for (int64_t idx = tid; idx < (int64_t)rank * len; idx += nthr) {
    const int k = (int)(idx / len), e = (int)(idx % len);
    const int v = keep[k];
    const float inv = 1.f / sig[v];
    float2 w = W[(size_t)v * ld + e];
    W[(size_t)v * ld + e] = make_float2(w.x * inv, w.y * inv);
  }
  __syncthreads();

  // ---- rebuild Z = U_r diag(d) U_r^H B, chunk of nc vectors of B at a time
  for (int c0 = 0; c0 < nv; c0 += nc) {
    const int ncur = min(nc, nv - c0);
    // B chunk: Bc[p + len*cc] = B(p, c0+cc)
    for (int idx = tid; idx < len * ncur; idx += nthr) {
      int p, cc;
      size_t gi;
      if (!sh.rows) {
        p = idx % len;
        cc = idx / len;
        gi = (size_t)p + (size_t)n1 * (c0 + cc);
      } else {
        cc = idx % ncur;
        p = idx / ncur;
        gi = (size_t)(c0 + cc) + (size_t)n1 * p;
      }
      Bc[p + (size_t)len * cc] = A[gi];
    }
    __syncthreads();
    // C(k, cc) = d_k * u_k^H B(:, c0+cc)
    for (int k = tid; k < rank; k += nthr) {
      const int v = keep[k];
      const float2* u = W + (size_t)v * ld;
      float accr[kNC], acci[kNC];
#pragma unroll
      for (int cc = 0; cc < kNC; ++cc) accr[cc] = acci[cc] = 0.f;
      for (int p = 0; p < len; ++p) {
        const float2 x = u[p];
#pragma unroll
        for (int cc = 0; cc < kNC; ++cc) {
          if (cc < ncur) {
            const float2 b = Bc[p + (size_t)len * cc];
            accr[cc] += x.x * b.x + x.y * b.y;
            acci[cc] += x.x * b.y - x.y * b.x;
          }
        }
      }
      const float d = dsc[v];
#pragma unroll
      for (int cc = 0; cc < kNC; ++cc)
        if (cc < ncur) Cc[(size_t)k * nc + cc] = make_float2(d * accr[cc], d * acci[cc]);
    }
    __syncthreads();
    // Z(p, cc) = sum_k u_k(p) C(k, cc), written over the B chunk
    for (int p = tid; p < len; p += nthr) {
      float accr[kNC], acci[kNC];
#pragma unroll
      for (int cc = 0; cc < kNC; ++cc) accr[cc] = acci[cc] = 0.f;
      for (int k = 0; k < rank; ++k) {
        const float2 x = W[(size_t)keep[k] * ld + p];
#pragma unroll
        for (int cc = 0; cc < kNC; ++cc) {
          if (cc < ncur) {
            const float2 c = Cc[(size_t)k * nc + cc];
            accr[cc] += x.x * c.x - x.y * c.y;
            acci[cc] += x.x * c.y + x.y * c.x;
          }
        }
      }
#pragma unroll
      for (int cc = 0; cc < kNC; ++cc)
        if (cc < ncur) Bc[p + (size_t)len * cc] = make_float2(accr[cc], acci[cc]);
    }
    __syncthreads();
    for (int idx = tid; idx < len * ncur; idx += nthr) {
      int p, cc;
      size_t gi;
      if (!sh.rows) {
        p = idx % len;
        cc = idx / len;
        gi = (size_t)p + (size_t)n1 * (c0 + cc);
      } else {
        cc = idx % ncur;
        p = idx / ncur;
        gi = (size_t)(c0 + cc) + (size_t)n1 * p;
      }
      Z[gi] = Bc[p + (size_t)len * cc];
    }
    __syncthreads();
  }
}

bool plan_slice(int n1, int n2, SliceShape& sh, size_t& smem) {
  static int max_optin = -1;
  if (max_optin < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
        cudaSuccess)
      max_optin = 227 * 1024;
  }
  sh.rows = n1 < n2 ? 1 : 0;
  sh.nv = n1 < n2 ? n1 : n2;
  sh.len = n1 < n2 ? n2 : n1;
  sh.ld = sh.len | 1;
  for (int nc = kNC; nc >= 1; nc >>= 1) {
    sh.nc = nc;
    smem = slice_smem_bytes(sh);
    if (smem + kStaticSmemReserve <= (size_t)max_optin) return true;
  }
  return false;
}

}  // namespace

bool jacobi_svt_supported(int n1, int n2) {
  SliceShape sh;
  size_t smem;
  return n1 >= 1 && n2 >= 1 && plan_slice(n1, n2, sh, smem);
}

cudaError_t launch_jacobi_svt(const SliceArgs& a, cudaStream_t st) {
  if (a.nslices <= 0) return cudaSuccess;
  SliceShape sh;
  size_t smem;
  if (!plan_slice(a.n1, a.n2, sh, smem)) return cudaErrorInvalidValue;
  const int P = sh.nv + (sh.nv & 1);
  const int npairs = P / 2;
  const int passes = (npairs + 31) / 32;
  int nwarps = (npairs + passes - 1) / passes;
  if (nwarps < kMinWarps) nwarps = kMinWarps;
  if (nwarps > 32) nwarps = 32;
  cudaError_t e = cudaFuncSetAttribute(jacobi_svt_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  jacobi_svt_kernel<<<a.nslices, nwarps * 32, smem, st>>>(a, sh);
  return cudaGetLastError();
}

}  // namespace tsvd
