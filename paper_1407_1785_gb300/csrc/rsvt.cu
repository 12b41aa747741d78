// rsvt.cu -- randomized, rank-adaptive singular value thresholding of the Fourier slices:
// the mixed-precision form of the per-slice step D_tau of the Lemma in Sec. 4.1 (used by the
// completion Z-step, eq. shrink / shrink2, and the RPCA L-step, eq. low_rank).
//
// Per slice, the working matrix Aw (mw x nw complex) is the slice or its transpose, whichever
// has fewer columns (D_tau(A^T) = D_tau(A)^T).  With a sketch width k and a right basis
// P (nw x k) carried from the previous call:
//   Y  = Aw P                              sketch                              (GEMM)
//   Q  = orth(Y)                           CholeskyQR2 (cholqr_factor_kernel)
//   Bt = Aw^T conj(Q)  = (Q^H Aw)^T        projection onto range(Q), nw x k    (GEMM)
//   Dt = D_tau(Bt)                         SVT of the small matrix: two-sided Jacobi on its
//                                          k x k Gram (k <= 112), else one-sided Jacobi
//   Zw = Q Dt^T        = Q D_tau(Q^H Aw)   rebuild                             (GEMM)
//   P' = conj(Bt J), J the accumulated Jacobi rotations: the right singular vectors of Q^H Aw
//        scaled by sigma: the next call starts from the Ritz basis (one step of subspace
//        iteration per call), so Y' = Aw P' has nearly orthogonal columns and the small
//        Jacobi converges in a few sweeps.
// Because Q has orthonormal columns, Q D_tau(Q^H Aw) = D_tau(Q Q^H Aw): the result is the exact
// thresholding of the projection of Aw onto the sketched subspace, and it equals D_tau(Aw)
// when that subspace holds every singular direction above tau.
//
// Rank adaptivity.  After each call the kernel rsvt_refill_kernel counts, per slice, the
// singular values above max(tau, floor * sigma_max) (floor is the product precision's noise
// level) and records the maximum over slices; the caller picks the next k as that count plus
// an oversampling margin.  Columns of P that carry no direction (dropped by the Cholesky
// factorisation, or beyond the previous k) are refilled with counter-based random vectors.
//
// Orthonormalisation (CholeskyQR2).  G = Y^H Y (FP32), scaled to unit diagonal,
// Gs = D^-1 G D^-1 = R^H R, Q = Y D^-1 R^-1, done twice.  The column scaling makes the FP32
// rounding of G relative to each column's norm, so graded sketches (columns of norm sigma^2)
// factor accurately.  The Schur complement is updated in FP32 and the pivots in double-single
// arithmetic (FP32 pairs).  A pivot
// below chol_tol marks a column that depends on the previous ones: it is dropped (its column of
// Q is zero) instead of failing the factorisation.
//
// Products.  The three slice products (sketch, projection, rebuild) run on the engine the
// caller selects: FP32 CUDA cores here, or the tensor-core engines of tc_gemm.cu.  The Gram
// matrices and the k x k triangular applications of CholeskyQR2 need FP32-level accuracy:
// they run as split-TF32 tensor-core products when the caller's engine uses tensor cores,
// else in FP32 on CUDA cores.
#include "tsvd_internal.h"

#include <algorithm>

namespace tsvd {
namespace {

constexpr int TM = 64, TN = 64, TK = 16;

__device__ __forceinline__ float2 cload(const float2* p, int64_t o, int conj) {
  float2 v = p[o];
  if (conj) v.y = -v.y;
  return v;
}

// C = op(A) op(B), batched, generic strides (see CGemm in tsvd_internal.h).  64 x 64 tile per
// CTA, 4 x 4 complex outputs per thread; operand tiles staged through shared memory with
// threads running along whichever index is contiguous in global memory.
__global__ void __launch_bounds__(256) cgemm_fp32_kernel(CGemm g) {
  __shared__ float2 As[TK][TM + 1];
  __shared__ float2 Bs[TK][TN + 1];
  if (g.kdev) {
    const int kk = *g.kdev;
    if (g.dynM) g.M = kk;
    if (g.dynN) g.N = kk;
    if (g.dynK) g.K = kk;
  }
  if ((int)blockIdx.x * TM >= g.M || (int)blockIdx.y * TN >= g.N) return;
  const int bz = blockIdx.z;
  const float2* A = g.a.p + (int64_t)(g.a.idx ? g.a.idx[bz] : bz) * g.a.bs;
  const float2* B = g.b.p + (int64_t)(g.b.idx ? g.b.idx[bz] : bz) * g.b.bs;
  float2* C = const_cast<float2*>(g.c.p) + (int64_t)(g.c.idx ? g.c.idx[bz] : bz) * g.c.bs;
  const int i0 = blockIdx.x * TM, j0 = blockIdx.y * TN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const bool a_rows = g.a.s0 == 1;
  const bool b_ctr = g.b.s0 == 1;
  float accr[4][4], acci[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) accr[r][c] = acci[r][c] = 0.f;
  for (int l0 = 0; l0 < g.K; l0 += TK) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + 256 * u;
      int ii, ll;
      if (a_rows) {
        ii = e % TM;
        ll = e / TM;
      } else {
        ll = e % TK;
        ii = e / TK;
      }
      int i = i0 + ii, l = l0 + ll;
      As[ll][ii] = (i < g.M && l < g.K) ? cload(A, i * g.a.s0 + l * g.a.s1, g.a.conj)
                                         : make_float2(0.f, 0.f);
      int jj;
      if (b_ctr) {
        ll = e % TK;
        jj = e / TK;
      } else {
        jj = e % TN;
        ll = e / TN;
      }
      const int j = j0 + jj;
      l = l0 + ll;
      Bs[ll][jj] = (j < g.N && l < g.K) ? cload(B, l * g.b.s0 + j * g.b.s1, g.b.conj)
                                         : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 4
    for (int l = 0; l < TK; ++l) {
      float2 a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[l][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[l][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          accr[r][c] = fmaf(a[r].x, b[c].x, fmaf(-a[r].y, b[c].y, accr[r][c]));
          acci[r][c] = fmaf(a[r].x, b[c].y, fmaf(a[r].y, b[c].x, acci[r][c]));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + ty + 16 * r;
    if (i >= g.M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + tx + 16 * c;
      if (j < g.N) C[i * g.c.s0 + j * g.c.s1] = make_float2(accr[r][c], acci[r][c]);
    }
  }
}

// (hi, lo) -= ax^2 + ay^2 in double-single arithmetic: the squares are split exactly with
// FMA, the sums are two-sums (the _rn intrinsics keep the compiler from contracting them).
__device__ __forceinline__ void ds_sub_norm2(float& hi, float& lo, float ax, float ay) {
  const float p = __fmul_rn(ax, ax), pe = fmaf(ax, ax, -p);
  const float q = __fmul_rn(ay, ay), qe = fmaf(ay, ay, -q);
  const float s = __fadd_rn(p, q);
  const float bq = __fsub_rn(s, p);
  const float se = __fadd_rn(__fadd_rn(__fsub_rn(p, __fsub_rn(s, bq)), __fsub_rn(q, bq)),
                             __fadd_rn(pe, qe));
  const float t = __fsub_rn(hi, s);
  const float bt = __fsub_rn(t, hi);
  const float te = __fadd_rn(__fadd_rn(__fsub_rn(hi, __fsub_rn(t, bt)), __fsub_rn(-s, bt)),
                             __fsub_rn(lo, se));
  const float nh = __fadd_rn(t, te);
  lo = __fsub_rn(te, __fsub_rn(nh, t));
  hi = nh;
}

// One CTA per slice: column-scaled Cholesky factorisation Gs = R^H R of the k x k Gram G
// (col-major, ld ldg) with dropped pivots, and T = D^-1 R^-1 (zero columns for dropped
// pivots), written over the same layout.  R^-1 is built in the same k steps as R, as the
// coefficients of Gram-Schmidt on the scaled columns: at step j column x_j of R^-1 is final
// once scaled by 1 / R_jj, and every later column subtracts R_jl x_j.  Shared memory: S
// (k x (k+1) complex) holds R in the upper triangle and (R^-1)^T in the strict lower one; the
// diagonal of R^-1, the pivots and the column scales sit in separate arrays.  The pivots are
// accumulated in double-single arithmetic (an FP32 pair updated with exact products and
// two-sums): about twice FP32's precision against the cancellation in 1 - sum |R_ij|^2,
// without FP64 instructions, which run at a small fraction of the FP32 rate on this GPU.
// Threads form a 32 x 32 grid over the trailing block.  A Gram that is already the identity
// to FP32 resolution (every scaled off-diagonal entry below 1e-6, the usual case of the second
// pass) skips the factorisation: R = I, T = D^-1.
__global__ void __launch_bounds__(1024) cholqr_factor_kernel(const float2* G, float2* T,
                                                            const int* slices, int k, int ldg,
                                                            int64_t gs, float tol,
                                                            RsvtStat* rstat, const int* kdev) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (kdev) k = *kdev;
  const int s = slices[blockIdx.x];
  const int ldS = k + 1;
  float2* S = reinterpret_cast<float2*>(smem_raw);
  float* ddh = reinterpret_cast<float*>(S + (size_t)k * ldS);   // pivots: hi + lo
  float* ddl = ddh + k;
  double* dsc = reinterpret_cast<double*>(ddl + k);
  float2* xd = reinterpret_cast<float2*>(dsc + k);
  float* isc = reinterpret_cast<float*>(xd + k);
  int* okc = reinterpret_cast<int*>(isc + k);
  __shared__ double s_dmax;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int tx = tid & 31, ty = tid >> 5;
  const float2* Gp = G + (size_t)s * gs;
  float2* Tp = T + (size_t)s * gs;

  for (int i = tid; i < k; i += nthr) {
    const double g = (double)Gp[i + (size_t)i * ldg].x;
    dsc[i] = g > 0.0 ? sqrt(g) : 0.0;
  }
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int i = 0; i < k; ++i) m = fmax(m, dsc[i]);
    s_dmax = m;
  }
  __syncthreads();
  const double dmin = 1e-30 * s_dmax;
  for (int i = tid; i < k; i += nthr) {
    const bool zero = !(dsc[i] > dmin) || s_dmax == 0.0;
    ddh[i] = zero ? 0.f : 1.f;
    ddl[i] = 0.f;
    if (zero) dsc[i] = 1.0;
    isc[i] = (float)(1.0 / dsc[i]);
    xd[i] = make_float2(1.f, 0.f);
  }
  __syncthreads();
  // scaled Gram in the upper triangle, zero (R^-1)^T in the strict lower triangle
  for (int r = ty; r < k; r += 32)
    for (int c = tx; c < k; c += 32) {
      float2 v = make_float2(0.f, 0.f);
      if (r <= c && ddh[r] != 0.f && ddh[c] != 0.f) {
        v = Gp[r + (size_t)c * ldg];
        const float inv = isc[r] * isc[c];
        v.x *= inv;
        v.y *= inv;
      }
      S[(size_t)r * ldS + c] = v;
    }
  __syncthreads();
  {
    int far = 0;
    for (int r = ty; r < k; r += 32)
      for (int c = r + 1 + tx; c < k; c += 32) {
        const float2 v = S[(size_t)r * ldS + c];
        far |= fabsf(v.x) + fabsf(v.y) > 1e-6f;
      }
    for (int r = tid; r < k; r += nthr) far |= ddh[r] == 0.f;
    if (__syncthreads_or(far) == 0) {
      // R = I: T = D^-1
      for (int c = ty; c < k; c += 32)
        for (int i = tx; i < k; i += 32)
          Tp[i + (size_t)c * ldg] = i == c ? make_float2(isc[i], 0.f) : make_float2(0.f, 0.f);
      return;
    }
  }

  __shared__ float s_rjj, s_irjj;
  __shared__ int s_ok;
  for (int j = 0; j < k; ++j) {
    // the pivot 1 - sum |R_ij|^2 cancels; it is accumulated in double-single arithmetic and
    // one thread turns it into R_jj
    if (tid == 0) {
      const float pj = ddh[j] + ddl[j];
      const bool ok = pj > tol;
      const float r = ok ? sqrtf(pj) : 1.f;
      s_ok = ok ? 1 : 0;
      s_rjj = r;
      s_irjj = ok ? 1.f / r : 0.f;
    }
    __syncthreads();
    const bool okj = s_ok != 0;
    const float rjj = s_rjj;
    const float irjj = s_irjj;
    // row j of R; x_j scaled by 1 / R_jj (zeroed when the column is dropped)
    for (int l = j + 1 + tid; l < k; l += nthr) {
      const float2 v = S[(size_t)j * ldS + l];
      S[(size_t)j * ldS + l] = make_float2(v.x * irjj, v.y * irjj);
    }
    for (int i = tid; i < j; i += nthr) {
      const float2 v = S[(size_t)j * ldS + i];
      S[(size_t)j * ldS + i] = make_float2(v.x * irjj, v.y * irjj);
    }
    if (tid == 0) {
      S[(size_t)j * ldS + j] = make_float2(rjj, 0.f);
      const float2 v = xd[j];
      xd[j] = make_float2(v.x * irjj, v.y * irjj);
      okc[j] = okj ? 1 : 0;
    }
    __syncthreads();
    if (okj) {
      // trailing Schur complement (upper triangle) and its FP64 pivots
      for (int l = j + 1 + ty; l < k; l += 32) {
        const float2 a = S[(size_t)j * ldS + l];
        for (int l2 = l + tx; l2 < k; l2 += 32) {
          const float2 b = S[(size_t)j * ldS + l2];
          float2 v = S[(size_t)l * ldS + l2];
          v.x -= a.x * b.x + a.y * b.y;
          v.y -= a.x * b.y - a.y * b.x;
          S[(size_t)l * ldS + l2] = v;
        }
        if (tx == 0) ds_sub_norm2(ddh[l], ddl[l], a.x, a.y);
        // x_l -= R_jl x_j on entries i <= j (X(i, l) kept at S(l, i), X(j, j) in xd)
        for (int i = tx; i <= j; i += 32) {
          const float2 xj = i == j ? xd[j] : S[(size_t)j * ldS + i];
          float2 v = S[(size_t)l * ldS + i];
          v.x -= a.x * xj.x - a.y * xj.y;
          v.y -= a.x * xj.y + a.y * xj.x;
          S[(size_t)l * ldS + i] = v;
        }
      }
    }
    __syncthreads();
  }
  // T(i, c) = X(i, c) / d_i, zero below the diagonal and in dropped columns
  for (int c = ty; c < k; c += 32)
    for (int i = tx; i < k; i += 32) {
      float2 v = make_float2(0.f, 0.f);
      if (okc[c] && i <= c) {
        v = i == c ? xd[c] : S[(size_t)c * ldS + i];
        v.x *= isc[i];
        v.y *= isc[i];
      }
      Tp[i + (size_t)c * ldg] = v;
    }
  if (rstat && tid == 0) {
    int nd = 0;
    for (int c = 0; c < k; ++c) nd += okc[c] ? 0 : 1;
    if (nd) atomicAdd(&rstat->drops, nd);
  }
}

// Circle-method pair (p, q) of slot `slot` in round r over P (even) players.
__device__ __forceinline__ void circle_pair(int r, int slot, int P, int& p, int& q) {
  if (slot == 0) {
    p = P - 1;
    q = r;
  } else {
    p = r + slot;
    if (p >= P - 1) p -= P - 1;
    q = r - slot + P - 1;
    if (q >= P - 1) q -= P - 1;
  }
}

// One CTA per slice: the SVD of the projected nw x k matrix Bt through its k x k Gram
// H = Bt^H Bt (col-major, ld ldh, in G), by cyclic two-sided Jacobi: H <- J^H H J over all
// pairs of a circle-method round at once, J accumulated into W.  The pair rotation is the one
// of the one-sided form (same parameters from a = H_pp, b = H_qq, c = H_pq, the same
// cos - 1 form), so this computes what one-sided Jacobi on the columns of Bt computes, with
// the inner products read from H instead of recomputed.  At convergence the eigenvalues are
// sigma^2 and Bt = (Bt W Sigma^-1) Sigma W^H.  Writes W (into T), Wf = W diag(f) with
// f = (sigma - tau)_+ / sigma (into G), sigma (sig) and the slice statistics.  Shared memory:
// H and W as k x (k + 1) complex matrices, the round's rotations.
__global__ void __launch_bounds__(1024) eig_svt_kernel(float2* G, float2* T, float* sig,
                                                       const int* slices, int k, int ldg,
                                                       int64_t gs, int64_t sig_stride,
                                                       float tau, float tol, int max_sweeps,
                                                       SliceStat* stat, SweepAccum* acc,
                                                       const int* kdev, int abs_stop) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (kdev) k = *kdev;
  const int s = slices[blockIdx.x];
  const int ldh = k + 1;
  float2* H = reinterpret_cast<float2*>(smem_raw);
  float2* W = H + (size_t)k * ldh;
  float4* rot = reinterpret_cast<float4*>(W + (size_t)k * ldh);   // (cm, kr, ki, on)
  int2* prs = reinterpret_cast<int2*>(rot + (k + 1) / 2);
  __shared__ int s_flags;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nthr >> 5;
  float2* Gp = G + (size_t)s * gs;
  float2* Tp = T + (size_t)s * gs;
  for (int c = warp; c < k; c += nwarps)
    for (int m = lane; m < k; m += 32) {
      H[m + (size_t)c * ldh] = Gp[m + (size_t)c * ldg];
      W[m + (size_t)c * ldh] = make_float2(m == c ? 1.f : 0.f, 0.f);
    }
  const int kp = k + (k & 1);
  const int npair = kp / 2;
  const float tol2 = tol * tol;
  const float big2 = tol / (2.f * (float)k);
  int sweeps = 0, converged = 0;
  __shared__ float s_floor2;
  __syncthreads();
  // the SVT stopping test of the one-sided kernel (abs_stop): a pair also stops once
  // |H_pq|^2 <= tol^2 (trace(H) / k^2) min(H_pp, H_qq); trace(H) = ||Bt||_F^2 is invariant
  // under the rotations and summed in a fixed order
  if (tid == 0) {
    float tr = 0.f;
    for (int m = 0; m < k; ++m) tr += fmaxf(H[m + (size_t)m * ldh].x, 0.f);
    s_floor2 = abs_stop ? tol2 * (tr / ((float)k * (float)k)) : 0.f;
  }
  __syncthreads();
  const float floor2 = s_floor2;
  for (int sw = 0; sw < max_sweeps && !converged; ++sw) {
    if (tid == 0) s_flags = 0;
    __syncthreads();
    for (int r = 0; r < kp - 1; ++r) {
      // rotation parameters, one thread per pair (t, 1/r and the phase with the approximate
      // reciprocal square root and division: cs - 1 = -t sn / (1 + r) keeps cs^2 + sn^2 = 1
      // up to ~1.5 t^2 times their relative error)
      if (tid < npair) {
        int p, q;
        circle_pair(r, tid, kp, p, q);
        float4 ro = make_float4(0.f, 0.f, 0.f, 0.f);
        if (p < k && q < k) {
          const float al = fmaxf(H[p + (size_t)p * ldh].x, 0.f);
          const float be = fmaxf(H[q + (size_t)q * ldh].x, 0.f);
          const float2 c = H[p + (size_t)q * ldh];   // H_pq = col_p^H col_q
          const float c2 = c.x * c.x + c.y * c.y;
          const float ab = al * be;
          if (c2 > tol2 * ab && c2 > floor2 * fminf(al, be)) {
            const float inv_g = c2 >= 1e-30f ? rsqrtf(c2) : 1.f / sqrtf(c2);
            const float zeta = (be - al) * (0.5f * inv_g);
            const float az = fabsf(zeta);
            const float z1 = fmaf(zeta, zeta, 1.f);
            const float t0 = __fdividef(1.f, az + z1 * rsqrtf(z1));
            float t = az > 1e18f ? __fdividef(0.5f, az) : t0;
            t = zeta >= 0.f ? t : -t;
            if (t != 0.f) {
              const float q1 = fmaf(t, t, 1.f);
              const float rs = rsqrtf(q1);
              const float sn = t * rs;
              const float cm = __fdividef(-(t * sn), 1.f + q1 * rs);
              ro = make_float4(cm, sn * (c.x * inv_g), sn * (c.y * inv_g), 1.f);
              atomicOr(&s_flags, c2 > big2 * ab ? 3 : 1);
            }
          }
        }
        rot[tid] = ro;
        prs[tid] = make_int2(p, q);
      }
      __syncthreads();
      // columns: [x, y] <- [x + cm x - conj(kk) y, y + cm y + kk x] on H and W; a warp per
      // pair, a lane per row; packed FP32x2: (re, im) of an entry in one register pair
      for (int i = warp; i < npair; i += nwarps) {
        const float4 ro = rot[i];
        if (ro.w == 0.f) continue;
        const int2 pq = prs[i];
        const float2 CM = make_float2(ro.x, ro.x), KR = make_float2(ro.y, ro.y),
                     NKR = make_float2(-ro.y, -ro.y), KI = make_float2(-ro.z, ro.z);
        for (int m = lane; m < k; m += 32) {
#pragma unroll
          for (int mat = 0; mat < 2; ++mat) {
            float2* X = mat == 0 ? H : W;
            float2& x = X[m + (size_t)pq.x * ldh];
            float2& y = X[m + (size_t)pq.y * ldh];
            const float2 xv = x, yv = y;
            // -conj(kk) y = (-kr yr - ki yi, -kr yi + ki yr);  kk x = (kr xr - ki xi, kr xi + ki xr)
            x = __ffma2_rn(KI, make_float2(yv.y, yv.x), __ffma2_rn(NKR, yv, __ffma2_rn(CM, xv, xv)));
            y = __ffma2_rn(KI, make_float2(xv.y, xv.x), __ffma2_rn(KR, xv, __ffma2_rn(CM, yv, yv)));
          }
        }
      }
      __syncthreads();
      // rows: row_p <- row_p + cm row_p - kk row_q, row_q <- row_q + cm row_q + conj(kk) row_p
      for (int i = warp; i < npair; i += nwarps) {
        const float4 ro = rot[i];
        if (ro.w == 0.f) continue;
        const int2 pq = prs[i];
        const float2 CM = make_float2(ro.x, ro.x), KR = make_float2(ro.y, ro.y),
                     NKR = make_float2(-ro.y, -ro.y), KI = make_float2(ro.z, -ro.z);
        for (int m = lane; m < k; m += 32) {
          float2& x = H[pq.x + (size_t)m * ldh];
          float2& y = H[pq.y + (size_t)m * ldh];
          const float2 xv = x, yv = y;
          // -kk y = (-kr yr + ki yi, -kr yi - ki yr);  conj(kk) x = (kr xr + ki xi, kr xi - ki xr)
          x = __ffma2_rn(KI, make_float2(yv.y, yv.x), __ffma2_rn(NKR, yv, __ffma2_rn(CM, xv, xv)));
          y = __ffma2_rn(KI, make_float2(xv.y, xv.x), __ffma2_rn(KR, xv, __ffma2_rn(CM, yv, yv)));
        }
      }
      __syncthreads();
    }
    const int fl = s_flags;
    ++sweeps;
    // converged: nothing rotated, or only rotations too small to leave a cosine above tol
    if (!(fl & 1) || !(fl & 2)) converged = 1;
    __syncthreads();
  }
  // sigma_v = sqrt(lambda_v); W and W diag(f) out
  __shared__ int s_rank;
  __shared__ double s_nuc;
  if (tid == 0) {
    int rank = 0;
    double nuc = 0.0;
    for (int v = 0; v < k; ++v) {
      const float sv = sqrtf(fmaxf(H[v + (size_t)v * ldh].x, 0.f));
      sig[(size_t)s * sig_stride + v] = sv;
      nuc += (double)sv;
      rank += sv > tau ? 1 : 0;
    }
    s_rank = rank;
    s_nuc = nuc;
  }
  for (int v = warp; v < k; v += nwarps) {
    const float sv = sqrtf(fmaxf(H[v + (size_t)v * ldh].x, 0.f));
    const float f = sv > tau ? (sv - tau) / sv : 0.f;
    for (int m = lane; m < k; m += 32) {
      const float2 w = W[m + (size_t)v * ldh];
      Tp[m + (size_t)v * ldg] = w;
      Gp[m + (size_t)v * ldg] = make_float2(w.x * f, w.y * f);
    }
  }
  __syncthreads();
  if (tid == 0) {
    if (stat) {
      SliceStat st;
      st.rank = s_rank;
      st.sweeps = sweeps;
      st.converged = converged;
      st.pad = 0;
      st.nuc = s_nuc;
      stat[s] = st;
    }
    if (acc) {
      atomicAdd(&acc->total_sweeps, (unsigned long long)sweeps);
      if (!converged) atomicAdd(&acc->nonconverged, 1ull);
      atomicMax(&acc->max_sweeps, sweeps);
    }
  }
}


// ---- FP64 variants of the two k x k solves (RsvtArgs::small_fp64): the same algorithms as
// cholqr_factor_kernel and eig_svt_kernel with the factorisation and the eigen-solve carried
// in FP64 (the Grams arrive in FP32 from the products; the factors T and the rotations W go
// back in FP32).  GB300's FP64 rate is a small fraction of its FP32 rate, so these are the
// reference for the FP32 / double-single defaults (their accuracy and time are compared by
// the tests and the benchmark).
__global__ void __launch_bounds__(1024) cholqr_factor_fp64_kernel(const float2* G, float2* T,
                                                                 const int* slices, int k,
                                                                 int ldg, int64_t gs, float tol,
                                                                 RsvtStat* rstat,
                                                                 const int* kdev) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (kdev) k = *kdev;
  const int s = slices[blockIdx.x];
  const int ldS = k + 1;
  double2* S = reinterpret_cast<double2*>(smem_raw);
  double* piv = reinterpret_cast<double*>(S + (size_t)k * ldS);
  double* dsc = piv + k;
  double2* xd = reinterpret_cast<double2*>(dsc + k);
  int* okc = reinterpret_cast<int*>(xd + k);
  __shared__ double s_dmax;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int tx = tid & 31, ty = tid >> 5;
  const float2* Gp = G + (size_t)s * gs;
  float2* Tp = T + (size_t)s * gs;
  for (int i = tid; i < k; i += nthr) {
    const double g = (double)Gp[i + (size_t)i * ldg].x;
    dsc[i] = g > 0.0 ? sqrt(g) : 0.0;
  }
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int i = 0; i < k; ++i) m = fmax(m, dsc[i]);
    s_dmax = m;
  }
  __syncthreads();
  const double dmin = 1e-30 * s_dmax;
  for (int i = tid; i < k; i += nthr) {
    const bool zero = !(dsc[i] > dmin) || s_dmax == 0.0;
    piv[i] = zero ? 0.0 : 1.0;
    if (zero) dsc[i] = 1.0;
    xd[i] = make_double2(1.0, 0.0);
  }
  __syncthreads();
  for (int r = ty; r < k; r += 32)
    for (int c = tx; c < k; c += 32) {
      double2 v = make_double2(0.0, 0.0);
      if (r <= c && piv[r] != 0.0 && piv[c] != 0.0) {
        const float2 g = Gp[r + (size_t)c * ldg];
        const double inv = 1.0 / (dsc[r] * dsc[c]);
        v = make_double2((double)g.x * inv, (double)g.y * inv);
      }
      S[(size_t)r * ldS + c] = v;
    }
  __syncthreads();
  {
    int far = 0;
    for (int r = ty; r < k; r += 32)
      for (int c = r + 1 + tx; c < k; c += 32) {
        const double2 v = S[(size_t)r * ldS + c];
        far |= fabs(v.x) + fabs(v.y) > 1e-6;
      }
    for (int r = tid; r < k; r += nthr) far |= piv[r] == 0.0;
    if (__syncthreads_or(far) == 0) {
      for (int c = ty; c < k; c += 32)
        for (int i = tx; i < k; i += 32)
          Tp[i + (size_t)c * ldg] = i == c ? make_float2((float)(1.0 / dsc[i]), 0.f)
                                           : make_float2(0.f, 0.f);
      return;
    }
  }
  __shared__ double s_rjj, s_irjj;
  __shared__ int s_ok;
  for (int j = 0; j < k; ++j) {
    if (tid == 0) {
      const double pj = piv[j];
      const bool ok = pj > (double)tol;
      const double r = ok ? sqrt(pj) : 1.0;
      s_ok = ok ? 1 : 0;
      s_rjj = r;
      s_irjj = ok ? 1.0 / r : 0.0;
    }
    __syncthreads();
    const bool okj = s_ok != 0;
    const double rjj = s_rjj, irjj = s_irjj;
    for (int l = j + 1 + tid; l < k; l += nthr) {
      const double2 v = S[(size_t)j * ldS + l];
      S[(size_t)j * ldS + l] = make_double2(v.x * irjj, v.y * irjj);
    }
    for (int i = tid; i < j; i += nthr) {
      const double2 v = S[(size_t)j * ldS + i];
      S[(size_t)j * ldS + i] = make_double2(v.x * irjj, v.y * irjj);
    }
    if (tid == 0) {
      S[(size_t)j * ldS + j] = make_double2(rjj, 0.0);
      const double2 v = xd[j];
      xd[j] = make_double2(v.x * irjj, v.y * irjj);
      okc[j] = okj ? 1 : 0;
    }
    __syncthreads();
    if (okj) {
      for (int l = j + 1 + ty; l < k; l += 32) {
        const double2 a = S[(size_t)j * ldS + l];
        for (int l2 = l + tx; l2 < k; l2 += 32) {
          const double2 b = S[(size_t)j * ldS + l2];
          double2 v = S[(size_t)l * ldS + l2];
          v.x -= a.x * b.x + a.y * b.y;
          v.y -= a.x * b.y - a.y * b.x;
          S[(size_t)l * ldS + l2] = v;
        }
        if (tx == 0) piv[l] -= a.x * a.x + a.y * a.y;
        for (int i = tx; i <= j; i += 32) {
          const double2 xj = i == j ? xd[j] : S[(size_t)j * ldS + i];
          double2 v = S[(size_t)l * ldS + i];
          v.x -= a.x * xj.x - a.y * xj.y;
          v.y -= a.x * xj.y + a.y * xj.x;
          S[(size_t)l * ldS + i] = v;
        }
      }
    }
    __syncthreads();
  }
  for (int c = ty; c < k; c += 32)
    for (int i = tx; i < k; i += 32) {
      double2 v = make_double2(0.0, 0.0);
      if (okc[c] && i <= c) {
        v = i == c ? xd[c] : S[(size_t)c * ldS + i];
        v.x /= dsc[i];
        v.y /= dsc[i];
      }
      Tp[i + (size_t)c * ldg] = make_float2((float)v.x, (float)v.y);
    }
  if (rstat && tid == 0) {
    int nd = 0;
    for (int c = 0; c < k; ++c) nd += okc[c] ? 0 : 1;
    if (nd) atomicAdd(&rstat->drops, nd);
  }
}

// Widest sketch whose FP64 Gram and rotations fit one CTA's shared memory.
constexpr int eig_fp64_max_k() { return 80; }

__global__ void __launch_bounds__(1024) eig_svt_fp64_kernel(float2* G, float2* T, float* sig,
                                                            const int* slices, int k, int ldg,
                                                            int64_t gs, int64_t sig_stride,
                                                            float tau, float tol, int max_sweeps,
                                                            SliceStat* stat, SweepAccum* acc,
                                                            const int* kdev, int abs_stop) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (kdev) k = *kdev;
  const int s = slices[blockIdx.x];
  const int ldh = k + 1;
  double2* H = reinterpret_cast<double2*>(smem_raw);
  double2* W = H + (size_t)k * ldh;
  double* rot = reinterpret_cast<double*>(W + (size_t)k * ldh);   // 4 per pair
  int2* prs = reinterpret_cast<int2*>(rot + 4 * ((k + 1) / 2));
  __shared__ int s_flags;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nthr >> 5;
  float2* Gp = G + (size_t)s * gs;
  float2* Tp = T + (size_t)s * gs;
  for (int c = warp; c < k; c += nwarps)
    for (int m = lane; m < k; m += 32) {
      const float2 g = Gp[m + (size_t)c * ldg];
      H[m + (size_t)c * ldh] = make_double2(g.x, g.y);
      W[m + (size_t)c * ldh] = make_double2(m == c ? 1.0 : 0.0, 0.0);
    }
  const int kp = k + (k & 1);
  const int npair = kp / 2;
  const double tol2 = (double)tol * (double)tol;
  const double big2 = (double)tol / (2.0 * (double)k);
  int sweeps = 0, converged = 0;
  __shared__ double s_floor2;
  __syncthreads();
  // the SVT stopping test (abs_stop), as in eig_svt_kernel
  if (tid == 0) {
    double tr = 0.0;
    for (int m = 0; m < k; ++m) tr += fmax(H[m + (size_t)m * ldh].x, 0.0);
    s_floor2 = abs_stop ? tol2 * (tr / ((double)k * (double)k)) : 0.0;
  }
  __syncthreads();
  const double floor2 = s_floor2;
  for (int sw = 0; sw < max_sweeps && !converged; ++sw) {
    if (tid == 0) s_flags = 0;
    __syncthreads();
    for (int r = 0; r < kp - 1; ++r) {
      if (tid < npair) {
        int p, q;
        circle_pair(r, tid, kp, p, q);
        double cm = 0.0, kr = 0.0, ki = 0.0, on = 0.0;
        if (p < k && q < k) {
          const double al = fmax(H[p + (size_t)p * ldh].x, 0.0);
          const double be = fmax(H[q + (size_t)q * ldh].x, 0.0);
          const double2 c = H[p + (size_t)q * ldh];
          const double c2 = c.x * c.x + c.y * c.y;
          const double ab = al * be;
          if (c2 > tol2 * ab && c2 > floor2 * fmin(al, be) && c2 > 0.0) {
            // the rotation of the one-sided form, in FP64: t = sign(zeta) / (|zeta| +
            // sqrt(1 + zeta^2)), sn = t / r, cs - 1 = -t sn / (1 + r), r = sqrt(1 + t^2)
            const double g = sqrt(c2);
            const double zeta = (be - al) / (2.0 * g);
            double t = 1.0 / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            t = zeta >= 0.0 ? t : -t;
            if (t != 0.0) {
              const double rr = sqrt(1.0 + t * t);
              const double sn = t / rr;
              cm = -(t * sn) / (1.0 + rr);
              kr = sn * (c.x / g);
              ki = sn * (c.y / g);
              on = 1.0;
              atomicOr(&s_flags, c2 > big2 * ab ? 3 : 1);
            }
          }
        }
        rot[4 * tid + 0] = cm;
        rot[4 * tid + 1] = kr;
        rot[4 * tid + 2] = ki;
        rot[4 * tid + 3] = on;
        prs[tid] = make_int2(p, q);
      }
      __syncthreads();
      // columns of H and W: x <- x + cm x - conj(k) y,  y <- y + cm y + k x
      for (int i = warp; i < npair; i += nwarps) {
        if (rot[4 * i + 3] == 0.0) continue;
        const double cm = rot[4 * i], kr = rot[4 * i + 1], ki = rot[4 * i + 2];
        const int2 pq = prs[i];
        for (int m = lane; m < k; m += 32) {
#pragma unroll
          for (int mat = 0; mat < 2; ++mat) {
            double2* X = mat == 0 ? H : W;
            double2& x = X[m + (size_t)pq.x * ldh];
            double2& y = X[m + (size_t)pq.y * ldh];
            const double2 xv = x, yv = y;
            x = make_double2(xv.x + cm * xv.x - (kr * yv.x + ki * yv.y),
                             xv.y + cm * xv.y - (kr * yv.y - ki * yv.x));
            y = make_double2(yv.x + cm * yv.x + (kr * xv.x - ki * xv.y),
                             yv.y + cm * yv.y + (kr * xv.y + ki * xv.x));
          }
        }
      }
      __syncthreads();
      // rows of H: row_p <- row_p + cm row_p - k row_q,  row_q <- row_q + cm row_q + conj(k) row_p
      for (int i = warp; i < npair; i += nwarps) {
        if (rot[4 * i + 3] == 0.0) continue;
        const double cm = rot[4 * i], kr = rot[4 * i + 1], ki = rot[4 * i + 2];
        const int2 pq = prs[i];
        for (int m = lane; m < k; m += 32) {
          double2& x = H[pq.x + (size_t)m * ldh];
          double2& y = H[pq.y + (size_t)m * ldh];
          const double2 xv = x, yv = y;
          x = make_double2(xv.x + cm * xv.x - (kr * yv.x - ki * yv.y),
                           xv.y + cm * xv.y - (kr * yv.y + ki * yv.x));
          y = make_double2(yv.x + cm * yv.x + (kr * xv.x + ki * xv.y),
                           yv.y + cm * yv.y + (kr * xv.y - ki * xv.x));
        }
      }
      __syncthreads();
    }
    const int fl = s_flags;
    ++sweeps;
    if (!(fl & 1) || !(fl & 2)) converged = 1;
    __syncthreads();
  }
  __shared__ int s_rank;
  __shared__ double s_nuc;
  if (tid == 0) {
    int rank = 0;
    double nuc = 0.0;
    for (int v = 0; v < k; ++v) {
      const double sv = sqrt(fmax(H[v + (size_t)v * ldh].x, 0.0));
      sig[(size_t)s * sig_stride + v] = (float)sv;
      nuc += sv;
      rank += sv > (double)tau ? 1 : 0;
    }
    s_rank = rank;
    s_nuc = nuc;
  }
  for (int v = warp; v < k; v += nwarps) {
    const double sv = sqrt(fmax(H[v + (size_t)v * ldh].x, 0.0));
    const double f = sv > (double)tau ? (sv - (double)tau) / sv : 0.0;
    for (int m = lane; m < k; m += 32) {
      const double2 w = W[m + (size_t)v * ldh];
      Tp[m + (size_t)v * ldg] = make_float2((float)w.x, (float)w.y);
      Gp[m + (size_t)v * ldg] = make_float2((float)(w.x * f), (float)(w.y * f));
    }
  }
  __syncthreads();
  if (tid == 0) {
    if (stat) {
      SliceStat st;
      st.rank = s_rank;
      st.sweeps = sweeps;
      st.converged = converged;
      st.pad = 0;
      st.nuc = s_nuc;
      stat[s] = st;
    }
    if (acc) {
      atomicAdd(&acc->total_sweeps, (unsigned long long)sweeps);
      if (!converged) atomicAdd(&acc->nonconverged, 1ull);
      atomicMax(&acc->max_sweeps, sweeps);
    }
  }
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Uniform in [-1, 1) from a counter (SplitMix64 finaliser of key + counter * golden gamma).
__device__ __forceinline__ float urand(unsigned long long key, unsigned long long ctr) {
  const unsigned long long h = mix64(key + (ctr + 1ull) * 0x9e3779b97f4a7c15ull);
  return (float)(unsigned)(h >> 40) * (1.0f / 8388608.0f) - 1.0f;   // 24 bits, FP32
}

// One CTA per slice.  Counts the singular values above max(tau, floor * sigma_max) among the
// k of this call (max over slices into rstat), then refills with random vectors the columns
// c < kfill of P that carry no direction: c >= k, or sigma_c <= 1e-6 sigma_max.
__global__ void __launch_bounds__(256) rsvt_refill_kernel(float2* P, const float* sig,
                                                          const int* slices,
                                                          const unsigned char* isreal, int nw,
                                                          int kmax, int k, int kfill, float tau,
                                                          float floor_rel,
                                                          unsigned long long seed, int iter,
                                                          RsvtStat* rstat, const int* kdev) {
  if (kdev) k = *kdev;
  const int s = slices[blockIdx.x];
  const int tid = threadIdx.x, nthr = blockDim.x;
  __shared__ float s_max;
  const float* sg = sig + (size_t)s * kmax;
  if (tid < 32) {
    // sigma_max and the count above max(tau, floor sigma_max) by one warp (both exact in any
    // order)
    float m = 0.f;
    for (int v = tid; v < k; v += 32) m = fmaxf(m, sg[v]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    const float thr = fmaxf(tau, floor_rel * m);
    int cnt = 0;
    for (int v = tid; v < k; v += 32) cnt += sg[v] > thr ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (tid == 0) {
      s_max = m;
      if (rstat && k > 0) {
        atomicMax(&rstat->rank_max, cnt);
        if (cnt >= k) atomicAdd(&rstat->saturated, 1);
      }
    }
  }
  __syncthreads();
  const float smax = s_max;
  const bool real = isreal && isreal[s];
  const unsigned long long key =
      mix64(seed ^ ((unsigned long long)(unsigned)iter << 32) ^ (unsigned long long)s);
  float2* Ps = P + (size_t)s * nw * kmax;
  // columns to refill, then all their entries spread over the whole CTA
  __shared__ unsigned char need[128];
  for (int c = tid; c < kfill; c += nthr) need[c] = (c >= k || !(sg[c] > 1e-6f * smax)) ? 1 : 0;
  __syncthreads();
  for (int idx = tid; idx < kfill * nw; idx += nthr) {
    const int c = idx / nw, e = idx - c * nw;
    if (!need[c]) continue;
    const unsigned long long ctr = 2ull * ((unsigned long long)c * nw + e);
    Ps[(size_t)e + (size_t)nw * c] = make_float2(urand(key, ctr), real ? 0.f : urand(key, ctr + 1ull));
  }
}

// Device-chosen width: after a call, the next width is the rank seen (max over slices) plus
// the oversampling margin, rounded up to 8, never below the current width, at most kmax; the
// rank maximum restarts for the next call.
__global__ void rsvt_next_k_kernel(RsvtStat* st, int oversample, int kmax) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double kc = st->k;   // the width this iteration ran with
  st->ksum[0] += kc;
  st->ksum[1] += kc * kc;
  st->ksum[2] += kc * kc * kc;
  int kn = (st->rank_max + oversample + 7) / 8 * 8;
  kn = kn > st->k ? kn : st->k;
  kn = kn < kmax ? kn : kmax;
  st->k = kn > 1 ? kn : 1;
  st->rank_max = 0;
}

__global__ void rsvt_state_init_kernel(RsvtStat* st, int k0) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st->rank_max = 0;
  st->saturated = 0;
  st->drops = 0;
  st->k = k0;
  st->ksum[0] = st->ksum[1] = st->ksum[2] = 0.0;
}

// Largest sketch width whose Gram and eigenvectors fit one CTA's shared memory.
constexpr int eig_max_k() { return 112; }

size_t eig_smem(int k) {
  return 2 * (size_t)k * (k + 1) * sizeof(float2) + (size_t)((k + 1) / 2) * (sizeof(float4) + sizeof(int2));
}

size_t eig_fp64_smem(int k) {
  return 2 * (size_t)k * (k + 1) * sizeof(double2) +
         (size_t)((k + 1) / 2) * (4 * sizeof(double) + sizeof(int2));
}

size_t cholqr_fp64_smem(int k) {
  return (size_t)k * (k + 1) * sizeof(double2) + 2 * (size_t)k * sizeof(double) +
         (size_t)k * sizeof(double2) + (size_t)k * sizeof(int);
}

size_t cholqr_smem(int k) {
  return (size_t)k * (k + 1) * sizeof(float2) + 2 * (size_t)k * sizeof(double) +
         (size_t)k * sizeof(float2) + (size_t)k * sizeof(float) + (size_t)k * sizeof(int);
}

cudaError_t gemm_fp32(const CGemm& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  dim3 grid((g.M + TM - 1) / TM, (g.N + TN - 1) / TN, g.batch);
  cgemm_fp32_kernel<<<grid, 256, 0, st>>>(g);
  return cudaGetLastError();
}

CMat mat(const float2* p, const int* idx, int64_t bs, int64_t s0, int64_t s1, int conj = 0) {
  CMat m;
  m.p = p;
  m.idx = idx;
  m.bs = bs;
  m.s0 = s0;
  m.s1 = s1;
  m.conj = conj;
  return m;
}

CGemm gemm(int M, int N, int K, int batch, const CMat& a, const CMat& b, const CMat& c) {
  CGemm g;
  g.M = M;
  g.N = N;
  g.K = K;
  g.batch = batch;
  g.a = a;
  g.b = b;
  g.c = c;
  return g;
}

}  // namespace

cudaError_t launch_cgemm(const CGemm& g, int engine, cudaStream_t st) {
  if (engine == RSVT_GEMM_FP32) return gemm_fp32(g, st);
  return launch_cgemm_tc(g, engine, st);
}

int rsvt_max_k() { return 128; }
int rsvt_eig_max_k() { return eig_max_k(); }

size_t rsvt_jacobi_scratch_bytes(int nw, int kmax, int nslices, const SliceKnobs& kn) {
  size_t b = 0;
  for (int k = 1; k <= kmax; ++k)
    if (jacobi_svt_plan_ok(nw, k, nslices, kn))
      b = std::max(b, jacobi_svt_scratch_bytes(nw, k, nslices, kn));
  return b;
}

cudaError_t launch_rsvt_state_init(RsvtStat* st_dev, int k0, cudaStream_t st) {
  rsvt_state_init_kernel<<<1, 32, 0, st>>>(st_dev, k0);
  return cudaGetLastError();
}

cudaError_t launch_rsvt_refill(const RsvtArgs& a, int k, int kfill, cudaStream_t st) {
  if (kfill > rsvt_max_k()) return cudaErrorInvalidValue;   // the kernel's column flags
  if (a.nslices <= 0) return cudaSuccess;
  // k = 0 (initialisation) refills every column whatever the device width says
  rsvt_refill_kernel<<<a.nslices, 256, 0, st>>>(a.P, a.sig, a.slices, a.isreal, a.nw, a.kmax, k,
                                                kfill, a.tau, a.floor_rel, a.seed, a.iter,
                                                a.rstat, k > 0 ? a.kdev : nullptr);
  return cudaGetLastError();
}

cudaError_t launch_rsvt(const RsvtArgs& a, cudaStream_t st) {
  if (a.nslices <= 0) return cudaSuccess;
  const int k = a.k, kmax = a.kmax, mw = a.mw, nw = a.nw, ns = a.nslices;
  if (k < 1 || k > kmax || kmax > rsvt_max_k() || k > nw) return cudaErrorInvalidValue;
  // with a device-chosen width (k = its bound) only the Gram path of the small SVD applies
  if (a.kdev && (k > eig_max_k() || !a.rstat)) return cudaErrorInvalidValue;
  cudaError_t e;
  const int64_t ys = (int64_t)mw * kmax, ps = (int64_t)nw * kmax, gs = (int64_t)kmax * kmax;
  const int64_t bs = (int64_t)nw * k;
  const int* idx = a.slices;
  // the working matrix Aw(i, j) = A(i, j) or A(j, i): strides (wr, wc) in the spectrum
  const CMat Aw = mat(a.ahat, idx, a.N12, a.wr, a.wc);
  const CMat AwT = mat(a.ahat, idx, a.N12, a.wc, a.wr);
  const size_t csm = cholqr_smem(k);
  static bool attr_set = false;
  if (!attr_set) {
    e = cudaFuncSetAttribute(cholqr_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)cholqr_smem(rsvt_max_k()));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(eig_svt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)eig_smem(eig_max_k()));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(cholqr_factor_fp64_kernel,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)cholqr_fp64_smem(eig_max_k()));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(eig_svt_fp64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)eig_fp64_smem(eig_fp64_max_k()));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  // stage boundaries for the caller's timing (power-step-free calls only)
  // the Gram matrices and triangular applications need FP32-level accuracy (orthogonality):
  // split-TF32 tensor-core products with the tensor-core engines, FP32 CUDA cores otherwise
  const int orth_engine = a.engine == RSVT_GEMM_FP32 ? RSVT_GEMM_FP32 : RSVT_GEMM_3XTF32;
  // products whose flagged dimensions equal the width read it from the device in that mode
  auto dyn = [&](CGemm g, int dm, int dn, int dk) {
    if (a.kdev) {
      g.kdev = a.kdev;
      g.dynM = dm;
      g.dynN = dn;
      g.dynK = dk;
    }
    return g;
  };
  auto mark = [&](int i) -> cudaError_t {
    return (a.stage_ev && a.power == 0) ? cudaEventRecord(a.stage_ev[i], st) : cudaSuccess;
  };
  if ((e = mark(0)) != cudaSuccess) return e;
  for (int pw = 0; pw <= a.power; ++pw) {
    // Y = Aw P   (power steps: P = conj(Bt) of the previous projection)
    const CMat Pm = pw == 0 ? mat(a.P, idx, ps, 1, nw) : mat(a.Bt, idx, bs, 1, nw, 1);
    e = launch_cgemm(dyn(gemm(mw, k, nw, ns, Aw, Pm, mat(a.Y, idx, ys, 1, mw)), 0, 1, 0),
                     a.engine, st);
    if (e != cudaSuccess) return e;
    if ((e = mark(1)) != cudaSuccess) return e;
    // CholeskyQR2: Y -> Q -> Y
    for (int pass = 0; pass < 2; ++pass) {
      float2* src = pass == 0 ? a.Y : a.Q;
      float2* dst = pass == 0 ? a.Q : a.Y;
      e = launch_cgemm(dyn(gemm(k, k, mw, ns, mat(src, idx, ys, mw, 1, 1),
                                mat(src, idx, ys, 1, mw), mat(a.G, idx, gs, 1, kmax)),
                           1, 1, 0),
                       orth_engine, st);
      if (e != cudaSuccess) return e;
      if (a.small_fp64 && k <= eig_max_k())   // (wider: the FP32 factorisation)
        cholqr_factor_fp64_kernel<<<ns, 1024, cholqr_fp64_smem(k), st>>>(
            a.G, a.T, idx, k, kmax, gs, a.chol_tol, a.rstat, a.kdev);
      else
        cholqr_factor_kernel<<<ns, 1024, csm, st>>>(a.G, a.T, idx, k, kmax, gs, a.chol_tol,
                                                   a.rstat, a.kdev);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      e = launch_cgemm(dyn(gemm(mw, k, k, ns, mat(src, idx, ys, 1, mw),
                                mat(a.T, idx, gs, 1, kmax), mat(dst, idx, ys, 1, mw)),
                           0, 1, 1),
                       orth_engine, st);
      if (e != cudaSuccess) return e;
    }
    if ((e = mark(2)) != cudaSuccess) return e;
    // Bt = Aw^T conj(Q)
    e = launch_cgemm(
        dyn(gemm(nw, k, mw, ns, AwT, mat(a.Y, idx, ys, 1, mw, 1), mat(a.Bt, idx, bs, 1, nw)), 0,
            1, 0),
        a.engine, st);
    if (e != cudaSuccess) return e;
    if ((e = mark(3)) != cudaSuccess) return e;
  }
  if (k <= eig_max_k()) {
    // Dt = D_tau(Bt) through the k x k Gram: H = Bt^H Bt, two-sided Jacobi -> W, W diag(f),
    // sigma; P = conj(Bt W); Dt = Bt W diag(f) W^H = conj(P) (W diag(f))^H
    e = launch_cgemm(dyn(gemm(k, k, nw, ns, mat(a.Bt, idx, bs, nw, 1, 1),
                              mat(a.Bt, idx, bs, 1, nw), mat(a.G, idx, gs, 1, kmax)),
                         1, 1, 0),
                     orth_engine, st);
    if (e != cudaSuccess) return e;
    if (a.small_fp64 && k <= eig_fp64_max_k())
      eig_svt_fp64_kernel<<<ns, 1024, eig_fp64_smem(k), st>>>(a.G, a.T, a.sig, idx, k, kmax, gs,
                                                              kmax, a.tau, a.tol, a.max_sweeps,
                                                              a.stat, a.acc, a.kdev, a.abs_stop);
    else
      eig_svt_kernel<<<ns, 1024, eig_smem(k), st>>>(a.G, a.T, a.sig, idx, k, kmax, gs, kmax,
                                                    a.tau, a.tol, a.max_sweeps, a.stat, a.acc,
                                                    a.kdev, a.abs_stop);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = launch_cgemm(dyn(gemm(nw, k, k, ns, mat(a.Bt, idx, bs, 1, nw, 1),
                              mat(a.T, idx, gs, 1, kmax, 1), mat(a.P, idx, ps, 1, nw)),
                         0, 1, 1),
                     orth_engine, st);
    if (e != cudaSuccess) return e;
    e = launch_cgemm(dyn(gemm(nw, k, k, ns, mat(a.P, idx, ps, 1, nw, 1),
                              mat(a.G, idx, gs, kmax, 1, 1), mat(a.Dt, idx, bs, 1, nw)),
                         0, 1, 1),
                     orth_engine, st);
    if (e != cudaSuccess) return e;
    if ((e = mark(4)) != cudaSuccess) return e;
    e = launch_cgemm(dyn(gemm(mw, nw, k, ns, mat(a.Y, idx, ys, 1, mw), mat(a.Dt, idx, bs, nw, 1),
                              mat(a.zhat, idx, a.N12, a.wr, a.wc)),
                         0, 0, 1),
                     a.engine, st);
    if (e != cudaSuccess) return e;
    if ((e = mark(5)) != cudaSuccess) return e;
    if ((e = launch_rsvt_refill(a, k, a.kfill, st)) != cudaSuccess) return e;
    if (a.kdev) {
      rsvt_next_k_kernel<<<1, 32, 0, st>>>(a.rstat, a.oversample, kmax < k ? kmax : k);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return mark(6);
  }
  // Dt = D_tau(Bt), converged vectors -> P (conjugated), singular values -> sig
  SliceArgs j;
  j.ahat = a.Bt;
  j.zhat = a.Dt;
  j.slices = idx;
  j.nslices = ns;
  j.n1 = nw;
  j.n2 = k;
  j.N12 = bs;
  j.tau = a.tau;
  j.tol = a.tol;
  j.abs_stop = a.abs_stop;
  j.max_sweeps = a.max_sweeps;
  j.stat = a.stat;
  j.acc = a.acc;
  j.scratch = a.jscratch;
  j.scratch_bytes = a.jscratch_bytes;
  j.knobs = a.jknobs;
  j.wout = a.P;
  j.wout_stride = ps;
  j.wout_conj = 1;
  j.sigout = a.sig;
  j.sig_stride = kmax;
  e = launch_jacobi_svt(j, st);
  if (e != cudaSuccess) return e;
  if ((e = mark(4)) != cudaSuccess) return e;
  // Zw = Q Dt^T, written into the output spectrum with the orientation of Aw
  e = launch_cgemm(gemm(mw, nw, k, ns, mat(a.Y, idx, ys, 1, mw), mat(a.Dt, idx, bs, nw, 1),
                        mat(a.zhat, idx, a.N12, a.wr, a.wc)),
                   a.engine, st);
  if (e != cudaSuccess) return e;
  if ((e = mark(5)) != cudaSuccess) return e;
  if ((e = launch_rsvt_refill(a, k, a.kfill, st)) != cudaSuccess) return e;
  return mark(6);
}

}  // namespace tsvd
