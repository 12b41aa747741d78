// slice_svt.cu -- singular value thresholding of every Fourier slice (the Z-step of the
// completion ADMM, eq. shrink split into the per-slice problems of eq. shrink2, and the
// L-step of tensor RPCA, eq. low_rank), solved by the Lemma of Sec. 4.1:
//     D_tau(A) = U diag((sigma_i - tau)_+) V^H.
//
// The SVD is a one-sided (Hestenes) Jacobi iteration on the nv = min(n1, n2) "vectors" of
// the slice (its columns when n1 >= n2, otherwise its rows, i.e. the columns of A^T, since
// D_tau(A^T) = D_tau(A)^T).  The plane rotation of a pair diagonalises its 2x2 Gram matrix
// [[a, c], [c*, b]]:
//     c = |c| e^{i phi},  zeta = (b - a) / (2|c|),  t = sign(zeta) / (|zeta| + sqrt(1+zeta^2)),
//     cs = 1/sqrt(1+t^2), sn = cs t,
//     x <- cs x - sn e^{-i phi} y,   y <- sn e^{i phi} x + cs y.
// A pair is rotated while |c|^2 > tol^2 a b; sweeps stop when a whole sweep rotates
// nothing (or at max_sweeps).  The converged vectors are W = B V = U diag(sigma).
//
// Rebuild.  Two forms:
//   U form (default):  D_tau(B) = sum_{sigma_i > tau} ((sigma_i - tau)/sigma_i) u_i (u_i^H B),
//            u_i = w_i / sigma_i, re-reading the original slice B from global memory (L2);
//   V form (opt-in):   the rotations are also applied to V (stored after each vector, V = I
//            at the start) and D_tau(B) = sum_{sigma_i > tau} ((sigma_i - tau)/sigma_i) w_i v_i^H.
// The V form costs one more rotation of an nv-vector per pair and halves the rebuild, but
// W and V collect independent rounding over the rotations, so W v^H drifts from B v v^H by
// about eps sqrt(rotations) |B|; the U form projects the original B and does not.  With V
// accumulated for a warm start (vin / vout), the rebuild can still be the U form (brb).
//
// Rounding.  Each rotation is applied as x + (cs - 1) x - conj(k) y with cs - 1 computed to
// full relative precision: in FP32, cs rounds to exactly 1 for small angles while sn = t
// does not, so the textbook form makes every late rotation slightly norm-increasing and the
// singular values drift upward over the thousands of rotations a vector takes.
//
// Work split.  A slice is owned by a thread-block cluster of C CTAs (C = 1, 2, 4, 8).  Its
// vectors form nb = 2C blocks of bs vectors (zero vectors pad the last block); a sweep is a
// round-robin tournament of the blocks: in block round r CTA c holds the pair of blocks of
// slot c of the circle method.  Round 0 rotates every vector pair inside the two blocks,
// later rounds only the bs x bs cross pairs, so each vector pair meets once per sweep.
// Inside a CTA the pairs of a local round are disjoint and run concurrently, G lanes per
// pair (32/G pairs per warp), with the inner products reduced by shuffles inside the group.
// Between block rounds the CTAs trade blocks through a double-buffered global buffer (one
// cluster barrier per exchange).  For the rebuild the CTAs pool their kept vectors in the
// exchange buffer (in cluster-rank order) and each CTA writes D_tau(B) for 1/C of the
// columns from all of them: every entry is summed in a fixed order (deterministic) and no
// CTA writes a partial slice.
//
// Shared memory holds a CTA's 2 bs vectors in planar form: a real plane and an imaginary
// plane, rows of pitch rowp floats (the vector's ld entries, then in the V form its ldv V
// entries; pitches are multiples of 4, zero padded).  A lane moves 4 consecutive entries of
// a plane with one 128-bit access and does the complex arithmetic of two entries at a time
// with packed FP32x2 instructions (__ffma2_rn / __fmul2_rn).  A pair's vector entries stay
// in registers between the inner products and the rotation; V entries are streamed.
//
// A slice whose matrix is exactly real (the self-conjugate Fourier slices) stays exactly
// real: every inner product then has a zero imaginary part and every rotation is real.
#include "tsvd_internal.h"
#include "tube_tile.cuh"

#include <algorithm>
#include <cooperative_groups.h>
#include <cstring>

namespace cg = cooperative_groups;

namespace tsvd {
namespace {

constexpr int kNC = 8;            // rebuild chunk width (columns of B per chunk)
constexpr int kMinWarps = 4;
constexpr int kMinBlock = 16;     // fewest vectors per block before a slice is split further
constexpr size_t kStaticSmemReserve = 1024;   // static __shared__ of the kernel, with margin

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 lo(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi(const float4& v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 f4(const float2& a, const float2& b) {
  return make_float4(a.x, a.y, b.x, b.y);
}

template <int G>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Pair (p, q) of slot `slot` in round r of the circle method over P (even) players.
__host__ __device__ inline void round_robin_pair(int r, int slot, int P, int& p, int& q) {
  if (slot == 0) {
    p = P - 1;
    q = r;
  } else {
    p = (r + slot) % (P - 1);
    q = (r - slot + P - 1) % (P - 1);
  }
}

struct SliceShape {
  int nv;     // number of vectors
  int len;    // vector length
  int ld;     // pitch of the vector entries in a row (floats, multiple of 4)
  int ldv;    // V form: pitch of the V entries (multiple of 4); 0 in the U form
  int rowp;   // row pitch = ld + ldv
  int rows;   // 1: vectors are the rows of the slice
  int nc;     // rebuild chunk width
  int G;      // lanes per pair
  int cpl;    // 4-entry chunks per lane
  int np;     // vector pairs a group keeps in flight (1 or 2)
  int vform;  // 1: V form rebuild
  int C;      // CTAs per slice (cluster size)
  int nb;     // vector blocks = 2C
  int bs;     // vectors per block
  int kcap;   // kept vectors per rebuild group: 2 bs, or as many rows of ld floats as the
              // 2 bs rows of rowp floats hold (a cluster's U-form rebuild imports those)
  size_t xbuf_floats;   // exchange buffer per slice (floats)
  int block;  // 1: block rounds run on the Gram of the local vectors (block form)
  int nlp;    // block form: row pitch of the Gram and of the accumulated rotation (odd)
};

// Floats of the block form's extra shared memory: the Gram G and the accumulated rotation W
// (nl x nlp, planar re / im each) and, per pair slot, its rotation (float4) and indices (int2).
__host__ __device__ inline size_t block_smem_floats(const SliceShape& sh) {
  if (!sh.block) return 0;
  const size_t nl = 2 * (size_t)sh.bs;
  return 4 * nl * sh.nlp + 6 * (size_t)sh.bs;
}

__host__ __device__ inline size_t slice_smem_bytes(const SliceShape& sh) {
  const size_t nl = 2 * (size_t)sh.bs;   // vectors held by one CTA
  const size_t kc = (size_t)sh.kcap;
  // the block form's region starts 16-byte aligned after the kept-vector indices
  const size_t base = 2 * nl * sh.rowp * sizeof(float) + (size_t)sh.len * sh.nc * sizeof(float2) +
                      kc * sh.nc * sizeof(float2) + nl * sizeof(float) +
                      kc * (sizeof(float) + sizeof(int));
  return (base + 15) / 16 * 16 + block_smem_floats(sh) * sizeof(float);
}

// x' = x + (cs-1) x - conj(k) y ;  y' = y + (cs-1) y + k x on two entries of each plane
// (planar re / im).  CM = cs - 1 is carried separately: cs itself rounds to 1 in FP32 for
// small angles while sn does not, which made every late rotation slightly norm-increasing.
__device__ __forceinline__ void rotate2(const float2 CM, const float2 KR, const float2 KI,
                                        const float2 NKR, const float2 NKI, float2& xr,
                                        float2& xi, float2& yr, float2& yi) {
  const float2 nxr = __ffma2_rn(NKI, yi, __ffma2_rn(NKR, yr, __ffma2_rn(CM, xr, xr)));
  const float2 nxi = __ffma2_rn(KI, yr, __ffma2_rn(NKR, yi, __ffma2_rn(CM, xi, xi)));
  const float2 nyr = __ffma2_rn(NKI, xi, __ffma2_rn(KR, xr, __ffma2_rn(CM, yr, yr)));
  const float2 nyi = __ffma2_rn(KI, xr, __ffma2_rn(KR, xi, __ffma2_rn(CM, yi, yi)));
  xr = nxr;
  xi = nxi;
  yr = nyr;
  yi = nyi;
}

__device__ __forceinline__ void rotate4(const float2 CS, const float2 KR, const float2 KI,
                                        const float2 NKR, const float2 NKI, float4& xr,
                                        float4& xi, float4& yr, float4& yi) {
  float2 xr0 = lo(xr), xr1 = hi(xr), xi0 = lo(xi), xi1 = hi(xi);
  float2 yr0 = lo(yr), yr1 = hi(yr), yi0 = lo(yi), yi1 = hi(yi);
  rotate2(CS, KR, KI, NKR, NKI, xr0, xi0, yr0, yi0);
  rotate2(CS, KR, KI, NKR, NKI, xr1, xi1, yr1, yi1);
  xr = f4(xr0, xr1);
  xi = f4(xi0, xi1);
  yr = f4(yr0, yr1);
  yi = f4(yi0, yi1);
}

// Reduce K values over the G lanes of a group, all K shuffles of a level back to back.
template <int G, int K>
__device__ __forceinline__ void group_sum_n(float (&v)[K]) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  }
}

// The rotation of a vector pair from its 2 x 2 Gram entries al = ||x||^2, be = ||y||^2 and
// x^H y = cr + i ci: 0 when the pair is orthogonal to the tolerance (|x^H y|^2 <= tol2 al be,
// or |x^H y|^2 <= floor2 min(al, be): see svt_slice) or the angle rounds to 0, else 1, or 3
// when |cos|^2 = |x^H y|^2 / (al be) > big2; with cm = cs - 1 and k = kr + i ki =
// sn e^{i phi} (see jacobi_pairs for the arithmetic).
__device__ __forceinline__ int pair_rotation(float al, float be, float cr, float ci, float tol2,
                                             float floor2, float big2, float& cm, float& kr,
                                             float& ki) {
  const float c2 = cr * cr + ci * ci;
  const float ab = al * be;
  if (!(c2 > tol2 * ab) || !(c2 > floor2 * fminf(al, be))) return 0;
  // ~ 1 / |x^H y| (the exact form below the normal range, where the approximation is not
  // defined: only vectors of norm ~1e-14 get there)
  const float inv_g = c2 >= 1e-30f ? rsqrtf(c2) : 1.f / sqrtf(c2);
  const float zeta = (be - al) * (0.5f * inv_g);
  const float az = fabsf(zeta);
  const float z1 = fmaf(zeta, zeta, 1.f);                         // inf past |zeta| ~ 1e19
  const float t0 = __fdividef(1.f, az + z1 * rsqrtf(z1));
  float t = az > 1e18f ? __fdividef(0.5f, az) : t0;
  t = zeta >= 0.f ? t : -t;
  if (t == 0.f) return 0;
  const float q1 = fmaf(t, t, 1.f);
  const float rs = rsqrtf(q1);                                    // ~ 1 / r
  const float r = q1 * rs;
  const float sn = t * rs;
  cm = __fdividef(-(t * sn), 1.f + r);
  kr = sn * (cr * inv_g);                                         // k = sn e^{i phi}
  ki = sn * (ci * inv_g);
  return c2 > big2 * ab ? 3 : 1;
}

// Local vectors (pp, qq) of pair slot `slot` < bs in local round lr of block round r: round 0
// pairs every two of the nl = 2 bs local vectors (circle method over nl - 1 rounds), later
// rounds only the bs x bs cross pairs (bs rounds).
__device__ __forceinline__ void local_pair(int r, int lr, int slot, int nl, int bs, int& pp,
                                           int& qq) {
  if (r == 0) {
    if (slot == 0) {
      pp = nl - 1;
      qq = lr;
    } else {
      pp = lr + slot;
      if (pp >= nl - 1) pp -= nl - 1;
      qq = lr - slot + nl - 1;
      if (qq >= nl - 1) qq -= nl - 1;
    }
  } else {
    pp = slot;
    qq = slot + lr;
    if (qq >= bs) qq -= bs;
    qq += bs;
  }
}

// Rotate NP independent vector pairs (p[i], q[i]) if they are not yet orthogonal; NP = 2
// interleaves two pairs so that one pair's inner products, shuffles and rotation-parameter
// chain overlap the other's.  All G lanes of the group call it with the same pairs; pairs
// with real[i] false are skipped.  A row holds exactly G * CPL vector chunks (zero padded
// past the vector, so no lane needs a bounds test) and then nchunkv V chunks, a multiple of
// G.  Returns bit 0 set when a rotation was applied and bit 1 set when one of them had
// |cos|^2 = |x^H y|^2 / (||x||^2 ||y||^2) above big2.
//
// Rotation parameters: the exact rotation of the pair's 2x2 Gram matrix needs t, and a
// unitary update needs cs^2 + sn^2 = 1.  t only steers convergence, so it is computed with
// the approximate reciprocal square root and division; cs and sn come from r = sqrt(1 + t^2)
// as sn = t / r and cs - 1 = -t sn / (1 + r), an identity that holds for any r, so a relative
// error d in r (or in 1/|x^H y| for the phase) changes cs^2 + sn^2 by only ~1.5 t^2 d: nothing
// for the small rotations that make up all but the first sweep.
template <int G, int CPL, int NP>
__device__ __forceinline__ int jacobi_pairs(float* __restrict__ Wr, float* __restrict__ Wi,
                                            int rowp, int nchunkv, const int (&p)[NP],
                                            const int (&q)[NP], const bool (&real)[NP],
                                            int gl, float tol2, float floor2, float big2) {
  float4 xr[NP][CPL], xi[NP][CPL], yr[NP][CPL], yi[NP][CPL];
  float2 acc[NP][8];
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    const float4* xr4 = reinterpret_cast<const float4*>(Wr + p[i] * rowp);
    const float4* xi4 = reinterpret_cast<const float4*>(Wi + p[i] * rowp);
    const float4* yr4 = reinterpret_cast<const float4*>(Wr + q[i] * rowp);
    const float4* yi4 = reinterpret_cast<const float4*>(Wi + q[i] * rowp);
#pragma unroll
    for (int u = 0; u < CPL; ++u) {
      const int c = gl + G * u;
      xr[i][u] = xr4[c];
      xi[i][u] = xi4[c];
      yr[i][u] = yr4[c];
      yi[i][u] = yi4[c];
    }
  }
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    float2* A = acc[i];
    // first chunk initialises the sums
    A[0] = __fmul2_rn(lo(xr[i][0]), lo(xr[i][0]));   // ||x||^2
    A[1] = __fmul2_rn(hi(xr[i][0]), hi(xr[i][0]));
    A[2] = __fmul2_rn(lo(yr[i][0]), lo(yr[i][0]));   // ||y||^2
    A[3] = __fmul2_rn(hi(yr[i][0]), hi(yr[i][0]));
    A[4] = __fmul2_rn(lo(xr[i][0]), lo(yr[i][0]));   // Re(x^H y) = xr.yr + xi.yi
    A[5] = __fmul2_rn(hi(xr[i][0]), hi(yr[i][0]));
    A[6] = __fmul2_rn(lo(xr[i][0]), lo(yi[i][0]));   // Im(x^H y) = xr.yi - xi.yr
    A[7] = __fmul2_rn(lo(xi[i][0]), lo(yr[i][0]));
    A[0] = __ffma2_rn(lo(xi[i][0]), lo(xi[i][0]), A[0]);
    A[1] = __ffma2_rn(hi(xi[i][0]), hi(xi[i][0]), A[1]);
    A[2] = __ffma2_rn(lo(yi[i][0]), lo(yi[i][0]), A[2]);
    A[3] = __ffma2_rn(hi(yi[i][0]), hi(yi[i][0]), A[3]);
    A[4] = __ffma2_rn(lo(xi[i][0]), lo(yi[i][0]), A[4]);
    A[5] = __ffma2_rn(hi(xi[i][0]), hi(yi[i][0]), A[5]);
    A[6] = __ffma2_rn(hi(xr[i][0]), hi(yi[i][0]), A[6]);
    A[7] = __ffma2_rn(hi(xi[i][0]), hi(yr[i][0]), A[7]);
  }
#pragma unroll
  for (int u = 1; u < CPL; ++u) {
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      float2* A = acc[i];
      A[0] = __ffma2_rn(lo(xr[i][u]), lo(xr[i][u]), A[0]);
      A[1] = __ffma2_rn(hi(xr[i][u]), hi(xr[i][u]), A[1]);
      A[0] = __ffma2_rn(lo(xi[i][u]), lo(xi[i][u]), A[0]);
      A[1] = __ffma2_rn(hi(xi[i][u]), hi(xi[i][u]), A[1]);
      A[2] = __ffma2_rn(lo(yr[i][u]), lo(yr[i][u]), A[2]);
      A[3] = __ffma2_rn(hi(yr[i][u]), hi(yr[i][u]), A[3]);
      A[2] = __ffma2_rn(lo(yi[i][u]), lo(yi[i][u]), A[2]);
      A[3] = __ffma2_rn(hi(yi[i][u]), hi(yi[i][u]), A[3]);
      A[4] = __ffma2_rn(lo(xr[i][u]), lo(yr[i][u]), A[4]);
      A[5] = __ffma2_rn(hi(xr[i][u]), hi(yr[i][u]), A[5]);
      A[4] = __ffma2_rn(lo(xi[i][u]), lo(yi[i][u]), A[4]);
      A[5] = __ffma2_rn(hi(xi[i][u]), hi(yi[i][u]), A[5]);
      A[6] = __ffma2_rn(lo(xr[i][u]), lo(yi[i][u]), A[6]);
      A[6] = __ffma2_rn(hi(xr[i][u]), hi(yi[i][u]), A[6]);
      A[7] = __ffma2_rn(lo(xi[i][u]), lo(yr[i][u]), A[7]);
      A[7] = __ffma2_rn(hi(xi[i][u]), hi(yr[i][u]), A[7]);
    }
  }
  float red[4 * NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    const float2* A = acc[i];
    red[4 * i + 0] = (A[0].x + A[0].y) + (A[1].x + A[1].y);
    red[4 * i + 1] = (A[2].x + A[2].y) + (A[3].x + A[3].y);
    red[4 * i + 2] = (A[4].x + A[4].y) + (A[5].x + A[5].y);
    red[4 * i + 3] = (A[6].x + A[6].y) - (A[7].x + A[7].y);
  }
  group_sum_n<G, 4 * NP>(red);
  const int ncv = nchunkv / G;
  int flags = 0;
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    if (!real[i]) continue;
    float cm, kr, ki;
    const int fl = pair_rotation(red[4 * i + 0], red[4 * i + 1], red[4 * i + 2], red[4 * i + 3],
                                 tol2, floor2, big2, cm, kr, ki);
    if (!fl) continue;
    const float2 CM = f2(cm, cm), KR = f2(kr, kr), KI = f2(ki, ki), NKR = f2(-kr, -kr),
                 NKI = f2(-ki, -ki);
    float4* xr4 = reinterpret_cast<float4*>(Wr + p[i] * rowp);
    float4* xi4 = reinterpret_cast<float4*>(Wi + p[i] * rowp);
    float4* yr4 = reinterpret_cast<float4*>(Wr + q[i] * rowp);
    float4* yi4 = reinterpret_cast<float4*>(Wi + q[i] * rowp);
#pragma unroll
    for (int u = 0; u < CPL; ++u) {
      const int c = gl + G * u;
      rotate4(CM, KR, KI, NKR, NKI, xr[i][u], xi[i][u], yr[i][u], yi[i][u]);
      xr4[c] = xr[i][u];
      xi4[c] = xi[i][u];
      yr4[c] = yr[i][u];
      yi4[c] = yi[i][u];
    }
    for (int u = 0; u < ncv; ++u) {
      const int c = G * CPL + gl + G * u;
      float4 vxr = xr4[c], vxi = xi4[c], vyr = yr4[c], vyi = yi4[c];
      rotate4(CM, KR, KI, NKR, NKI, vxr, vxi, vyr, vyi);
      xr4[c] = vxr;
      xi4[c] = vxi;
      yr4[c] = vyr;
      yi4[c] = vyi;
    }
    flags |= fl;
  }
  return flags;
}

// Largest CTA for a chunk count: the pair registers (16 floats per chunk) must fit.
// `chunks` = chunks per lane x pairs in flight.
__host__ __device__ constexpr int max_warps_for(int chunks) {
  return chunks <= 2 ? 24 : chunks == 3 ? 18 : chunks == 4 ? 16
       : chunks <= 8 ? 12 : 8;
}

// Copy block `blk` of the slice (vectors blk*bs .. blk*bs+bs-1, zero past nv) into local
// slot `slot`; in the V form the V entries of vector g start as the unit vector e_g.
__device__ void load_block_from_slice(float* Wr, float* Wi, const float2* __restrict__ A,
                                      const SliceShape& sh, int n1, int blk, int slot,
                                      const float2* __restrict__ Vin) {
  const int bs = sh.bs, len = sh.len, rowp = sh.rowp;
  const int v0 = blk * bs;
  const int nvalid = max(0, min(bs, sh.nv - v0));
  const int tid = threadIdx.x, nthr = blockDim.x;
  float* r0 = Wr + (size_t)slot * bs * rowp;
  float* i0 = Wi + (size_t)slot * bs * rowp;
  // zero everything the slice does not cover: the tail of each row and padding vectors
  const int tail = rowp - len;
  for (int idx = tid; idx < nvalid * tail; idx += nthr) {
    const int k = idx / tail, p = len + idx % tail;
    r0[(size_t)k * rowp + p] = 0.f;
    i0[(size_t)k * rowp + p] = 0.f;
  }
  for (int idx = tid; idx < (bs - nvalid) * rowp; idx += nthr) {
    const int k = nvalid + idx / rowp, p = idx % rowp;
    r0[(size_t)k * rowp + p] = 0.f;
    i0[(size_t)k * rowp + p] = 0.f;
  }
  __syncthreads();
  if (sh.vform && Vin) {
    // warm start: V entries of vector g are column g of the given V (nv x nv, col-major)
    for (int idx = tid; idx < nvalid * sh.nv; idx += nthr) {
      const int k = idx / sh.nv, i = idx % sh.nv;
      const float2 v = Vin[(size_t)i + (size_t)sh.nv * (v0 + k)];
      r0[(size_t)k * rowp + sh.ld + i] = v.x;
      i0[(size_t)k * rowp + sh.ld + i] = v.y;
    }
  } else if (sh.vform) {
    for (int k = tid; k < nvalid; k += nthr) r0[(size_t)k * rowp + sh.ld + v0 + k] = 1.f;
  }
  if (!sh.rows) {
    // vector v = column v0 + k: entries A[p + n1 (v0 + k)], contiguous in p
    for (int idx = tid; idx < nvalid * len; idx += nthr) {
      const int k = idx / len, p = idx % len;
      const float2 x = A[(size_t)p + (size_t)n1 * (v0 + k)];
      r0[(size_t)k * rowp + p] = x.x;
      i0[(size_t)k * rowp + p] = x.y;
    }
  } else {
    // vector v = row v0 + k: entries A[(v0 + k) + n1 p]; k fastest across threads
    for (int idx = tid; idx < nvalid * len; idx += nthr) {
      const int k = idx % nvalid, p = idx / nvalid;
      const float2 x = A[(size_t)(v0 + k) + (size_t)n1 * p];
      r0[(size_t)k * rowp + p] = x.x;
      i0[(size_t)k * rowp + p] = x.y;
    }
  }
}

// Exchange buffer of one slice: [parity][block][plane][bs][rowp] floats.
__device__ __forceinline__ float* xblock(float* xbuf, const SliceShape& sh, int par, int blk,
                                         int plane) {
  return xbuf + (((size_t)par * sh.nb + blk) * 2 + plane) * (size_t)sh.bs * sh.rowp;
}

// Copy n floats (n a multiple of 4) with 128-bit accesses; each thread issues up to 8 loads
// before its stores so the L2 latency of the block exchange overlaps.
__device__ void copy_floats4(float* __restrict__ dst, const float* __restrict__ src, size_t n) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
  float4* d4 = reinterpret_cast<float4*>(dst);
  const size_t n4 = n / 4, step = blockDim.x;
  for (size_t base = threadIdx.x; base < n4; base += 8 * step) {
    float4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const size_t i = base + u * step;
      v[u] = i < n4 ? s4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const size_t i = base + u * step;
      if (i < n4) d4[i] = v[u];
    }
  }
}

// Global index of entry p of column c of B (the slice in vector orientation).
__device__ __forceinline__ size_t b_index(const SliceShape& sh, int n1, int p, int c) {
  return sh.rows ? (size_t)c + (size_t)n1 * p : (size_t)p + (size_t)n1 * c;
}

// Register budget of a thread: the register file over the largest CTA for a chunk count
// (the launch trims the CTA when the allocation granularity leaves fewer threads).
__host__ __device__ constexpr int max_regs_for(int chunks) {
  return (65536 / (max_warps_for(chunks) * 32)) / 8 * 8 > 255
             ? 255
             : (65536 / (max_warps_for(chunks) * 32)) / 8 * 8;
}

// Shared-memory scalars of one slice SVT (static __shared__ in the kernels: the same offset
// in every CTA of a cluster, so they can be read across the cluster).
struct SliceShared {
  int flag[2];
  int rank;
  double nuc;
  float energy;   // this CTA's part of ||B||_F^2
};

// The vectors of blocks bx (local slot 0) and by (slot 1) of the pre-rotated slice, computed
// while loading: vector g = sum_l V(l, g) b_l, where b_l is vector l of the slice B (its
// column, or its row when the vectors are rows) and V the nv x nv matrix Vin -- i.e. column g
// of B V (columns) or row g of V^T B (rows), the input the V form expects with vin = V.  The
// V entries of vector g start as column g of V.  The slice's vectors are staged nc at a time
// in the rebuild's chunk buffer Bc (len x nc) and the matching rows of V in Cc (2 bs x nc).
__device__ void load_blocks_rotated(float* Wr, float* Wi, const float2* __restrict__ B,
                                    const float2* __restrict__ Vin, const SliceShape& sh, int n1,
                                    int bx, int by, float2* Bc, float2* Cc) {
  const int bs = sh.bs, len = sh.len, rowp = sh.rowp, nv = sh.nv, nc = sh.nc, nl = 2 * bs;
  const int tid = threadIdx.x, nthr = blockDim.x;
  auto gidx = [&](int k) { return k < bs ? bx * bs + k : by * bs + k - bs; };
  for (int idx = tid; idx < nl * rowp; idx += nthr) {
    Wr[idx] = 0.f;
    Wi[idx] = 0.f;
  }
  __syncthreads();
  for (int idx = tid; idx < nl * nv; idx += nthr) {
    const int k = idx / nv, i = idx % nv, g = gidx(k);
    if (g >= nv) continue;
    const float2 v = Vin[(size_t)i + (size_t)nv * g];
    Wr[(size_t)k * rowp + sh.ld + i] = v.x;
    Wi[(size_t)k * rowp + sh.ld + i] = v.y;
  }
  const int len4 = (len + 3) / 4;
  for (int l0 = 0; l0 < nv; l0 += nc) {
    const int ncur = min(nc, nv - l0);
    for (int idx = tid; idx < len * ncur; idx += nthr) {
      int e, cc;
      if (!sh.rows) {
        e = idx % len;
        cc = idx / len;
      } else {
        cc = idx % ncur;
        e = idx / ncur;
      }
      Bc[e + (size_t)len * cc] = B[sh.rows ? (size_t)(l0 + cc) + (size_t)n1 * e
                                           : (size_t)e + (size_t)n1 * (l0 + cc)];
    }
    for (int idx = tid; idx < nl * ncur; idx += nthr) {
      const int k = idx / ncur, cc = idx % ncur, g = gidx(k);
      Cc[(size_t)k * nc + cc] =
          g < nv ? Vin[(size_t)(l0 + cc) + (size_t)nv * g] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int idx = tid; idx < nl * len4; idx += nthr) {
      const int k = idx / len4, e0 = 4 * (idx % len4);
      float* wr = Wr + (size_t)k * rowp + e0;
      float* wi = Wi + (size_t)k * rowp + e0;
      float4 ar = *reinterpret_cast<const float4*>(wr), ai = *reinterpret_cast<const float4*>(wi);
      float accr[4] = {ar.x, ar.y, ar.z, ar.w}, acci[4] = {ai.x, ai.y, ai.z, ai.w};
      for (int cc = 0; cc < ncur; ++cc) {
        const float2 c = Cc[(size_t)k * nc + cc];
        const float2* bcol = Bc + (size_t)len * cc + e0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (e0 + j < len) {
            const float2 b = bcol[j];
            accr[j] = fmaf(c.x, b.x, fmaf(-c.y, b.y, accr[j]));
            acci[j] = fmaf(c.x, b.y, fmaf(c.y, b.x, acci[j]));
          }
        }
      }
      *reinterpret_cast<float4*>(wr) = make_float4(accr[0], accr[1], accr[2], accr[3]);
      *reinterpret_cast<float4*>(wi) = make_float4(acci[0], acci[1], acci[2], acci[3]);
    }
    __syncthreads();
  }
}

// ---- block form of a block round.  The rotations of a block round (the local rounds below)
// act on the CTA's nl = 2 bs local vectors X (columns of a len x nl matrix) only through their
// inner products, so they can run on the Gram G = X^H X instead: a rotation J of pair (p, q),
// computed from G_pp, G_qq, G_pq exactly as from the vectors, updates G <- J^H G J (columns p,
// q, then rows p, q) and accumulates W <- W J; after the round X <- X W.  In exact arithmetic
// this is the same rotation sequence as the pairwise form (the same sweeps to converge); the
// len-long vector work becomes one Gram product and one rotation product per block round.
struct BlockSmem {
  float* gr;     // G, nl x nlp, real part
  float* gi;
  float* wr;     // W, nl x nlp
  float* wi;
  float4* prm;   // per pair slot: (cs - 1, Re k, Im k, 1 if rotated)
  int2* idx;     // per pair slot: (p, q)
  int nlp;
};

__device__ __forceinline__ BlockSmem block_carve(unsigned char* smem_raw, const SliceShape& sh) {
  const size_t nl = 2 * (size_t)sh.bs, kc = (size_t)sh.kcap;
  const size_t base = 2 * nl * sh.rowp * sizeof(float) + (size_t)sh.len * sh.nc * sizeof(float2) +
                      kc * sh.nc * sizeof(float2) + nl * sizeof(float) +
                      kc * (sizeof(float) + sizeof(int));
  float* f = reinterpret_cast<float*>(smem_raw + (base + 15) / 16 * 16);
  BlockSmem b;
  b.nlp = sh.nlp;
  const size_t m = nl * sh.nlp;
  b.gr = f;
  b.gi = f + m;
  b.wr = f + 2 * m;
  b.wi = f + 3 * m;
  b.prm = reinterpret_cast<float4*>(f + 4 * m);   // 4 m is a multiple of 4 (nl even)
  b.idx = reinterpret_cast<int2*>(b.prm + sh.bs);
  return b;
}

// G = X^H X over the first 4 len4 entries of the nl local rows (zero past the vector), and
// W = I.  Upper-triangle tiles of 4 x 4 entries, each summed by S consecutive lanes over
// interleaved 4-entry chunks and reduced with shuffles (a fixed order: deterministic).
__device__ void block_gram(const float* __restrict__ Xr, const float* __restrict__ Xi, int rowp,
                           int len4, int nl, const BlockSmem& b) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int nlp = b.nlp;
  for (int e = tid; e < nl * nlp; e += nthr) {
    const int i = e / nlp, j = e % nlp;
    b.wr[e] = i == j ? 1.f : 0.f;
    b.wi[e] = 0.f;
  }
  const int nb4 = (nl + 3) / 4;
  const int ntile = nb4 * (nb4 + 1) / 2;
  int S = 1;
  while (S < 32 && 2 * S * ntile <= nthr) S *= 2;
  const int part = tid % S, grp = tid / S, ngrp = nthr / S;
  const int ntrip = (ntile + ngrp - 1) / ngrp;
  for (int trip = 0; trip < ntrip; ++trip) {
    const int tile = grp + trip * ngrp;
    const bool live = grp < ngrp && tile < ntile;
    int pb = 0, qb = 0;
    if (live) {   // tile -> (pb <= qb), row pb holding nb4 - pb tiles
      int t = tile;
      while (t >= nb4 - pb) {
        t -= nb4 - pb;
        ++pb;
      }
      qb = pb + t;
    }
    float ar[4][4], ai[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) ar[a][c] = ai[a][c] = 0.f;
    if (live) {
      for (int ch = part; ch < len4; ch += S) {
        float4 qr[4], qi[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int q = 4 * qb + c;
          const bool ok = q < nl;
          qr[c] = ok ? *reinterpret_cast<const float4*>(Xr + (size_t)q * rowp + 4 * ch)
                     : make_float4(0.f, 0.f, 0.f, 0.f);
          qi[c] = ok ? *reinterpret_cast<const float4*>(Xi + (size_t)q * rowp + 4 * ch)
                     : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const int p = 4 * pb + a;
          if (p >= nl) break;
          const float4 pr = *reinterpret_cast<const float4*>(Xr + (size_t)p * rowp + 4 * ch);
          const float4 pi = *reinterpret_cast<const float4*>(Xi + (size_t)p * rowp + 4 * ch);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            // conj(x_p) . x_q
            float sr = ar[a][c], si = ai[a][c];
            sr = fmaf(pr.x, qr[c].x, fmaf(pi.x, qi[c].x, sr));
            si = fmaf(pr.x, qi[c].x, fmaf(-pi.x, qr[c].x, si));
            sr = fmaf(pr.y, qr[c].y, fmaf(pi.y, qi[c].y, sr));
            si = fmaf(pr.y, qi[c].y, fmaf(-pi.y, qr[c].y, si));
            sr = fmaf(pr.z, qr[c].z, fmaf(pi.z, qi[c].z, sr));
            si = fmaf(pr.z, qi[c].z, fmaf(-pi.z, qr[c].z, si));
            sr = fmaf(pr.w, qr[c].w, fmaf(pi.w, qi[c].w, sr));
            si = fmaf(pr.w, qi[c].w, fmaf(-pi.w, qr[c].w, si));
            ar[a][c] = sr;
            ai[a][c] = si;
          }
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      if (o >= S) continue;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          ar[a][c] += __shfl_xor_sync(0xffffffffu, ar[a][c], o);
          ai[a][c] += __shfl_xor_sync(0xffffffffu, ai[a][c], o);
        }
    }
    if (live && part == 0) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int p = 4 * pb + a, q = 4 * qb + c;
          if (p < nl && q < nl && (pb < qb || p <= q)) {
            b.gr[(size_t)p * nlp + q] = ar[a][c];
            b.gi[(size_t)p * nlp + q] = ai[a][c];
            b.gr[(size_t)q * nlp + p] = ar[a][c];
            b.gi[(size_t)q * nlp + p] = -ai[a][c];
          }
        }
    }
  }
}

// The local rounds of block round r on G (and W): per local round, the rotation of every pair
// slot from the current G, then the column updates of G and W, then the row updates of G.
// Returns the rotation flags of the slots this thread computed (see pair_rotation).
__device__ int block_inner(const BlockSmem& b, const SliceShape& sh, int r, int bx, int by,
                           float tol2, float floor2, float big2) {
  const int bs = sh.bs, nl = 2 * bs, nlp = b.nlp;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int nlr = r == 0 ? nl - 1 : bs;
  int flags = 0;
  for (int lr = 0; lr < nlr; ++lr) {
    for (int slot = tid; slot < bs; slot += nthr) {
      int pp, qq;
      local_pair(r, lr, slot, nl, bs, pp, qq);
      const int gp = pp < bs ? bx * bs + pp : by * bs + pp - bs;
      const int gq = qq < bs ? bx * bs + qq : by * bs + qq - bs;
      float cm = 0.f, kr = 0.f, ki = 0.f;
      int fl = 0;
      if (gp < sh.nv && gq < sh.nv)
        fl = pair_rotation(b.gr[(size_t)pp * nlp + pp], b.gr[(size_t)qq * nlp + qq],
                           b.gr[(size_t)pp * nlp + qq], b.gi[(size_t)pp * nlp + qq], tol2,
                           floor2, big2, cm, kr, ki);
      flags |= fl;
      b.prm[slot] = make_float4(cm, kr, ki, fl ? 1.f : 0.f);
      b.idx[slot] = make_int2(pp, qq);
    }
    __syncthreads();
    // columns: [a_p, a_q] <- [a_p + cm a_p - conj(k) a_q, a_q + cm a_q + k a_p] for the rows
    // of G and of W
    for (int e = tid; e < 2 * bs * nl; e += nthr) {
      const int slot = e / (2 * nl), rem = e % (2 * nl);
      const float4 pr = b.prm[slot];
      if (pr.w == 0.f) continue;
      const int2 pq = b.idx[slot];
      const bool onw = rem >= nl;
      const int i = onw ? rem - nl : rem;
      float* mr = onw ? b.wr : b.gr;
      float* mi = onw ? b.wi : b.gi;
      const size_t op = (size_t)i * nlp + pq.x, oq = (size_t)i * nlp + pq.y;
      const float xr = mr[op], xi = mi[op], yr = mr[oq], yi = mi[oq];
      mr[op] = fmaf(-pr.z, yi, fmaf(-pr.y, yr, fmaf(pr.x, xr, xr)));
      mi[op] = fmaf(pr.z, yr, fmaf(-pr.y, yi, fmaf(pr.x, xi, xi)));
      mr[oq] = fmaf(-pr.z, xi, fmaf(pr.y, xr, fmaf(pr.x, yr, yr)));
      mi[oq] = fmaf(pr.z, xr, fmaf(pr.y, xi, fmaf(pr.x, yi, yi)));
    }
    __syncthreads();
    // rows of G: [g_p, g_q] <- [g_p + cm g_p - k g_q, g_q + cm g_q + conj(k) g_p]
    for (int e = tid; e < bs * nl; e += nthr) {
      const int slot = e / nl, j = e % nl;
      const float4 pr = b.prm[slot];
      if (pr.w == 0.f) continue;
      const int2 pq = b.idx[slot];
      const size_t op = (size_t)pq.x * nlp + j, oq = (size_t)pq.y * nlp + j;
      const float xr = b.gr[op], xi = b.gi[op], yr = b.gr[oq], yi = b.gi[oq];
      b.gr[op] = fmaf(pr.z, yi, fmaf(-pr.y, yr, fmaf(pr.x, xr, xr)));
      b.gi[op] = fmaf(-pr.z, yr, fmaf(-pr.y, yi, fmaf(pr.x, xi, xi)));
      b.gr[oq] = fmaf(pr.z, xi, fmaf(pr.y, xr, fmaf(pr.x, yr, yr)));
      b.gi[oq] = fmaf(-pr.z, xr, fmaf(pr.y, xi, fmaf(pr.x, yi, yi)));
    }
    __syncthreads();
  }
  return flags;
}

// X <- X W on the nl local rows (all rowp4 4-float chunks of each row: the vector and, in the
// V form, its V entries), in place: entry e of the new row j is sum_i X(e, i) W(i, j), so each
// chunk of entries is independent; a warp computes the chunks it owns for every j into
// registers (lanes = chunks x 4-column blocks of W) and stores them after a warp barrier.
__device__ void block_update(float* __restrict__ Xr, float* __restrict__ Xi, int rowp, int rowp4,
                             int nl, const BlockSmem& b) {
  const int nlp = b.nlp;
  const int jbs = (nl + 3) / 4;      // <= 32
  const int ech = 32 / jbs;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int lj = lane % jbs, le = lane / jbs;
  for (int c0 = warp * ech; c0 < rowp4; c0 += nwarps * ech) {
    const int ch = c0 + le;
    const bool live = le < ech && ch < rowp4;
    float accr[4][4], acci[4][4];
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
      for (int c = 0; c < 4; ++c) accr[e][c] = acci[e][c] = 0.f;
    if (live) {
      for (int i = 0; i < nl; ++i) {
        const float4 xr = *reinterpret_cast<const float4*>(Xr + (size_t)i * rowp + 4 * ch);
        const float4 xi = *reinterpret_cast<const float4*>(Xi + (size_t)i * rowp + 4 * ch);
        const float xre[4] = {xr.x, xr.y, xr.z, xr.w}, xie[4] = {xi.x, xi.y, xi.z, xi.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int j = 4 * lj + c;
          const float wr = j < nl ? b.wr[(size_t)i * nlp + j] : 0.f;
          const float wi = j < nl ? b.wi[(size_t)i * nlp + j] : 0.f;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            accr[e][c] = fmaf(xre[e], wr, fmaf(-xie[e], wi, accr[e][c]));
            acci[e][c] = fmaf(xre[e], wi, fmaf(xie[e], wr, acci[e][c]));
          }
        }
      }
    }
    __syncwarp();
    if (live) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = 4 * lj + c;
        if (j < nl) {
          *reinterpret_cast<float4*>(Xr + (size_t)j * rowp + 4 * ch) =
              make_float4(accr[0][c], accr[1][c], accr[2][c], accr[3][c]);
          *reinterpret_cast<float4*>(Xi + (size_t)j * rowp + 4 * ch) =
              make_float4(acci[0][c], acci[1][c], acci[2][c], acci[3][c]);
        }
      }
    }
    __syncwarp();
  }
}

// The SVT of slice ordinal `so` of a launch (the slice index is a.slices[so]) by the C = sh.C
// CTAs of a cluster (this CTA is cluster rank `crank`; C = 1: this CTA alone), with the
// cluster's block-exchange buffer xbuf (C > 1) and the CTA's dynamic shared memory smem_raw.
// With a.prerot (V form, a.vin set) the initial vectors are B V / V^T B computed from the
// slice B = a.ahat itself (load_blocks_rotated) rather than read from a pre-rotated input.
template <int G, int CPL, int NP>
__device__ void svt_slice(const SliceArgs& a, const SliceShape& sh, int so, int crank,
                          float* xbuf, unsigned char* smem_raw, SliceShared& ss) {
  const int len = sh.len, ld = sh.ld, rowp = sh.rowp, nc = sh.nc, bs = sh.bs, nb = sh.nb;
  const int C = sh.C;
  const int nl = 2 * bs;
  float* Wr = reinterpret_cast<float*>(smem_raw);
  float* Wi = Wr + (size_t)nl * rowp;
  float2* Bc = reinterpret_cast<float2*>(Wi + (size_t)nl * rowp);
  float2* Cc = Bc + (size_t)len * nc;
  float* sig = reinterpret_cast<float*>(Cc + (size_t)sh.kcap * nc);
  float* dsc = sig + nl;
  int* keep = reinterpret_cast<int*>(dsc + sh.kcap);
  int* s_flag = ss.flag;
  int& s_rank = ss.rank;
  double& s_nuc = ss.nuc;

  cg::cluster_group cluster = cg::this_cluster();
  const int s = a.slices ? a.slices[so] : so;
  const int n1 = a.n1;
  const int64_t N12 = a.N12;
  const float2* __restrict__ A = a.ahat + (size_t)s * N12;
  // the slice the U-form rebuild reads, and which rebuild runs
  const float2* __restrict__ Ab = a.brb ? a.brb + (size_t)s * N12 : A;
  const bool uform = !sh.vform || a.brb != nullptr;
  float2* __restrict__ Z = a.zhat + (size_t)s * N12;
  if (C <= 1) xbuf = nullptr;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nthr >> 5;

  // ---- initial blocks: slot 0 / slot 1 hold the blocks of circle slot `crank`, round 0
  int bx, by;
  round_robin_pair(0, crank, nb, bx, by);
  const float2* Vin = a.vin ? a.vin + (size_t)s * a.vstride : nullptr;
  if (a.prerot && Vin && sh.vform) {
    load_blocks_rotated(Wr, Wi, A, Vin, sh, n1, bx, by, Bc, Cc);
  } else {
    load_block_from_slice(Wr, Wi, A, sh, n1, bx, 0, Vin);
    load_block_from_slice(Wr, Wi, A, sh, n1, by, 1, Vin);
  }
  __syncthreads();

  // ---- Jacobi sweeps
  const BlockSmem bsm = block_carve(smem_raw, sh);
  const int gpw = 32 / G;                    // groups per warp
  const int group = warp * gpw + lane / G;   // group index in the CTA
  const int ngroups = nwarps * gpw;
  const int gl = lane % G;
  const int nchunkv = sh.ldv / 4;
  const float tol2 = a.tol * a.tol;
  // Once a sweep's rotations all have |cos| <= big, the later rotations of that sweep move
  // each pair's cosine by at most ~big^2 per rotation touching it (2 nv of them), so after
  // the sweep every cosine is below 2 nv big^2 = tol and the checking sweep is skipped.
  const float big2 = a.tol / (2.f * (float)sh.nv);
  // SVT stopping test (a.abs_stop): left unrotated, a pair with |x^H y| = g moves the rebuilt
  // slice by about g / min(||x||, ||y||) (the rebuild projects B on the kept normalised
  // vectors), so a pair also stops once that is below tol ||B||_F / nv:
  // g^2 <= floor2 min(||x||^2, ||y||^2).  The nv (nv - 1) / 2 pairs stopped this way then move
  // D_tau(B) by at most about tol ||B||_F / sqrt(2) together (summed in quadrature), whatever
  // nv is, and each stays within the relative test's worst case per pair, tol times the
  // largest vector norm (||B||_F / nv <= sigma_max / sqrt(nv)).  ||B||_F^2 (invariant under the
  // rotations) is summed per vector in a fixed order, so the test is deterministic.
  float floor2 = 0.f;
  if (a.abs_stop) {
    for (int v = warp; v < nl; v += nwarps) {
      const float* wr = Wr + (size_t)v * rowp;
      const float* wi = Wi + (size_t)v * rowp;
      float e2 = 0.f;
      for (int e = lane; e < len; e += 32) e2 += wr[e] * wr[e] + wi[e] * wi[e];
      e2 = group_sum<32>(e2);
      if (lane == 0) sig[v] = e2;
    }
    __syncthreads();
    if (tid == 0) {
      float e2 = 0.f;
      for (int v = 0; v < nl; ++v) e2 += sig[v];
      ss.energy = e2;
    }
    if (C > 1) cluster.sync();
    else __syncthreads();
    float total = 0.f;
    for (int c = 0; c < C; ++c) total += C > 1 ? *cluster.map_shared_rank(&ss.energy, c) : ss.energy;
    floor2 = tol2 * (total / ((float)sh.nv * (float)sh.nv));
  }
  const int trips = (bs + ngroups - 1) / ngroups;
  const size_t slotf = (size_t)bs * rowp;    // floats of one plane of one block
  int sweeps = 0, converged = 0, par = 0;
  for (int sw = 0; sw < a.max_sweeps; ++sw) {
    int rotated = 0;
    for (int r = 0; r < nb - 1; ++r) {
      round_robin_pair(r, crank, nb, bx, by);
      const int vx0 = bx * bs, vy0 = by * bs;
      const int nlr = sh.block ? 0 : (r == 0 ? nl - 1 : bs);   // local rounds (pairwise form)
      if (sh.block) {
        block_gram(Wr, Wi, rowp, (len + 3) / 4, nl, bsm);
        __syncthreads();
        rotated |= block_inner(bsm, sh, r, bx, by, tol2, floor2, big2);
        block_update(Wr, Wi, rowp, rowp / 4, nl, bsm);
        __syncthreads();
      }
      for (int lr = 0; lr < nlr; ++lr) {
        for (int k0 = 0; k0 < trips; k0 += NP) {
          int p[NP], q[NP];
          bool real[NP];
          bool any_real = false;
#pragma unroll
          for (int i = 0; i < NP; ++i) {
            const int slot = group + (k0 + i) * ngroups;
            int pp = nl, qq = nl;
            if (k0 + i < trips && slot < bs) local_pair(r, lr, slot, nl, bs, pp, qq);
            // a local vector is real if its global index is below nv
            bool rp = pp < nl && qq < nl;
            if (rp) {
              const int gp = pp < bs ? vx0 + pp : vy0 + pp - bs;
              const int gq = qq < bs ? vx0 + qq : vy0 + qq - bs;
              rp = gp < sh.nv && gq < sh.nv;
            }
            real[i] = rp;
            p[i] = rp ? pp : 0;
            q[i] = rp ? qq : 1;
            any_real |= rp;
          }
          // every lane of the warp takes part in the shuffles when any group has work
          if (!__ballot_sync(0xffffffffu, any_real)) continue;
          rotated |= jacobi_pairs<G, CPL, NP>(Wr, Wi, rowp, nchunkv, p, q, real, gl, tol2,
                                              floor2, big2);
        }
        __syncthreads();
      }
      const bool sweep_end = r == nb - 2;
      int local_any = 0;
      if (sweep_end)
        local_any = (__syncthreads_or(rotated & 1) ? 1 : 0) | (__syncthreads_or(rotated & 2) ? 2 : 0);
      if (C > 1) {
        // trade blocks: write both, barrier, read the next round's pair
        if (sweep_end && tid == 0) s_flag[sw & 1] = local_any;
        copy_floats4(xblock(xbuf, sh, par, bx, 0), Wr, slotf);
        copy_floats4(xblock(xbuf, sh, par, bx, 1), Wi, slotf);
        copy_floats4(xblock(xbuf, sh, par, by, 0), Wr + slotf, slotf);
        copy_floats4(xblock(xbuf, sh, par, by, 1), Wi + slotf, slotf);
        __threadfence();
        cluster.sync();
        int nbx, nby;
        round_robin_pair(sweep_end ? 0 : r + 1, crank, nb, nbx, nby);
        copy_floats4(Wr, xblock(xbuf, sh, par, nbx, 0), slotf);
        copy_floats4(Wi, xblock(xbuf, sh, par, nbx, 1), slotf);
        copy_floats4(Wr + slotf, xblock(xbuf, sh, par, nby, 0), slotf);
        copy_floats4(Wi + slotf, xblock(xbuf, sh, par, nby, 1), slotf);
        par ^= 1;
        if (sweep_end) {
          int any = 0;
          for (int c = 0; c < C; ++c) any |= *cluster.map_shared_rank(&s_flag[sw & 1], c);
          local_any = any;
        }
        __syncthreads();
      }
      if (sweep_end) {
        ++sweeps;
        // converged: nothing rotated, or only rotations too small to leave a cosine > tol
        if (!(local_any & 1) || !(local_any & 2)) converged = 1;
      }
    }
    if (converged) break;
  }
  // the blocks now held are those of round 0: (bx, by) of circle slot crank
  round_robin_pair(0, crank, nb, bx, by);

  // ---- singular values of the local vectors: sigma = ||w||
  for (int v = warp; v < nl; v += nwarps) {
    const float* wr = Wr + (size_t)v * rowp;
    const float* wi = Wi + (size_t)v * rowp;
    float acc = 0.f;
    for (int e = lane; e < len; e += 32) acc += wr[e] * wr[e] + wi[e] * wi[e];
    acc = group_sum<32>(acc);
    if (lane == 0) sig[v] = sqrtf(acc);
  }
  __syncthreads();
  if (a.vout && sh.vform) {
    // the accumulated right rotations V (columns of the local vectors), for a warm start
    float2* vo = a.vout + (size_t)s * a.vstride;
    for (int v = warp; v < nl; v += nwarps) {
      const int gv = v < bs ? bx * bs + v : by * bs + v - bs;
      if (gv >= sh.nv) continue;
      const float* vr = Wr + (size_t)v * rowp + ld;
      const float* vi = Wi + (size_t)v * rowp + ld;
      for (int i = lane; i < sh.nv; i += 32)
        vo[(size_t)i + (size_t)sh.nv * gv] = make_float2(vr[i], vi[i]);
    }
  }
  if (a.wout) {
    // the converged vectors (and their norms) for callers that continue from them
    const float si = a.wout_conj ? -1.f : 1.f;
    float2* wo = a.wout + (size_t)s * a.wout_stride;
    for (int v = warp; v < nl; v += nwarps) {
      const int gv = v < bs ? bx * bs + v : by * bs + v - bs;
      if (gv >= sh.nv) continue;
      const float* wr = Wr + (size_t)v * rowp;
      const float* wi = Wi + (size_t)v * rowp;
      for (int e = lane; e < len; e += 32)
        wo[(size_t)e + (size_t)len * gv] = make_float2(wr[e], si * wi[e]);
      if (lane == 0 && a.sigout) a.sigout[(size_t)s * a.sig_stride + gv] = sig[v];
    }
  }
  const float tau = a.tau;
  if (tid == 0) {
    int r = 0;
    double nuc = 0.0;
    for (int v = 0; v < nl; ++v) {
      const int gv = v < bs ? bx * bs + v : by * bs + v - bs;
      if (gv >= sh.nv) continue;
      nuc += (double)sig[v];
      if (sig[v] > tau) {
        keep[r++] = v;
        dsc[v] = (sig[v] - tau) / sig[v];
      }
    }
    s_rank = r;
    s_nuc = nuc;
  }
  if (C > 1) cluster.sync();
  else __syncthreads();
  if (crank == 0 && tid == 0) {
    int rank_all = 0;
    double nuc_all = 0.0;
    for (int c = 0; c < C; ++c) {
      rank_all += C > 1 ? *cluster.map_shared_rank(&s_rank, c) : s_rank;
      nuc_all += C > 1 ? *cluster.map_shared_rank(&s_nuc, c) : s_nuc;
    }
    if (a.stat) {
      SliceStat st;
      st.rank = rank_all;
      st.sweeps = sweeps;
      st.converged = converged;
      st.pad = 0;
      st.nuc = nuc_all;
      a.stat[s] = st;
    }
    if (a.acc) {
      atomicAdd(&a.acc->total_sweeps, (unsigned long long)sweeps);
      if (!converged) atomicAdd(&a.acc->nonconverged, 1ull);
      atomicMax(&a.acc->max_sweeps, sweeps);
    }
  }
  // ---- rebuild.  One CTA: its kept vectors, all columns.  A cluster: every CTA exports its
  // kept vectors (U form: u = w / sigma; V form: w with its V entries) and shrink factors to
  // the exchange buffer, idle after the sweeps, in cluster-rank order; then each CTA
  // rebuilds the columns [col0, col1) of D_tau(B) from all kept vectors, imported nl at a
  // time, so no CTA writes a partial slice.
  const int rank_loc = s_rank;
  int off = 0, rank_all = rank_loc;
  if (C > 1) {
    rank_all = 0;
    for (int c = 0; c < C; ++c) {
      const int rc = *cluster.map_shared_rank(&s_rank, c);
      if (c < crank) off += rc;
      rank_all += rc;
    }
  }
  if (uform) {
    // ---- U form: normalise the kept vectors, u = w / sigma
    for (int64_t idx = tid; idx < (int64_t)rank_loc * len; idx += nthr) {
      const int k = (int)(idx / len), e = (int)(idx % len);
      const int v = keep[k];
      const float inv = 1.f / sig[v];
      Wr[(size_t)v * rowp + e] *= inv;
      Wi[(size_t)v * rowp + e] *= inv;
    }
    __syncthreads();
  }
  const int nv = sh.nv;
  const int col0 = C > 1 ? (int)((int64_t)nv * crank / C) : 0;
  const int col1 = C > 1 ? (int)((int64_t)nv * (crank + 1) / C) : nv;
  // exported rows: [kept index][plane][rowp] floats, then the shrink factors
  const int xw = uform ? ld : rowp;          // floats of a row the rebuild reads
  float* xd = xbuf ? xbuf + (size_t)2 * nv * rowp : nullptr;
  if (C > 1) {
    for (int k = warp; k < rank_loc; k += nwarps) {
      const int v = keep[k];
      float* dr = xbuf + (size_t)2 * (off + k) * rowp;
      for (int e = lane * 4; e < xw; e += 128) {
        *reinterpret_cast<float4*>(dr + e) = *reinterpret_cast<const float4*>(Wr + (size_t)v * rowp + e);
        *reinterpret_cast<float4*>(dr + rowp + e) =
            *reinterpret_cast<const float4*>(Wi + (size_t)v * rowp + e);
      }
      if (lane == 0) xd[off + k] = dsc[v];
    }
    __threadfence();
    cluster.sync();
  }
  if (rank_all == 0) {
    for (int64_t idx = tid; idx < (int64_t)len * (col1 - col0); idx += nthr) {
      const int p = (int)(idx % len), col = col0 + (int)(idx / len);
      Z[b_index(sh, n1, p, col)] = make_float2(0.f, 0.f);
    }
  }
  // kept rows in shared memory: the local rows (pitch rowp) with one CTA; imported rows with a
  // cluster, at pitch ld in the U form (only the vector part is read), kcap of them per group
  const int kpit = (C > 1 && uform) ? ld : rowp;
  const int gcap = (C > 1 && uform) ? sh.kcap : nl;
  for (int g0 = 0; g0 < rank_all; g0 += gcap) {
    const int rank = C > 1 ? min(gcap, rank_all - g0) : rank_loc;
    if (C > 1) {
      // import kept vectors g0 .. g0 + rank - 1 into local slots 0 .. rank - 1
      __syncthreads();
      for (int k = warp; k < rank; k += nwarps) {
        const float* sr = xbuf + (size_t)2 * (g0 + k) * rowp;
        for (int e = lane * 4; e < xw; e += 128) {
          *reinterpret_cast<float4*>(Wr + (size_t)k * kpit + e) = *reinterpret_cast<const float4*>(sr + e);
          *reinterpret_cast<float4*>(Wi + (size_t)k * kpit + e) =
              *reinterpret_cast<const float4*>(sr + rowp + e);
        }
        if (lane == 0) {
          keep[k] = k;
          dsc[k] = xd[g0 + k];
        }
      }
      __syncthreads();
    }
    const bool first = g0 == 0;
    // ---- D_tau(B) columns [col0, col1), a chunk of nc columns at a time
    for (int c0 = col0; c0 < col1; c0 += nc) {
      const int ncur = min(nc, col1 - c0);
      if (!uform) {
        // C(k, cc) = d_k conj(v_k(c0 + cc))
        for (int idx = tid; idx < rank * ncur; idx += nthr) {
          const int k = idx / ncur, cc = idx % ncur;
          const int v = keep[k];
          const float d = dsc[v];
          const size_t o = (size_t)v * kpit + ld + c0 + cc;
          Cc[(size_t)k * nc + cc] = make_float2(d * Wr[o], -d * Wi[o]);
        }
        __syncthreads();
      } else {
        // B chunk: Bc[p + len*cc] = B(p, c0+cc)
        for (int idx = tid; idx < len * ncur; idx += nthr) {
          int p, cc;
          if (!sh.rows) {
            p = idx % len;
            cc = idx / len;
          } else {
            cc = idx % ncur;
            p = idx / ncur;
          }
          Bc[p + (size_t)len * cc] = Ab[b_index(sh, n1, p, c0 + cc)];
        }
        __syncthreads();
        // C(k, cc) = d_k u_k^H B(:, c0+cc): one warp per kept vector, its lanes striding over
        // the entries (consecutive banks), then a butterfly sum over the warp
        {
          for (int k = warp; k < rank; k += nwarps) {
            const int v = keep[k];
            const float* ur = Wr + (size_t)v * kpit;
            const float* ui = Wi + (size_t)v * kpit;
            float accr[kNC], acci[kNC];
#pragma unroll
            for (int cc = 0; cc < kNC; ++cc) accr[cc] = acci[cc] = 0.f;
            for (int p = lane; p < len; p += 32) {
              const float xr = ur[p], xi = ui[p];
#pragma unroll
              for (int cc = 0; cc < kNC; ++cc) {
                if (cc < ncur) {
                  const float2 b = Bc[p + (size_t)len * cc];
                  accr[cc] += xr * b.x + xi * b.y;
                  acci[cc] += xr * b.y - xi * b.x;
                }
              }
            }
#pragma unroll
            for (int cc = 0; cc < kNC; ++cc) {
              accr[cc] = group_sum<32>(accr[cc]);
              acci[cc] = group_sum<32>(acci[cc]);
            }
            const float d = dsc[v];
            if (lane < ncur) {
              float cr = 0.f, ci = 0.f;
#pragma unroll
              for (int cc = 0; cc < kNC; ++cc)
                if (cc == lane) {
                  cr = accr[cc];
                  ci = acci[cc];
                }
              Cc[(size_t)k * nc + lane] = make_float2(d * cr, d * ci);
            }
          }
        }
        __syncthreads();
      }
      // Z(p, cc) = sum_k w_k(p) C(k, cc) (U form: w_k = u_k), written into the B chunk
      for (int p = tid; p < len; p += nthr) {
        float accr[kNC], acci[kNC];
#pragma unroll
        for (int cc = 0; cc < kNC; ++cc) accr[cc] = acci[cc] = 0.f;
        for (int k = 0; k < rank; ++k) {
          const int v = keep[k];
          const float xr = Wr[(size_t)v * kpit + p], xi = Wi[(size_t)v * kpit + p];
#pragma unroll
          for (int cc = 0; cc < kNC; ++cc) {
            if (cc < ncur) {
              const float2 c = Cc[(size_t)k * nc + cc];
              accr[cc] += xr * c.x - xi * c.y;
              acci[cc] += xr * c.y + xi * c.x;
            }
          }
        }
#pragma unroll
        for (int cc = 0; cc < kNC; ++cc)
          if (cc < ncur) Bc[p + (size_t)len * cc] = make_float2(accr[cc], acci[cc]);
      }
      __syncthreads();
      // later groups add to the columns the first wrote (this CTA owns them; the
      // __syncthreads between groups orders the accesses)
      for (int idx = tid; idx < len * ncur; idx += nthr) {
        int p, cc;
        if (!sh.rows) {
          p = idx % len;
          cc = idx / len;
        } else {
          cc = idx % ncur;
          p = idx / ncur;
        }
        const size_t o = b_index(sh, n1, p, c0 + cc);
        float2 zv = Bc[p + (size_t)len * cc];
        if (!first) {
          const float2 prev = Z[o];
          zv.x += prev.x;
          zv.y += prev.y;
        }
        Z[o] = zv;
      }
      __syncthreads();
    }
  }
}

template <int G, int CPL, int NP>
__global__ void __maxnreg__(max_regs_for(CPL * NP))
    jacobi_svt_kernel(SliceArgs a, SliceShape sh) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ SliceShared ss;
  const int C = sh.C;
  const int crank = C > 1 ? (int)cg::this_cluster().block_rank() : 0;
  const int so = blockIdx.x / C;     // slice ordinal in this launch
  float* xbuf = C > 1 ? reinterpret_cast<float*>(static_cast<char*>(a.scratch) +
                                                 (size_t)so * sh.xbuf_floats * sizeof(float))
                      : nullptr;
  svt_slice<G, CPL, NP>(a, sh, so, crank, xbuf, smem_raw, ss);
}

int max_optin_smem() {
  static int max_optin = -1;
  if (max_optin < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
        cudaSuccess)
      max_optin = 227 * 1024;
  }
  return max_optin;
}

// Lanes per pair and 4-entry chunks per lane for vectors of ld floats (a multiple of 4).
// `prefer` = 0 picks the narrowest group with at most 2 chunks per lane, else 16 lanes;
// `prefer` = 4, 8 or 16 asks for that group width (more chunks per lane = more independent
// work per lane, fewer lanes = fewer shuffle levels and more pairs per warp).
bool pick_group(int ld, int prefer, int& G, int& cpl) {
  const int nchunk = ld / 4;
  const int opts[6] = {1, 2, 3, 4, 6, 8};
  auto fit = [&](int g) {
    const int need = (nchunk + g - 1) / g;
    if (g == 4 && need > 2) return false;
    for (int o : opts)
      if (need <= o) {
        G = g;
        cpl = o;
        return true;
      }
    return false;
  };
  if (prefer) return fit(prefer);
  const int Gs[2] = {4, 8};
  for (int gi = 0; gi < 2; ++gi)
    if ((nchunk + Gs[gi] - 1) / Gs[gi] <= 2) return fit(Gs[gi]);
  return fit(16);
}

bool plan_with_ctas(int n1, int n2, int C, const SliceKnobs& k, SliceShape& sh, size_t& smem) {
  const int max_optin = max_optin_smem();
  sh.rows = n1 < n2 ? 1 : 0;
  sh.nv = n1 < n2 ? n1 : n2;
  sh.len = n1 < n2 ? n2 : n1;
  sh.vform = k.vform ? 1 : 0;
  sh.block = k.block ? 1 : 0;
  sh.C = C;
  sh.nb = 2 * C;
  sh.bs = (sh.nv + sh.nb - 1) / sh.nb;
  if (sh.block) {
    // block form: rows of the vector's 4-entry chunks (and its V entries), no lane layout;
    // it runs in the 16-lane, 4-chunk kernel instance (its register budget), nl <= 128
    if (2 * sh.bs > 128 || k.ppg > 1) return false;
    sh.G = 16;
    sh.cpl = 4;
    sh.np = 1;
    sh.ld = 4 * ((sh.len + 3) / 4);
    sh.ldv = sh.vform ? 4 * ((sh.nv + 3) / 4) : 0;
    sh.nlp = 2 * sh.bs + 1;
  } else {
    // lanes and chunks for the vector's own 4-entry chunks (the row pitch is made odd below;
    // sizing the chunks from an odd pitch instead padded e.g. a 128-entry vector to 192)
    if (!pick_group(4 * ((sh.len + 3) / 4), k.lanes, sh.G, sh.cpl)) return false;
    // rows padded so that the vector part is exactly G * cpl chunks and the V part a multiple
    // of G chunks: every lane's chunks lie inside the row and the rotation needs no tests
    sh.ld = 4 * sh.G * sh.cpl;
    sh.ldv = sh.vform ? 4 * (((sh.nv + 3) / 4 + sh.G - 1) / sh.G * sh.G) : 0;
    sh.np = k.ppg == 2 ? 2 : 1;
    if (k.ppg != 0 && k.ppg != 1 && k.ppg != 2) return false;
    if (sh.np == 2 && (sh.G == 4 || sh.cpl > 4)) return false;   // register budget
    if (sh.G == 32 && (sh.np == 2 || sh.cpl > 4)) return false;   // no such kernel instances
    sh.nlp = 0;
  }
  sh.rowp = sh.ld + sh.ldv;
  if (((sh.rowp / 4) & 1) == 0) sh.rowp += 4;   // pitch / 4 odd
  sh.kcap = C > 1 ? 2 * sh.bs * sh.rowp / sh.ld : 2 * sh.bs;
  sh.xbuf_floats = C > 1 ? (size_t)2 * sh.nb * 2 * sh.bs * sh.rowp : 0;
  for (int nc = kNC; nc >= 1; nc >>= 1) {
    sh.nc = nc;
    smem = slice_smem_bytes(sh);
    if (smem + kStaticSmemReserve <= (size_t)max_optin) return true;
  }
  return false;
}

// CTAs per slice: the fewest waves of one CTA per SM, weighted by the work of one CTA
// (1/C), without blocks thinner than kMinBlock vectors; the smallest C on ties.  k.ctas = -1:
// the fewest CTAs that hold the slice (for launches that share the GPU with others).
bool plan_slice(int n1, int n2, int nslices, const SliceKnobs& k, SliceShape& sh,
                size_t& smem) {
  const int nv = n1 < n2 ? n1 : n2;
  const int cands[4] = {1, 2, 4, 8};
  if (k.ctas == -1) {
    SliceKnobs k1 = k;
    for (int C : cands) {
      k1.ctas = C;
      if (plan_with_ctas(n1, n2, C, k1, sh, smem)) return true;
    }
    return false;
  }
  const int force = k.ctas;
  double best = 1e300;
  bool found = false;
  for (int C : cands) {
    if (force && C != force) continue;
    if (!force && C > 1 && nv < 2 * C * kMinBlock) continue;
    SliceShape t;
    size_t sm;
    if (!plan_with_ctas(n1, n2, C, k, t, sm)) continue;
    const int sms = device_sm_count();
    const int waves = (nslices * C + sms - 1) / sms;
    const double cost = (double)waves / C;
    if (cost < best - 1e-12) {
      best = cost;
      sh = t;
      smem = sm;
      found = true;
    }
  }
  if (!found && !force) {
    // slices too large for the thin-block rule: take the smallest C that fits
    for (int C : cands) {
      SliceShape t;
      size_t sm;
      if (plan_with_ctas(n1, n2, C, k, t, sm)) {
        sh = t;
        smem = sm;
        return true;
      }
    }
  }
  return found;
}

size_t scratch_for(const SliceShape& sh, int64_t N12, int nslices) {
  (void)N12;
  if (sh.C <= 1) return 0;
  return (size_t)nslices * sh.xbuf_floats * sizeof(float);
}

template <int G, int CPL, int NP>
cudaError_t launch_gc(const SliceArgs& a, const SliceShape& sh, size_t smem, int threads,
                      cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(jacobi_svt_kernel<G, CPL, NP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // the register budget can allow fewer threads than the warp cap: the kernel takes any
  // multiple of 32 (it runs a local round's pairs in as many trips as its groups need)
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, jacobi_svt_kernel<G, CPL, NP>);
  if (e != cudaSuccess) return e;
  if (threads > fa.maxThreadsPerBlock) threads = fa.maxThreadsPerBlock / 32 * 32;
  if (threads < 32) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.nslices * sh.C), 1, 1);
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)sh.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, jacobi_svt_kernel<G, CPL, NP>, a, sh);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------------------------
// Persistent batched launch.  One launch per ADMM iteration runs, for every tensor of a batch,
// the slice SVTs of that iteration (Lemma of Sec. 4.1 per Fourier slice; the slices of all
// tensors are independent, eq. shrink2) and then the fused tube pass that follows them
// (completion: eq. proj and the dual update of Sec. 4; RPCA: eq. sparse / sparse2 and eq.
// dual of Sec. 5).  Work is taken from device queues:
//   1. cluster items: (tensor, slice) pairs of the tensors planned with C CTAs per slice, in
//      decreasing cost; crank 0 of a cluster takes the next one and shares it over DSMEM;
//   2. CTA items: slices of the small tensors planned with one CTA per slice, in decreasing
//      cost, taken by each CTA once the cluster items are gone;
//   3. tube tiles: (tensor, 32 tubes) in the order in which the tensors' slices finish.
// A tube tile of tensor t starts when t's slices of this iteration are all written: a per-tensor
// counter, raised after each slice, is waited on with a bounded wait (globaltimer, 2 s) that
// sets an error word instead of hanging.  Only taken items are waited on, and a taken item is
// held by a running CTA, so the waits always end.
// ---------------------------------------------------------------------------------------------
constexpr int kBatchG = 16;                               // lanes per vector pair
constexpr unsigned long long kBatchWaitNs = 2000000000ull; // bounded wait of a tube tile

struct BatchDesc {
  BatchTensor t;
  SliceShape sh;   // slice-SVT plan (sh.C = 1: CTA items, else cluster items)
  int rm;          // tube tile rows per thread (2, 4, 8)
  int pad;
};

struct BatchLaunch {
  const BatchDesc* desc;
  const int2* big;
  const int2* small;
  const int* tile_start;    // n + 1 prefix of tiles, in tile order
  const int* tile_tensor;   // tensor at each tile-order position
  int n, nbig, nsmall, ntiles;
  BatchIter it;
  float* xbuf;
  size_t xbuf_floats;
  int C;
};

__device__ __forceinline__ unsigned long long batch_clock() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned batch_ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Bounded wait (one thread): until *p >= target, polling with a short sleep; gives up after
// limit_ns of globaltimer time and returns false.  The persistent kernel's only wait.
__device__ bool wait_counter_geq(const unsigned* p, unsigned target, unsigned long long limit_ns) {
  const unsigned long long t0 = batch_clock();
  while (batch_ld_acquire(p) < target) {
    if (batch_clock() - t0 > limit_ns) return false;
    __nanosleep(256);
  }
  return true;
}

// The bounded wait on a counter nothing raises (tsvd_selftest_bounded_wait): must give up.
__global__ void wait_selftest_kernel(const unsigned* counter, unsigned long long limit_ns, int* err) {
  if (threadIdx.x == 0 && !wait_counter_geq(counter, 1u, limit_ns)) atomicExch(err, 1);
}

__device__ SliceArgs batch_slice_args(const BatchDesc& d, const BatchIter& it) {
  const BatchTensor& t = d.t;
  SliceArgs a{};
  a.ahat = t.spec_a;
  a.zhat = t.spec_b;
  a.slices = t.slices;
  a.nslices = t.nslices;
  a.n1 = t.n1;
  a.n2 = t.n2;
  a.N12 = t.g.N12;
  a.tau = (float)(t.scale / it.r);
  a.tol = it.tol;
  a.max_sweeps = it.max_sweeps;
  a.stat = t.stat;
  a.acc = t.acc;
  a.abs_stop = it.abs_stop;
  if (t.warm) {
    // V form from the previous iteration's V (cold every kWarmColdEvery iterations), rebuilt
    // in the U form from B itself
    const int nv = min(t.n1, t.n2);
    a.vout = t.vwarm;
    a.vstride = (int64_t)nv * nv;
    a.brb = t.spec_a;
    if (it.k % kWarmColdEvery != 0) {
      a.vin = t.vwarm;
      a.prerot = 1;
    }
  }
  return a;
}

// The tube pass of tensor t that follows iteration it.k (it.k < 0: the first pass); false
// when the tensor has none there.
__device__ bool batch_tube_args(const BatchDesc& d, const BatchIter& it, TubeArgs& a) {
  const BatchTensor& t = d.t;
  a = TubeArgs{};
  a.g = t.g;
  a.twid_h = t.twid_h;
  a.twid_f = t.twid_f;
  a.ratio = 1.f;
  const bool complete = t.kind == 1;
  if (it.k < 0) {
    a.in = t.in;
    a.spec_out = t.spec_a;
    if (complete) {
      a.mode = TUBE_COMPLETE;
      a.state = t.state;
      a.first = 1;
      a.write_out = it.iters == 1;
      a.out0 = t.out0;
    } else {
      a.mode = TUBE_FWD;
    }
    return true;
  }
  const int k = it.k;
  if (complete) {
    if (k + 1 < it.iters) {
      a.mode = TUBE_COMPLETE;
      a.in = t.in;
      a.state = t.state;
      a.spec_in = t.spec_b;
      a.spec_out = t.spec_a;
      a.ratio = (float)(it.r / it.r_next);
      a.write_out = k + 2 == it.iters;
      a.out0 = t.out0;
      return true;
    }
    if (t.out1) {
      a.mode = TUBE_INV;
      a.spec_in = t.spec_b;
      a.out0 = t.out1;
      return true;
    }
    return false;
  }
  a.mode = TUBE_RPCA;
  a.in = t.in;
  a.state = t.state;
  a.spec_in = t.spec_b;
  a.spec_out = t.spec_a;
  a.ratio = (float)(it.r / it.r_next);
  a.kappa = (float)((double)t.lambda / it.r);
  a.first = k == 0;
  a.last = k + 1 == it.iters;
  a.out0 = t.out0;
  a.out1 = t.out1;
  a.tube_sparse = t.tube_sparse;
  return true;
}

template <int CMAX>
__device__ void batch_slice(const SliceArgs& a, const SliceShape& sh, int so, int crank,
                            float* xbuf, unsigned char* smem_raw, SliceShared& ss) {
  switch (sh.cpl) {
    case 1: svt_slice<kBatchG, 1, 1>(a, sh, so, crank, xbuf, smem_raw, ss); break;
    case 2:
      if constexpr (CMAX >= 2) svt_slice<kBatchG, 2, 1>(a, sh, so, crank, xbuf, smem_raw, ss);
      break;
    case 3:
      if constexpr (CMAX >= 3) svt_slice<kBatchG, 3, 1>(a, sh, so, crank, xbuf, smem_raw, ss);
      break;
    case 4:
      if constexpr (CMAX >= 4) svt_slice<kBatchG, 4, 1>(a, sh, so, crank, xbuf, smem_raw, ss);
      break;
    case 6:
      if constexpr (CMAX >= 6) svt_slice<kBatchG, 6, 1>(a, sh, so, crank, xbuf, smem_raw, ss);
      break;
    case 8:
      if constexpr (CMAX >= 8) svt_slice<kBatchG, 8, 1>(a, sh, so, crank, xbuf, smem_raw, ss);
      break;
    default: break;
  }
}

template <int CMAX>
__global__ void __maxnreg__(max_regs_for(CMAX)) batch_iter_kernel(BatchLaunch L) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ SliceShared ss;
  __shared__ int s_item;
  const BatchIter& it = L.it;
  const int C = L.C;
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = C > 1 ? (int)cluster.block_rank() : 0;
  float* xbuf = C > 1 ? L.xbuf + (size_t)(blockIdx.x / C) * L.xbuf_floats : nullptr;
  if (it.k >= 0) {
    // 1. cluster items (every CTA of a cluster takes the same number of turns)
    if (C > 1 && L.nbig > 0) {
      for (;;) {
        if (crank == 0 && threadIdx.x == 0) s_item = atomicAdd(&it.ctr[0], 1);
        cluster.sync();
        const int item = *cluster.map_shared_rank(&s_item, 0);
        cluster.sync();
        if (item >= L.nbig) break;
        const int2 w = L.big[item];
        const BatchDesc& d = L.desc[w.x];
        batch_slice<CMAX>(batch_slice_args(d, it), d.sh, w.y, crank, xbuf, smem_raw, ss);
        __threadfence();
        cluster.sync();   // every CTA of the cluster has written its columns of the slice
        if (crank == 0 && threadIdx.x == 0) atomicAdd(&it.done[w.x], 1u);
      }
    }
    // 2. single-CTA items
    for (;;) {
      if (threadIdx.x == 0) s_item = atomicAdd(&it.ctr[1], 1);
      __syncthreads();
      const int item = s_item;
      __syncthreads();
      if (item >= L.nsmall) break;
      const int2 w = L.small[item];
      const BatchDesc& d = L.desc[w.x];
      batch_slice<CMAX>(batch_slice_args(d, it), d.sh, w.y, 0, nullptr, smem_raw, ss);
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) atomicAdd(&it.done[w.x], 1u);
    }
    if (it.slices_only) return;
  }
  // 3. tube tiles (threads TILE_THREADS and up skip the tile work); the tile tables are
  // rebuilt only when the tensor changes
  int last_tix = -1;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(&it.ctr[2], 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= L.ntiles) break;
    int lo = 0, hi = L.n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (L.tile_start[mid] <= item) lo = mid;
      else hi = mid - 1;
    }
    const int tix = L.tile_tensor[lo];
    const BatchDesc& d = L.desc[tix];
    TubeArgs ta;
    if (!batch_tube_args(d, it, ta)) continue;
    if (it.k >= 0) {
      if (threadIdx.x == 0 &&
          !wait_counter_geq(&it.done[tix], (unsigned)(it.k + 1) * (unsigned)d.t.nslices,
                            kBatchWaitNs))
        atomicExch(it.err, 1);
      __syncthreads();
      __threadfence();
    }
    if (threadIdx.x < TILE_THREADS) {
      const int64_t t0 = (int64_t)(item - L.tile_start[lo]) * TT;
      const bool build = tix != last_tix;
      switch (d.rm) {
        case 2: tube_tile_body<2>(ta, t0, smem_raw, build); break;
        case 4: tube_tile_body<4>(ta, t0, smem_raw, build); break;
        default: tube_tile_body<8>(ta, t0, smem_raw, build); break;
      }
    }
    last_tix = tix;
  }
}

template <int CMAX>
cudaError_t batch_occupancy(const BatchPlan& p, int* clusters) {
  cudaError_t e = cudaFuncSetAttribute(batch_iter_kernel<CMAX>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
  if (e != cudaSuccess) return e;
  if (p.C == 1) {
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_iter_kernel<CMAX>, p.threads,
                                                      p.smem);
    *clusters = per_sm * device_sm_count();
    return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(p.C * device_sm_count()), 1, 1);
  cfg.blockDim = dim3((unsigned)p.threads, 1, 1);
  cfg.dynamicSmemBytes = p.smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)p.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaOccupancyMaxActiveClusters(clusters, batch_iter_kernel<CMAX>, &cfg);
}

template <int CMAX>
cudaError_t batch_launch(const BatchPlan& p, const BatchLaunch& L, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(batch_iter_kernel<CMAX>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)p.grid, 1, 1);
  cfg.blockDim = dim3((unsigned)p.threads, 1, 1);
  cfg.dynamicSmemBytes = p.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)p.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, batch_iter_kernel<CMAX>, L);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

size_t align16(size_t x) { return (x + 15) / 16 * 16; }
}  // namespace

bool jacobi_svt_supported(int n1, int n2) {
  SliceShape sh;
  size_t smem;
  const SliceKnobs k = {0, 0, 0, 0};
  return n1 >= 1 && n2 >= 1 && plan_slice(n1, n2, 1, k, sh, smem);
}

bool jacobi_svt_plan_ok(int n1, int n2, int nslices, const SliceKnobs& k) {
  SliceShape sh;
  size_t smem;
  return n1 >= 1 && n2 >= 1 && plan_slice(n1, n2, nslices, k, sh, smem);
}

size_t jacobi_svt_scratch_bytes(int n1, int n2, int nslices, const SliceKnobs& k) {
  SliceShape sh;
  size_t smem;
  if (!plan_slice(n1, n2, nslices, k, sh, smem)) return 0;
  return scratch_for(sh, (int64_t)n1 * n2, nslices);
}

int jacobi_svt_ctas_per_slice(int n1, int n2, int nslices, const SliceKnobs& k) {
  SliceShape sh;
  size_t smem;
  if (!plan_slice(n1, n2, nslices, k, sh, smem)) return 0;
  return sh.C;
}

cudaError_t launch_jacobi_svt(const SliceArgs& a, cudaStream_t st) {
  if (a.nslices <= 0) return cudaSuccess;
  SliceShape sh;
  size_t smem;
  if (!plan_slice(a.n1, a.n2, a.nslices, a.knobs, sh, smem)) return cudaErrorInvalidValue;
  if (sh.C > 1 && (a.scratch == nullptr || a.scratch_bytes < scratch_for(sh, a.N12, a.nslices)))
    return cudaErrorInvalidValue;
  if (a.wout && a.wout_stride < (int64_t)a.n1 * a.n2) return cudaErrorInvalidValue;
  if ((a.vin || a.vout) && (!sh.vform || a.vstride < (int64_t)sh.nv * sh.nv))
    return cudaErrorInvalidValue;
  const int gpw = 32 / sh.G;
  const int per_warp = gpw * sh.np;           // pairs a warp has in flight
  const int maxw = max_warps_for(sh.cpl * sh.np);
  // enough groups for all pairs of a local round in as few passes as fit, balanced
  const int passes = (sh.bs + maxw * per_warp - 1) / (maxw * per_warp);
  int nwarps = (sh.bs + passes * per_warp - 1) / (passes * per_warp);
  // block form: a warp per 4 local vectors (the Gram tiles and update chunks spread over them)
  if (sh.block) nwarps = (2 * sh.bs + 3) / 4;
  if (nwarps < kMinWarps) nwarps = kMinWarps;
  if (nwarps > maxw) nwarps = maxw;
  const int threads = nwarps * 32;
#define TSVD_CASE(G_, C_, N_) \
  if (sh.G == G_ && sh.cpl == C_ && sh.np == N_) \
    return launch_gc<G_, C_, N_>(a, sh, smem, threads, st);
  TSVD_CASE(4, 1, 1) TSVD_CASE(4, 2, 1) TSVD_CASE(8, 1, 1) TSVD_CASE(8, 2, 1)
  TSVD_CASE(8, 3, 1) TSVD_CASE(8, 4, 1) TSVD_CASE(8, 6, 1) TSVD_CASE(8, 8, 1)
  TSVD_CASE(16, 1, 1) TSVD_CASE(16, 2, 1) TSVD_CASE(16, 3, 1) TSVD_CASE(16, 4, 1)
  TSVD_CASE(16, 6, 1) TSVD_CASE(16, 8, 1)
  TSVD_CASE(32, 1, 1) TSVD_CASE(32, 2, 1) TSVD_CASE(32, 3, 1) TSVD_CASE(32, 4, 1)
  TSVD_CASE(8, 1, 2) TSVD_CASE(8, 2, 2) TSVD_CASE(8, 3, 2) TSVD_CASE(8, 4, 2)
  TSVD_CASE(16, 1, 2) TSVD_CASE(16, 2, 2) TSVD_CASE(16, 3, 2) TSVD_CASE(16, 4, 2)
#undef TSVD_CASE
  return cudaErrorInvalidValue;
}


bool batch_plan(const BatchTensor* ts, int n, int C, int small_nv, BatchPlan& plan,
                std::vector<unsigned char>& table) {
  if (n <= 0 || (C != 1 && C != 2 && C != 4 && C != 8)) return false;
  plan = BatchPlan{};
  plan.C = C;
  plan.small_nv = small_nv < 0 ? 2 * C * kMinBlock : small_nv;
  plan.ntensors = n;
  std::vector<BatchDesc> desc((size_t)n);
  size_t smem = 0;
  int cmax = 1;
  for (int i = 0; i < n; ++i) {
    const BatchTensor& t = ts[i];
    BatchDesc& d = desc[(size_t)i];
    std::memset(&d, 0, sizeof d);
    d.t = t;
    const int nv = std::min(t.n1, t.n2);
    const SliceKnobs k1 = {1, kBatchG, 1, t.warm ? 1 : 0};
    const SliceKnobs kc = {C, kBatchG, 1, t.warm ? 1 : 0};
    size_t sm = 0;
    SliceShape sh;
    bool ok = false;
    if (C == 1 || nv < plan.small_nv) ok = plan_with_ctas(t.n1, t.n2, 1, k1, sh, sm);
    if (!ok && C > 1) ok = plan_with_ctas(t.n1, t.n2, C, kc, sh, sm);
    if (!ok || sh.G != kBatchG || sh.np != 1) return false;
    d.sh = sh;
    d.rm = tile_rm(t.g);
    if (d.rm == 0) return false;
    smem = std::max(smem, std::max(sm, tile_smem_bytes(t.g)));
    cmax = std::max(cmax, sh.cpl);
    if (sh.C > 1) plan.xbuf_floats = std::max(plan.xbuf_floats, sh.xbuf_floats);
  }
  plan.cmax = cmax <= 4 ? 4 : 8;   // (a 2-chunk instance would run at 80 registers and spill)
  plan.threads = max_warps_for(plan.cmax) * 32;
  if (plan.threads < TILE_THREADS) return false;
  plan.smem = smem;
  if (smem + kStaticSmemReserve > (size_t)max_optin_smem()) return false;
  // items in decreasing cost: m n^2 per slice, a cold start ~3x the sweeps of a warm one
  std::vector<double> cost((size_t)n);
  for (int i = 0; i < n; ++i) {
    const double m = std::max(ts[i].n1, ts[i].n2), nn = std::min(ts[i].n1, ts[i].n2);
    cost[(size_t)i] = m * nn * nn * (ts[i].warm ? 1.0 : 3.0);
  }
  std::vector<int2> big, small;
  for (int i = 0; i < n; ++i)
    for (int so = 0; so < ts[i].nslices; ++so)
      (desc[(size_t)i].sh.C > 1 ? big : small).push_back(make_int2(i, so));
  auto by_cost = [&](const int2& a, const int2& b) {
    if (cost[(size_t)a.x] != cost[(size_t)b.x]) return cost[(size_t)a.x] > cost[(size_t)b.x];
    return a.x != b.x ? a.x < b.x : a.y < b.y;
  };
  std::sort(big.begin(), big.end(), by_cost);
  std::sort(small.begin(), small.end(), by_cost);
  plan.nbig = (int)big.size();
  plan.nsmall = (int)small.size();
  // tube tiles: tensors in the order their last slice item is taken
  std::vector<int> last((size_t)n, -1), order((size_t)n);
  for (int j = 0; j < plan.nbig; ++j) last[(size_t)big[(size_t)j].x] = j;
  for (int j = 0; j < plan.nsmall; ++j) last[(size_t)small[(size_t)j].x] = plan.nbig + j;
  for (int i = 0; i < n; ++i) order[(size_t)i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return last[(size_t)a] < last[(size_t)b]; });
  std::vector<int> tstart((size_t)n + 1, 0), ttensor((size_t)n);
  for (int j = 0; j < n; ++j) {
    const int i = order[(size_t)j];
    ttensor[(size_t)j] = i;
    tstart[(size_t)j + 1] = tstart[(size_t)j] + (int)((ts[i].g.N12 + TT - 1) / TT);
  }
  plan.ntiles = tstart[(size_t)n];
  // device table
  plan.off_desc = 0;
  plan.off_big = align16(sizeof(BatchDesc) * (size_t)n);
  plan.off_small = plan.off_big + align16(sizeof(int2) * big.size());
  plan.off_tstart = plan.off_small + align16(sizeof(int2) * small.size());
  plan.off_ttensor = plan.off_tstart + align16(sizeof(int) * ((size_t)n + 1));
  plan.table_bytes = plan.off_ttensor + align16(sizeof(int) * (size_t)n);
  table.assign(plan.table_bytes, 0);
  std::memcpy(table.data() + plan.off_desc, desc.data(), sizeof(BatchDesc) * (size_t)n);
  if (!big.empty()) std::memcpy(table.data() + plan.off_big, big.data(), sizeof(int2) * big.size());
  if (!small.empty())
    std::memcpy(table.data() + plan.off_small, small.data(), sizeof(int2) * small.size());
  std::memcpy(table.data() + plan.off_tstart, tstart.data(), sizeof(int) * ((size_t)n + 1));
  std::memcpy(table.data() + plan.off_ttensor, ttensor.data(), sizeof(int) * (size_t)n);
  // persistent grid: the clusters that fit on the device at once
  int clusters = 0;
  cudaError_t e = plan.cmax == 4 ? batch_occupancy<4>(plan, &clusters)
                                 : batch_occupancy<8>(plan, &clusters);
  if (e != cudaSuccess || clusters <= 0) {
    cudaGetLastError();
    clusters = std::max(1, device_sm_count() / C);
  }
  plan.grid = clusters * C;
  plan.scratch_bytes = C > 1 ? (size_t)clusters * plan.xbuf_floats * sizeof(float) : 0;
  return true;
}

cudaError_t launch_wait_selftest(const unsigned* counter, unsigned long long limit_ns, int* err,
                                 cudaStream_t st) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(counter, limit_ns, err);
  return cudaGetLastError();
}

cudaError_t launch_batch_iteration(const BatchPlan& p, const void* table_dev, void* scratch,
                                   const BatchIter& it, cudaStream_t st) {
  const char* tb = static_cast<const char*>(table_dev);
  BatchLaunch L;
  L.desc = reinterpret_cast<const BatchDesc*>(tb + p.off_desc);
  L.big = reinterpret_cast<const int2*>(tb + p.off_big);
  L.small = reinterpret_cast<const int2*>(tb + p.off_small);
  L.tile_start = reinterpret_cast<const int*>(tb + p.off_tstart);
  L.tile_tensor = reinterpret_cast<const int*>(tb + p.off_ttensor);
  L.n = p.ntensors;
  L.nbig = p.nbig;
  L.nsmall = p.nsmall;
  L.ntiles = p.ntiles;
  L.it = it;
  L.xbuf = static_cast<float*>(scratch);
  L.xbuf_floats = p.xbuf_floats;
  L.C = p.C;
  if (p.C > 1 && p.nbig > 0 && !scratch) return cudaErrorInvalidValue;
  if (p.cmax == 4) return batch_launch<4>(p, L, st);
  return batch_launch<8>(p, L, st);
}

}  // namespace tsvd
