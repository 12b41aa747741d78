// tube_tile.cuh -- the tile form of the tube pass (see tube_pass.cu for the fused ADMM
// steps it runs), shared by the standalone tube kernel and the persistent batched kernel.
// Device code and two small host helpers in an anonymous namespace: each translation unit
// that includes it gets its own copy.
#pragma once
#include "tsvd_internal.h"

namespace tsvd {
namespace {

// ---------------------------------------------------------------------------------------------
// Tile form (used whenever the shape fits): a CTA runs tiles of TT = 32 consecutive tubes with
// TILE_THREADS = 256 threads.  Global accesses are rows of 32 consecutive tubes (128 B real,
// 256 B complex).  The tile lives in shared memory as
//   zt[jf][jh][t]            the real tube entries (blocks of znb rows),
//   yt[jf][c][kh][t]         the half spectrum, real rows (c = 0) then imaginary rows (c = 1),
//                            blocks of q2 rows each,
// and the half-mode DFT of length nh uses the real input's symmetry.  With KR = nh/2 + 1 (rounded
// down) cosine rows and KI = nh - KR sine rows of one matrix
//   F[r][kh] = cos(2 pi r kh / nh) for r < KR,   F[r][kh] = -sin(2 pi r kh / nh) for r >= KR,
// the forward (R2C) first folds every pair of a tube, (x_j, x_nh-j) <- (x_j + x_nh-j,
// x_nh-j - x_j), and then Re X[kh] = sum_{r < KR} F[r][kh] x'_r and Im X[kh] = sum_{r >= KR}
// F[r][kh] x'_r; the inverse (C2R) forms A_r = sum_kh F[r][kh] w Re X[kh] for r < KR and
// B_r = sum_kh F[r][kh] w Im X[kh] for r >= KR (B_r = sum w Im X sin(2 pi (nh - r) kh / nh))
// and unfolds (x_j, x_nh-j) = (A_j - B_nh-j, A_j + B_nh-j).  Each transform is thus two small
// real matrix products of about nh/2 x nh/2 per tube (half the multiply-adds of the full
// cos/sin matrix), computed by tile_product on blocks zero-padded to multiples of 4, two tubes
// per packed FP32x2 FMA.  The weights w_kh = c_kh / (nf nh) (c = 1 at kh = 0 and nh/2, else 2)
// are applied when the spectrum is loaded.  The full-mode DFT of the 4-way case (length nf <=
// 8) runs in registers per (kh, tube).  The tables depend only on the tube geometry: a CTA
// builds them once and then takes tile after tile.  The fused ADMM steps are those of the
// thread-per-tube form above, on the tile in shared memory.
constexpr int TT = 32;
constexpr int TILE_THREADS = 256;
constexpr int NF_MAX = 8;

// Barrier of the TILE_THREADS threads that run a tile (named barrier 1): a CTA with more
// threads runs tiles on its first TILE_THREADS threads while the others skip them.
__device__ __forceinline__ void tile_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(TILE_THREADS) : "memory");
}

// j / nf for the mode-3 length nf <= NF_MAX without a division instruction: floor(j m / 2^16)
// with m = ceil(2^16 / nf) is exact for j < 8192 (checked for every nf <= 8), and the tile
// form's indices stay below nf nh <= 8 x 254 (tube offsets) and nf hh <= 8 x 128 (spectrum
// rows).
struct DivNf {
  unsigned m;
  int nf;
  __device__ explicit DivNf(int n) : m((65536u + (unsigned)n - 1u) / (unsigned)n), nf(n) {}
  __device__ __forceinline__ int div(int j) const { return (int)(((unsigned)j * m) >> 16); }
  __device__ __forceinline__ int mod(int j) const { return j - div(j) * nf; }
};

struct TileSmem {
  float* fre;    // [kr4][ldf]  cos rows r < KR, zero-padded (product form)
  float* fim;    // [ki4][ldf]  -sin rows r >= KR, zero-padded (product form)
  float2* tw;    // [nh] (cos, sin)(2 pi m / nh) (FFT form)
  float* zt;     // [nf][znb][TT]
  float* yt;     // [nf][2 q2][TT]
  float* nrm;    // [RS][TT] partial tube norms (RPCA tube mode)
  int ldf, kr, ki, znb, q2;
  bool fft;
};

// FFT form of the half-mode transform: for even nh >= kTileFftMinNh whose half length
// M = nh / 2 has no prime factor above 5, the R2C of a tube packs it into the complex sequence
// c_j = x_2j + i x_2j+1 of length M, transforms that with a mixed-radix Stockham FFT (radices
// 4, 2, 3, 5) and splits the result into the M + 1 stored coefficients; the C2R runs the same
// steps backwards.  Shorter tubes use the DFT products above, which measured faster there: the
// products run two tubes per packed FMA from register-blocked rows, while the FFT's stages are
// separated by barriers (128 x 128 slices: products 0.027 / 0.041 / 0.069 ms per tube pass at
// nh = 60 / 100 / 128, FFT 0.045 / 0.046 / 0.059; at nh = 200 and 250 the FFT takes 0.086 and
// 0.097 ms against 0.136 and 0.167).
constexpr int kTileFftMinNh = 128;
__host__ __device__ inline bool tile_fft_ok(const TubeGeom& g) {
  if (g.nh < kTileFftMinNh || (g.nh & 1)) return false;
  int m = g.nh / 2;
  while (m % 2 == 0) m /= 2;
  while (m % 3 == 0) m /= 3;
  while (m % 5 == 0) m /= 5;
  return m == 1;
}

__host__ __device__ inline int tile_kr(const TubeGeom& g) { return g.nh / 2 + 1; }
__host__ __device__ inline int tile_ki(const TubeGeom& g) { return g.nh - tile_kr(g); }
__host__ __device__ inline int tile_round4(int x) { return (x + 3) & ~3; }
// table row length: hh rounded up to 8 (an RM-row group of the forward product reads inside it)
__host__ __device__ inline int tile_ldf(const TubeGeom& g) { return (g.hh + 7) & ~7; }
// zt block rows: the sine product reads KI rounded up to 4 rows from row KR, up to row nh + 2
__host__ __device__ inline int tile_znb(const TubeGeom& g) { return tile_round4(g.nh + 3); }
__host__ __device__ inline int tile_q2(const TubeGeom& g) { return tile_round4(g.hh); }

__host__ __device__ inline size_t tile_table_floats(const TubeGeom& g) {
  if (tile_fft_ok(g)) return (size_t)tile_round4(2 * g.nh);
  const int ki4 = tile_round4(tile_ki(g) > 0 ? tile_ki(g) : 1);
  return (size_t)(tile_round4(tile_kr(g)) + ki4) * tile_ldf(g);
}

__host__ __device__ inline size_t tile_smem_bytes(const TubeGeom& g) {
  return (tile_table_floats(g) + (size_t)g.nf * tile_znb(g) * TT +
          (size_t)g.nf * 2 * tile_q2(g) * TT + (size_t)(TILE_THREADS / TT) * TT) *
         sizeof(float);
}

__device__ __forceinline__ TileSmem tile_carve(unsigned char* raw, const TubeGeom& g) {
  TileSmem s;
  s.ldf = tile_ldf(g);
  s.kr = tile_kr(g);
  s.ki = tile_ki(g);
  s.znb = tile_znb(g);
  s.q2 = tile_q2(g);
  s.fft = tile_fft_ok(g);
  s.fre = reinterpret_cast<float*>(raw);
  s.fim = s.fre + (size_t)tile_round4(s.kr) * s.ldf;
  s.tw = reinterpret_cast<float2*>(raw);
  s.zt = s.fre + tile_table_floats(g);
  s.yt = s.zt + (size_t)g.nf * s.znb * TT;
  s.nrm = s.yt + (size_t)g.nf * 2 * s.q2 * TT;
  return s;
}

// The tables F (from the twiddle table, exact at the quarter points: the index r kh mod nh is
// stepped by r) and the zero padding of the zt and yt blocks, which the tile steps never write.
__device__ void tile_build(const TileSmem& s, const TubeGeom& g, const float2* __restrict__ twid_h) {
  const int nh = g.nh, hh = g.hh, ldf = s.ldf;
  if (s.fft) {
    for (int m = threadIdx.x; m < nh; m += TILE_THREADS) s.tw[m] = twid_h[m];
    return;   // the FFT form reads no padding
  }
  const int rows = tile_round4(s.kr) + tile_round4(s.ki > 0 ? s.ki : 1);
  for (int r = threadIdx.x; r < rows; r += TILE_THREADS) {
    const bool cosrow = r < tile_round4(s.kr);
    const int jr = cosrow ? r : s.kr + (r - tile_round4(s.kr));   // the DFT index of the row
    const bool live = cosrow ? r < s.kr : jr < nh;
    float* row = s.fre + (size_t)r * ldf;   // fim follows fre directly
    int m = 0;
    for (int kh = 0; kh < ldf; ++kh) {
      float v = 0.f;
      if (live && kh < hh) {
        const float2 w = twid_h[m];
        v = cosrow ? w.x : -w.y;
      }
      row[kh] = v;
      m += jr;
      while (m >= nh) m -= nh;
    }
  }
  for (int f = 0; f < g.nf; ++f) {
    for (int idx = threadIdx.x; idx < (s.znb - nh) * TT; idx += TILE_THREADS)
      s.zt[((size_t)f * s.znb + nh) * TT + idx] = 0.f;
    for (int c = 0; c < 2; ++c)
      for (int idx = threadIdx.x; idx < (s.q2 - hh) * TT; idx += TILE_THREADS)
        s.yt[((size_t)f * 2 * s.q2 + (size_t)c * s.q2 + hh) * TT + idx] = 0.f;
  }
}

__device__ __forceinline__ float2 ffma2s(float a, float2 b, float2 c) {
  return __ffma2_rn(make_float2(a, a), b, c);
}

// out[r][t] = sum_{k < K} A(r, k) B[k][t] for r < M <= 16 RM and the 32 tubes of the tile; K is a
// multiple of 4 (B rows and A entries past the true extent are zero).  FWD: A(r, k) =
// fr[k * ldq + r]; otherwise A(r, k) = fr[r * ldq + k].  Rows past Fr's extent (rext: ldq for
// FWD, the row count otherwise) read a clamped, in-bounds position once and are not stored.
// Row groups rg0 .. rg0 + 15 of the 32 take part (rows (rg - rg0) RM ..), so two products run
// side by side on the two halves of the tile's threads.
template <int RM, bool FWD>
__device__ __forceinline__ void tile_product(const float* __restrict__ fr, int ldq, int rext,
                                             const float* __restrict__ b, float* __restrict__ out,
                                             int M, int K, int rg0) {
  const int tg = threadIdx.x & 7, rg = (threadIdx.x >> 3) - rg0;
  if (rg < 0 || rg >= 16) return;
  const int r0 = rg * RM;
  float2 acc[RM][2];
#pragma unroll
  for (int i = 0; i < RM; ++i) acc[i][0] = acc[i][1] = make_float2(0.f, 0.f);
  const float* bp = b + 4 * tg;
  if (FWD) {
    const float* ap = fr + min(r0, rext - RM);
    for (int k = 0; k < K; k += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 bv = *reinterpret_cast<const float4*>(bp + (size_t)(k + u) * TT);
        const float2 b01 = make_float2(bv.x, bv.y), b23 = make_float2(bv.z, bv.w);
        float av[RM];
        const float* arow = ap + (size_t)(k + u) * ldq;
        if (RM == 2) {
          const float2 v = *reinterpret_cast<const float2*>(arow);
          av[0] = v.x;
          av[RM - 1] = v.y;
        } else {
#pragma unroll
          for (int i = 0; i < RM; i += 4) {
            const float4 v = *reinterpret_cast<const float4*>(arow + i);
            av[i] = v.x;
            av[i + 1] = v.y;
            av[i + 2] = v.z;
            av[i + 3] = v.w;
          }
        }
#pragma unroll
        for (int i = 0; i < RM; ++i) {
          acc[i][0] = ffma2s(av[i], b01, acc[i][0]);
          acc[i][1] = ffma2s(av[i], b23, acc[i][1]);
        }
      }
    }
  } else {
    const float* ap[RM];
#pragma unroll
    for (int i = 0; i < RM; ++i) ap[i] = fr + (size_t)min(r0 + i, rext - 1) * ldq;
    for (int k = 0; k < K; k += 4) {
      float4 bv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) bv[u] = *reinterpret_cast<const float4*>(bp + (size_t)(k + u) * TT);
#pragma unroll
      for (int i = 0; i < RM; ++i) {
        const float4 a4 = *reinterpret_cast<const float4*>(ap[i] + k);
        const float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          acc[i][0] = ffma2s(av[u], make_float2(bv[u].x, bv[u].y), acc[i][0]);
          acc[i][1] = ffma2s(av[u], make_float2(bv[u].z, bv[u].w), acc[i][1]);
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < RM; ++i) {
    const int r = r0 + i;
    if (r < M)
      *reinterpret_cast<float4*>(out + (size_t)r * TT + 4 * tg) =
          make_float4(acc[i][0].x, acc[i][0].y, acc[i][1].x, acc[i][1].y);
  }
}

// Full-mode DFT of length nf of every (kh, tube) column of the spectrum tile, in place:
// sign +1 (inverse, no scaling) or -1 (forward).
__device__ void tile_full_dft(const TileSmem& s, const TubeGeom& g, const float2* __restrict__ twf,
                              float sign, const float2* __restrict__ fm) {
  const int nf = g.nf, hh = g.hh, q2 = s.q2;
  for (int idx = threadIdx.x; idx < hh * TT; idx += TILE_THREADS) {
    const int kh = idx / TT, t = idx % TT;
    float2 x[NF_MAX], y[NF_MAX];
    for (int f = 0; f < nf; ++f) {
      const size_t row = (size_t)f * 2 * q2 + kh;
      x[f] = make_float2(s.yt[row * TT + t], s.yt[(row + q2) * TT + t]);
    }
    for (int o = 0; o < nf; ++o) {
      float ar = 0.f, ai = 0.f;
      int m = 0;
      for (int f = 0; f < nf; ++f) {
        const float2 w = fm ? fm[(size_t)o * nf + f] : twf[m];
        const float ws = sign * w.y;
        ar += x[f].x * w.x - x[f].y * ws;
        ai += x[f].x * ws + x[f].y * w.x;
        m += o;
        if (m >= nf) m -= nf;
      }
      y[o] = make_float2(ar, ai);
    }
    for (int f = 0; f < nf; ++f) {
      const size_t row = (size_t)f * 2 * q2 + kh;
      s.yt[row * TT + t] = y[f].x;
      s.yt[(row + q2) * TT + t] = y[f].y;
    }
  }
}

// (x_j, x_nh-j) <- (x_j + x_nh-j, x_nh-j - x_j) (forward) or (x_j - x_nh-j, x_j + x_nh-j)
// (inverse) for j = 1 .. KI on every zt block.
__device__ void tile_fold(const TileSmem& s, const TubeGeom& g, bool forward) {
  const int nh = g.nh, ki = s.ki;
  for (int idx = threadIdx.x; idx < g.nf * ki * TT; idx += TILE_THREADS) {
    const int t = idx % TT, q = idx / TT;
    const int j = 1 + q % ki, f = q / ki;
    float* z = s.zt + (size_t)f * s.znb * TT + t;
    const float a = z[(size_t)j * TT], b = z[(size_t)(nh - j) * TT];
    z[(size_t)j * TT] = forward ? a + b : a - b;
    z[(size_t)(nh - j) * TT] = forward ? b - a : a + b;
  }
}

// ---- FFT form
// Each thread works on two adjacent tubes (t, t + 1) at once: a complex value of the pair is
// CP{re, im} with re = (Re x_t, Re x_t+1), im = (Im x_t, Im x_t+1), so the arithmetic runs on
// packed FP32x2 instructions and the shared-memory accesses are 8-byte rows of 16 lanes.
struct CP {
  float2 re, im;
};
__device__ __forceinline__ float2 f2s(float c) { return make_float2(c, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2s(-1.f), a); }
__device__ __forceinline__ CP cpadd(CP a, CP b) { return CP{add2(a.re, b.re), add2(a.im, b.im)}; }
__device__ __forceinline__ CP cpsub(CP a, CP b) { return CP{sub2(a.re, b.re), sub2(a.im, b.im)}; }
__device__ __forceinline__ CP cpscale(float c, CP a) {
  return CP{__fmul2_rn(a.re, f2s(c)), __fmul2_rn(a.im, f2s(c))};
}
// a w for one complex number w = (wr, wi) shared by both tubes
__device__ __forceinline__ CP cpmul(CP a, float wr, float wi) {
  return CP{__ffma2_rn(a.re, f2s(wr), __fmul2_rn(a.im, f2s(-wi))),
            __ffma2_rn(a.re, f2s(wi), __fmul2_rn(a.im, f2s(wr)))};
}
// i sg a for sg = +-1
__device__ __forceinline__ CP cpimul(float sg, CP a) {
  return CP{__fmul2_rn(a.im, f2s(-sg)), __fmul2_rn(a.re, f2s(sg))};
}
__device__ __forceinline__ CP cpconj(CP a) { return CP{a.re, __fmul2_rn(a.im, f2s(-1.f))}; }

// A complex [M][TT] buffer of every mode-3 block f of the tile: real rows at re + f * fstride,
// imaginary rows im rows further (row pitch TT); element (row, tube pair p) at 2 p.
struct FftBuf {
  float* re;
  int fstride;
  int im;
  __device__ CP get(int f, int row, int p) const {
    const float* q = re + (size_t)f * fstride + (size_t)row * TT + 2 * p;
    return CP{*reinterpret_cast<const float2*>(q), *reinterpret_cast<const float2*>(q + (size_t)im * TT)};
  }
  __device__ void put(int f, int row, int p, CP v) const {
    float* q = re + (size_t)f * fstride + (size_t)row * TT + 2 * p;
    *reinterpret_cast<float2*>(q) = v.re;
    *reinterpret_cast<float2*>(q + (size_t)im * TT) = v.im;
  }
};
// The two buffers of the FFT form: A in the spectrum block (yt), B in the real block (zt).
__device__ __forceinline__ FftBuf fft_buf_a(const TileSmem& s) {
  return FftBuf{s.yt, 2 * s.q2 * TT, s.q2};
}
__device__ __forceinline__ FftBuf fft_buf_b(const TileSmem& s, int M) {
  return FftBuf{s.zt, s.znb * TT, M};
}

constexpr int FFT_PAIRS = TT / 2;                       // tube pairs of a tile row
constexpr int FFT_GROUPS = TILE_THREADS / FFT_PAIRS;    // rows a pass works on at once

// v[m] <- sum_r v[r] e^{sg 2 pi i r m / R} (the small DFTs of the Stockham stages; radix 3 and 5
// in the symmetric form, their constants read from the table).
template <int R>
__device__ __forceinline__ void fft_butterfly(CP (&v)[R], float sg, const float2* tw, int nh) {
  static_assert(R == 2 || R == 3 || R == 4 || R == 5, "radix");
  if constexpr (R == 2) {
    const CP a = v[0], b = v[1];
    v[0] = cpadd(a, b);
    v[1] = cpsub(a, b);
  } else if constexpr (R == 4) {
    const CP s02 = cpadd(v[0], v[2]), d02 = cpsub(v[0], v[2]);
    const CP s13 = cpadd(v[1], v[3]), d13 = cpimul(sg, cpsub(v[1], v[3]));
    v[0] = cpadd(s02, s13);
    v[2] = cpsub(s02, s13);
    v[1] = cpadd(d02, d13);
    v[3] = cpsub(d02, d13);
  } else if constexpr (R == 3) {
    const float s3 = tw[nh / 3].y;   // sin(2 pi / 3)
    const CP t1 = cpadd(v[1], v[2]);
    const CP t2 = cpsub(v[0], cpscale(0.5f, t1));
    const CP t3 = cpimul(sg, cpscale(s3, cpsub(v[1], v[2])));
    v[0] = cpadd(v[0], t1);
    v[1] = cpadd(t2, t3);
    v[2] = cpsub(t2, t3);
  } else {
    const float2 w1 = tw[nh / 5], w2 = tw[2 * (nh / 5)];   // (cos, sin)(2 pi / 5), (4 pi / 5)
    const CP t1 = cpadd(v[1], v[4]), t2 = cpadd(v[2], v[3]);
    const CP t3 = cpsub(v[1], v[4]), t4 = cpsub(v[2], v[3]);
    const CP a1 = cpadd(v[0], cpadd(cpscale(w1.x, t1), cpscale(w2.x, t2)));
    const CP a2 = cpadd(v[0], cpadd(cpscale(w2.x, t1), cpscale(w1.x, t2)));
    const CP b1 = cpimul(sg, cpadd(cpscale(w1.y, t3), cpscale(w2.y, t4)));
    const CP b2 = cpimul(sg, cpsub(cpscale(w2.y, t3), cpscale(w1.y, t4)));
    v[0] = cpadd(v[0], cpadd(t1, t2));
    v[1] = cpadd(a1, b1);
    v[4] = cpsub(a1, b1);
    v[2] = cpadd(a2, b2);
    v[3] = cpsub(a2, b2);
  }
}

// One Stockham stage of radix R on every block (in -> out): Ns is the product of the earlier
// stages' radices; element j < M / R of the stage takes in[j + r M / R], turns entry r by
// e^{sg 2 pi i r k / (Ns R)} (k = j mod Ns), runs the radix-R DFT and writes
// out[(j / Ns) Ns R + k + m Ns] -- natural order after the last stage.  Thread (group g, pair
// p) takes elements q = g, g + FFT_GROUPS, ... of the nf M / R of the tile (f = q / nb,
// j = q mod nb), stepping f, j, j / Ns and j mod Ns without divisions.
template <int R>
__device__ void fft_stage(const FftBuf& in, const FftBuf& out, const float2* tw, int nh, int M,
                          int nf, int Ns, float sg) {
  const int nb = M / R;
  const int p = threadIdx.x % FFT_PAIRS;
  const int g = threadIdx.x / FFT_PAIRS;
  const int step = nh / (Ns * R);
  if (g >= nf * nb) return;
  int f = g / nb, j = g % nb;
  int jo = j / Ns, k = j % Ns;
  const int dq = FFT_GROUPS / Ns, rq = FFT_GROUPS % Ns;
  while (f < nf) {
    CP v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in.get(f, j + r * nb, p);
    if (k) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const float2 w = tw[r * k * step];
        v[r] = cpmul(v[r], w.x, sg * w.y);
      }
    }
    fft_butterfly<R>(v, sg, tw, nh);
    const int o = jo * Ns * R + k;
#pragma unroll
    for (int m = 0; m < R; ++m) out.put(f, o + m * Ns, p, v[m]);
    // next element: j += FFT_GROUPS, carrying into f
    j += FFT_GROUPS;
    if (j < nb) {
      jo += dq;
      k += rq;
      if (k >= Ns) {
        k -= Ns;
        ++jo;
      }
    } else {
      while (j >= nb) {
        j -= nb;
        ++f;
      }
      jo = j / Ns;
      k = j - jo * Ns;
    }
  }
}

// The radix of stage `stage` of a length-M transform (0 past the last stage): fours first,
// then 2, 3, 5.
__device__ __forceinline__ int fft_radix(int M, int stage) {
  int n = 0;
  for (int r = 4; r != 0; r = r == 4 ? 2 : r == 2 ? 3 : r == 3 ? 5 : 0) {
    while (M % r == 0) {
      if (n++ == stage) return r;
      M /= r;
    }
  }
  return 0;
}
__device__ __forceinline__ int fft_nstages(int M) {
  int n = 0;
  while (fft_radix(M, n)) ++n;
  return n;
}

// The Stockham stages of a length-M transform from buffer `a` (ping-ponging with `b`); returns
// true when the result ends in `b`.
__device__ bool fft_run(const TileSmem& s, const FftBuf& a, const FftBuf& b, int nh, int M,
                        int nf, float sg) {
  int Ns = 1;
  bool in_b = false;
  for (int st = 0;; ++st) {
    const int R = fft_radix(M, st);
    if (!R) break;
    const FftBuf& src = in_b ? b : a;
    const FftBuf& dst = in_b ? a : b;
    switch (R) {
      case 4: fft_stage<4>(src, dst, s.tw, nh, M, nf, Ns, sg); break;
      case 2: fft_stage<2>(src, dst, s.tw, nh, M, nf, Ns, sg); break;
      case 3: fft_stage<3>(src, dst, s.tw, nh, M, nf, Ns, sg); break;
      default: fft_stage<5>(src, dst, s.tw, nh, M, nf, Ns, sg); break;
    }
    tile_sync();
    in_b = !in_b;
    Ns *= R;
  }
  return in_b;
}

// Real tile (zt) -> spectrum tile (yt), FFT form: pack, transform, split
// X_k = E_k + e^{-2 pi i k / nh} O_k with E_k = (C_k + conj C_M-k) / 2 and
// O_k = (C_k - conj C_M-k) / 2i; one thread per pair (k, M - k), so the split may run in place.
__device__ void tile_forward_fft(const TileSmem& s, const TubeGeom& g) {
  const int nh = g.nh, M = nh / 2, nf = g.nf;
  const int p = threadIdx.x % FFT_PAIRS;
  const FftBuf A = fft_buf_a(s), B = fft_buf_b(s, M);
  for (int f = 0; f < nf; ++f) {
    const float* z = s.zt + (size_t)f * s.znb * TT + 2 * p;
    for (int j = threadIdx.x / FFT_PAIRS; j < M; j += FFT_GROUPS)
      A.put(f, j, p, CP{*reinterpret_cast<const float2*>(z + (size_t)(2 * j) * TT),
                        *reinterpret_cast<const float2*>(z + (size_t)(2 * j + 1) * TT)});
  }
  tile_sync();
  const FftBuf& C = fft_run(s, A, B, nh, M, nf, -1.f) ? B : A;
  const int np = M / 2 + 1;
  for (int f = 0; f < nf; ++f) {
    for (int k = threadIdx.x / FFT_PAIRS; k < np; k += FFT_GROUPS) {
      if (k == 0) {
        const CP c0 = C.get(f, 0, p);
        A.put(f, 0, p, CP{add2(c0.re, c0.im), f2s(0.f)});
        A.put(f, M, p, CP{sub2(c0.re, c0.im), f2s(0.f)});
        continue;
      }
      const int kk = M - k;
      const CP ck = C.get(f, k, p), cm = C.get(f, kk, p);
      const CP e = cpscale(0.5f, cpadd(ck, cpconj(cm)));
      const CP o = cpimul(-1.f, cpscale(0.5f, cpsub(ck, cpconj(cm))));   // (ck - conj cm) / 2i
      const float2 wk = s.tw[k];
      A.put(f, k, p, cpadd(e, cpmul(o, wk.x, -wk.y)));
      if (kk != k) {
        const float2 wm = s.tw[kk];
        A.put(f, kk, p, cpadd(cpconj(e), cpmul(cpconj(o), wm.x, -wm.y)));
      }
    }
  }
  tile_sync();
}

// Spectrum tile (yt, loaded with the uniform weight 1 / (nf nh)) -> real tile (zt), FFT form:
// C_k = (X_k + conj X_M-k) + i e^{2 pi i k / nh} (X_k - conj X_M-k) for k < M, the inverse
// transform, and x_2j = Re c_j, x_2j+1 = Im c_j.  The first step writes into B when the
// transform has an odd number of stages, so that it ends in A.
__device__ void tile_inverse_fft(const TileSmem& s, const TubeGeom& g) {
  const int nh = g.nh, M = nh / 2, nf = g.nf;
  const int p = threadIdx.x % FFT_PAIRS;
  const FftBuf A = fft_buf_a(s), B = fft_buf_b(s, M);
  const bool odd = fft_nstages(M) & 1;
  const FftBuf& D = odd ? B : A;
  const int np = M / 2 + 1;
  for (int f = 0; f < nf; ++f) {
    for (int k = threadIdx.x / FFT_PAIRS; k < np; k += FFT_GROUPS) {
      const int kk = M - k;
      CP xk = A.get(f, k, p), xm = A.get(f, kk, p);
      if (k == 0) xk.im = xm.im = f2s(0.f);   // a C2R reads only the real parts of X_0, X_M
      const float2 wk = s.tw[k];
      D.put(f, k, p, cpadd(cpadd(xk, cpconj(xm)), cpimul(1.f, cpmul(cpsub(xk, cpconj(xm)), wk.x, wk.y))));
      if (k != 0 && kk != k) {
        const float2 wm = s.tw[kk];
        D.put(f, kk, p,
              cpadd(cpadd(xm, cpconj(xk)), cpimul(1.f, cpmul(cpsub(xm, cpconj(xk)), wm.x, wm.y))));
      }
    }
  }
  tile_sync();
  fft_run(s, D, odd ? A : B, nh, M, nf, 1.f);   // ends in A by the choice of D
  for (int f = 0; f < nf; ++f) {
    float* z = s.zt + (size_t)f * s.znb * TT + 2 * p;
    for (int j = threadIdx.x / FFT_PAIRS; j < M; j += FFT_GROUPS) {
      const CP c = A.get(f, j, p);
      *reinterpret_cast<float2*>(z + (size_t)(2 * j) * TT) = c.re;
      *reinterpret_cast<float2*>(z + (size_t)(2 * j + 1) * TT) = c.im;
    }
  }
  tile_sync();
}

// Spectrum tile (loaded, weighted) -> real tile.
template <int RM>
__device__ void tile_inverse(const TileSmem& s, const TubeGeom& g, const float2* twf,
                             const float2* fm) {
  if (g.nf > 1) {
    tile_full_dft(s, g, twf, 1.f, fm);
    tile_sync();
  }
  if (s.fft) {
    tile_inverse_fft(s, g);
    return;
  }
  for (int f = 0; f < g.nf; ++f) {
    float* z = s.zt + (size_t)f * s.znb * TT;
    const float* y = s.yt + (size_t)f * 2 * s.q2 * TT;
    tile_product<RM, false>(s.fre, s.ldf, s.kr, y, z, s.kr, s.q2, 0);
    if (s.ki > 0)
      tile_product<RM, false>(s.fim, s.ldf, s.ki, y + (size_t)s.q2 * TT, z + (size_t)s.kr * TT,
                              s.ki, s.q2, 16);
  }
  tile_sync();
  if (s.ki > 0) {
    tile_fold(s, g, false);
    tile_sync();
  }
}

// Real tile -> spectrum tile, product form (before the mode-3 DFT).
template <int RM>
__device__ void tile_forward_products(const TileSmem& s, const TubeGeom& g) {
  if (s.ki > 0) {
    tile_fold(s, g, true);
    tile_sync();
  }
  for (int f = 0; f < g.nf; ++f) {
    const float* z = s.zt + (size_t)f * s.znb * TT;
    float* y = s.yt + (size_t)f * 2 * s.q2 * TT;
    tile_product<RM, true>(s.fre, s.ldf, s.ldf, z, y, g.hh, tile_round4(s.kr), 0);
    if (s.ki > 0) {
      tile_product<RM, true>(s.fim, s.ldf, s.ldf, z + (size_t)s.kr * TT, y + (size_t)s.q2 * TT,
                             g.hh, tile_round4(s.ki), 16);
    } else if (threadIdx.x >= TILE_THREADS / 2) {
      for (int idx = threadIdx.x - TILE_THREADS / 2; idx < g.hh * TT; idx += TILE_THREADS / 2)
        y[(size_t)s.q2 * TT + idx] = 0.f;
    }
  }
  tile_sync();
}

// Real tile -> spectrum tile.
template <int RM>
__device__ void tile_forward(const TileSmem& s, const TubeGeom& g, const float2* twf,
                             const float2* fm) {
  if (s.fft) {
    tile_forward_fft(s, g);
  } else {
    tile_forward_products<RM>(s, g);
  }
  if (g.nf > 1) {
    tile_full_dft(s, g, twf, -1.f, fm);
    tile_sync();
  }
}

// Loads the stored spectrum of the tile (conjugate partners on the self-conjugate columns)
// and applies the C2R weights: c_kh / (nf nh) for the product form (c = 1 at kh = 0 and nh/2,
// else 2), 1 / (nf nh) for the FFT form.
__device__ void tile_load_spectrum(const TileSmem& s, const TubeGeom& g,
                                   const float2* __restrict__ spec, int64_t t0,
                                   const int* __restrict__ fp) {
  const int nf = g.nf, nh = g.nh, hh = g.hh, q2 = s.q2;
  const DivNf dn(nf);
  const float inv = 1.f / (float)(nf * nh);
  const int total = nf * hh * TT;
  constexpr int U = 8;   // loads a thread keeps in flight (see the element loops)
  const int t = threadIdx.x % TT;   // TILE_THREADS is a multiple of TT
  const bool live = t0 + t < g.N12;
  for (int base = threadIdx.x; base < total; base += U * TILE_THREADS) {
    float2 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * TILE_THREADS;
      v[u] = make_float2(0.f, 0.f);
      if (idx < total && live) {
        const int q = idx / TT;
        const int kh = dn.div(q), kf = q - kh * nf;
        const bool selfcol = (kh == 0) || (2 * kh == nh);
        const int pk = fp ? fp[kf] : (kf == 0 ? 0 : nf - kf);
        // L2-only loads: in the persistent batched kernel the spectrum was written by other
        // SMs earlier in the same launch
        if (selfcol && pk < kf) {
          v[u] = __ldcg(spec + (size_t)(pk + nf * kh) * g.N12 + t0 + t);
          v[u].y = -v[u].y;
        } else {
          v[u] = __ldcg(spec + (size_t)q * g.N12 + t0 + t);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * TILE_THREADS;
      if (idx >= total) continue;
      const int q = idx / TT;
      const int kh = dn.div(q), kf = q - kh * nf;
      const bool selfcol = (kh == 0) || (2 * kh == nh);
      const float w = (selfcol || s.fft ? 1.f : 2.f) * inv;
      const size_t row = (size_t)kf * 2 * q2 + kh;
      s.yt[row * TT + t] = v[u].x * w;
      s.yt[(row + q2) * TT + t] = v[u].y * w;
    }
  }
}

__device__ void tile_store_spectrum(const TileSmem& s, const TubeGeom& g, float2* __restrict__ spec,
                                    int64_t t0) {
  const int nf = g.nf, hh = g.hh, q2 = s.q2;
  const DivNf dn(nf);
  for (int idx = threadIdx.x; idx < nf * hh * TT; idx += TILE_THREADS) {
    const int q = idx / TT, t = idx % TT;
    if (t0 + t >= g.N12) continue;
    const int kh = dn.div(q), kf = q - kh * nf;
    const size_t row = (size_t)kf * 2 * q2 + kh;
    spec[(size_t)q * g.N12 + t0 + t] = make_float2(s.yt[row * TT + t], s.yt[(row + q2) * TT + t]);
  }
}

// One tile of TT tubes starting at tube t0, run by threads 0 .. TILE_THREADS - 1 of the CTA
// (their barrier is tile_sync); smem_raw holds tile_smem_bytes(a.g) bytes.  build: (re)build
// the tables and paddings (the first tile of a CTA, or one of another geometry); a CTA that
// keeps the geometry passes false for its later tiles.
template <int RM>
__device__ void tube_tile_body(const TubeArgs& a, int64_t t0, unsigned char* smem_raw,
                               bool build = true) {
  const TubeGeom g = a.g;
  const TileSmem s = tile_carve(smem_raw, g);
  const int tid = threadIdx.x;
  const int nreal = g.nf * g.nh;
  const int64_t N12 = g.N12;
  tile_sync();   // the previous tile of this CTA is done with the shared memory
  if (build) tile_build(s, g, a.twid_h);
  const bool need_inv = a.mode == TUBE_INV || a.mode == TUBE_RPCA ||
                        (a.mode == TUBE_COMPLETE && !a.first);
  if (need_inv) tile_load_spectrum(s, g, a.spec_in, t0, a.fpart);
  tile_sync();
  if (need_inv) tile_inverse<RM>(s, g, a.twid_f, a.fmat);

  // element (j, t) of the tile; t = tid % TT is fixed per thread (TILE_THREADS % TT == 0).
  // Tube offset j = jf + nf*jh of the tensor (mode 3 fastest) is tile row jf*znb + jh.
  const int t = tid % TT;
  const int nf = g.nf;
  const int znb = s.znb;
  const DivNf dn(nf);
  auto zrow = [&](int j) -> size_t {
    const int jh = dn.div(j);
    return ((size_t)(j - jh * nf) * znb + jh) * TT + t;
  };
  const bool live = t0 + t < N12;
  // rows j0, j0 + RS, ... of a thread are processed U at a time: the U rows' global loads are
  // issued together before any of their stores (restrict pointers), so each thread keeps U
  // loads in flight instead of one
  constexpr int RS = TILE_THREADS / TT;
  constexpr int U = 8;
  const float* __restrict__ in = a.in;
  float* __restrict__ state = a.state;
  float* __restrict__ out0 = a.out0;
  float* __restrict__ out1 = a.out1;
  const int64_t tt = t0 + t;
  switch (a.mode) {
    case TUBE_FWD:
      for (int j0 = tid / TT; j0 < nreal; j0 += U * RS) {
        float v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int j = j0 + u * RS;
          v[u] = (live && j < nreal) ? in[tt + N12 * j] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int j = j0 + u * RS;
          if (j < nreal) s.zt[zrow(j)] = v[u];
        }
      }
      break;
    case TUBE_INV:
      for (int j = tid / TT; j < nreal; j += RS)
        if (live) out0[tt + N12 * j] = s.zt[zrow(j)];
      break;
    case TUBE_COMPLETE:
      for (int j0 = tid / TT; j0 < nreal; j0 += U * RS) {
        float yv[U], sv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int j = j0 + u * RS;
          const bool ok = live && j < nreal;
          yv[u] = ok ? in[tt + N12 * j] : 0.f;
          sv[u] = (ok && !a.first) ? state[tt + N12 * j] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int j = j0 + u * RS;
          if (j >= nreal) continue;
          float vn = 0.f;
          if (live) {
            const int64_t e = tt + N12 * j;
            float z = 0.f, q = 0.f;
            if (!a.first) {
              z = s.zt[zrow(j)];
              q = (sv[u] - z) * a.ratio;
            }
            const float y = yv[u];
            const float x = (y != y) ? z - q : y;   // NaN marks an unobserved entry
            vn = x + q;
            state[e] = vn;
            if (a.write_out) out0[e] = x;
          }
          s.zt[zrow(j)] = vn;
        }
      }
      break;
    case TUBE_RPCA: {
      const float kappa = a.kappa;
      float f = 0.f;
      if (a.tube_sparse) {
        // eq. sparse2: one shrink factor per tube; D kept in the tile
        float part = 0.f;
        for (int j0 = tid / TT; j0 < nreal; j0 += U * RS) {
          float mv[U], wv[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int j = j0 + u * RS;
            const bool ok = live && j < nreal;
            mv[u] = ok ? in[tt + N12 * j] : 0.f;
            wv[u] = (ok && !a.first) ? state[tt + N12 * j] : 0.f;
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int j = j0 + u * RS;
            if (j >= nreal) continue;
            float d = 0.f;
            if (live) {
              const float l = s.zt[zrow(j)];
              if (a.last) out0[tt + N12 * j] = l;
              d = mv[u] - wv[u] - l;
            }
            s.zt[zrow(j)] = d;
            part += d * d;
          }
        }
        // the RS partial sums of each tube, added in a fixed order (run-to-run identical)
        s.nrm[(tid / TT) * TT + t] = part;
        tile_sync();
        float sq = 0.f;
#pragma unroll
        for (int r = 0; r < RS; ++r) sq += s.nrm[r * TT + t];
        const float nrm = sqrtf(sq);
        f = nrm > 0.f ? fmaxf(1.f - kappa / nrm, 0.f) : 0.f;
      }
      for (int j0 = tid / TT; j0 < nreal; j0 += U * RS) {
        float mv[U], wv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int j = j0 + u * RS;
          const bool ok = live && j < nreal;
          mv[u] = ok ? in[tt + N12 * j] : 0.f;
          wv[u] = (ok && !a.tube_sparse && !a.first) ? state[tt + N12 * j] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int j = j0 + u * RS;
          if (j >= nreal) continue;
          float vnext = 0.f;
          if (live) {
            const int64_t e = tt + N12 * j;
            const float m = mv[u];
            float d;
            if (a.tube_sparse) {
              d = s.zt[zrow(j)];
            } else {
              const float l = s.zt[zrow(j)];
              if (a.last) out0[e] = l;
              d = m - wv[u] - l;
            }
            float sv;
            if (a.tube_sparse) {
              sv = f * d;
            } else {
              const float r = fabsf(d) - kappa;
              sv = r > 0.f ? (d > 0.f ? r : -r) : 0.f;
            }
            if (a.last) {
              out1[e] = sv;
            } else {
              const float wn = (sv - d) * a.ratio;
              state[e] = wn;
              vnext = m - sv - wn;
            }
          }
          s.zt[zrow(j)] = vnext;
        }
      }
      break;
    }
    default:
      break;
  }
  const bool need_fwd = a.mode == TUBE_FWD || a.mode == TUBE_COMPLETE ||
                        (a.mode == TUBE_RPCA && !a.last);
  if (!need_fwd) return;
  tile_sync();
  tile_forward<RM>(s, g, a.twid_f, a.fmat);
  tile_store_spectrum(s, g, a.spec_out, t0);
}

// The tile form handles nf <= NF_MAX, hh <= 128 (RM <= 8) and a tile that fits in shared
// memory.
inline int tile_rm(const TubeGeom& g) {
  // 16 row groups of RM rows cover the hh output rows of each forward product
  if (g.nf > NF_MAX || g.hh > 128 || tile_smem_bytes(g) > 200 * 1024) return 0;
  return g.hh <= 32 ? 2 : g.hh <= 64 ? 4 : 8;
}

}  // namespace
}  // namespace tsvd
