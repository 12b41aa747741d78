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

struct TileSmem {
  float* fre;    // [kr4][ldf]  cos rows r < KR, zero-padded
  float* fim;    // [ki4][ldf]  -sin rows r >= KR, zero-padded
  float* zt;     // [nf][znb][TT]
  float* yt;     // [nf][2 q2][TT]
  float* nrm;    // [RS][TT] partial tube norms (RPCA tube mode)
  int ldf, kr, ki, znb, q2;
};

__host__ __device__ inline int tile_kr(const TubeGeom& g) { return g.nh / 2 + 1; }
__host__ __device__ inline int tile_ki(const TubeGeom& g) { return g.nh - tile_kr(g); }
__host__ __device__ inline int tile_round4(int x) { return (x + 3) & ~3; }
// table row length: hh rounded up to 8 (an RM-row group of the forward product reads inside it)
__host__ __device__ inline int tile_ldf(const TubeGeom& g) { return (g.hh + 7) & ~7; }
// zt block rows: the sine product reads KI rounded up to 4 rows from row KR, up to row nh + 2
__host__ __device__ inline int tile_znb(const TubeGeom& g) { return tile_round4(g.nh + 3); }
__host__ __device__ inline int tile_q2(const TubeGeom& g) { return tile_round4(g.hh); }

__host__ __device__ inline size_t tile_table_floats(const TubeGeom& g) {
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
  s.fre = reinterpret_cast<float*>(raw);
  s.fim = s.fre + (size_t)tile_round4(s.kr) * s.ldf;
  s.zt = s.fre + tile_table_floats(g);
  s.yt = s.zt + (size_t)g.nf * s.znb * TT;
  s.nrm = s.yt + (size_t)g.nf * 2 * s.q2 * TT;
  return s;
}

// The tables F (from the twiddle table, exact at the quarter points: the index r kh mod nh is
// stepped by r) and the zero padding of the zt and yt blocks, which the tile steps never write.
__device__ void tile_build(const TileSmem& s, const TubeGeom& g, const float2* __restrict__ twid_h) {
  const int nh = g.nh, hh = g.hh, ldf = s.ldf;
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

// Spectrum tile (loaded, weighted) -> real tile.
template <int RM>
__device__ void tile_inverse(const TileSmem& s, const TubeGeom& g, const float2* twf,
                             const float2* fm) {
  if (g.nf > 1) {
    tile_full_dft(s, g, twf, 1.f, fm);
    tile_sync();
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

// Real tile -> spectrum tile.
template <int RM>
__device__ void tile_forward(const TileSmem& s, const TubeGeom& g, const float2* twf,
                             const float2* fm) {
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
  if (g.nf > 1) {
    tile_full_dft(s, g, twf, -1.f, fm);
    tile_sync();
  }
}

// Loads the stored spectrum of the tile (conjugate partners on the self-conjugate columns)
// and applies the C2R weights c_kh / (nf nh).
__device__ void tile_load_spectrum(const TileSmem& s, const TubeGeom& g,
                                   const float2* __restrict__ spec, int64_t t0,
                                   const int* __restrict__ fp) {
  const int nf = g.nf, nh = g.nh, hh = g.hh, q2 = s.q2;
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
        const int kf = q % nf, kh = q / nf;
        const bool selfcol = (kh == 0) || (2 * kh == nh);
        const int pk = fp ? fp[kf] : (nf - kf) % nf;
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
      const int kf = q % nf, kh = q / nf;
      const bool selfcol = (kh == 0) || (2 * kh == nh);
      const float w = (selfcol ? 1.f : 2.f) * inv;
      const size_t row = (size_t)kf * 2 * q2 + kh;
      s.yt[row * TT + t] = v[u].x * w;
      s.yt[(row + q2) * TT + t] = v[u].y * w;
    }
  }
}

__device__ void tile_store_spectrum(const TileSmem& s, const TubeGeom& g, float2* __restrict__ spec,
                                    int64_t t0) {
  const int nf = g.nf, hh = g.hh, q2 = s.q2;
  for (int idx = threadIdx.x; idx < nf * hh * TT; idx += TILE_THREADS) {
    const int q = idx / TT, t = idx % TT;
    if (t0 + t >= g.N12) continue;
    const int kf = q % nf, kh = q / nf;
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
  auto zrow = [&](int j) -> size_t { return ((size_t)(j % nf) * znb + j / nf) * TT + t; };
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
