// tube_tile.cuh -- the tile form of the tube pass (see tube_pass.cu for the fused ADMM
// steps it runs), shared by the standalone tube kernel and the persistent batched kernel.
// Device code and two small host helpers in an anonymous namespace: each translation unit
// that includes it gets its own copy.
#pragma once
#include "tsvd_internal.h"

namespace tsvd {
namespace {

// ---------------------------------------------------------------------------------------------
// Tile form (used whenever the shape fits): one CTA of 256 threads per tile of TT = 32
// consecutive tubes.  Global accesses are rows of 32 consecutive tubes (128 B real, 256 B
// complex).  The tile lives in shared memory as
//   zt[jf*nh + jh][t]          the real tube entries,
//   yt[jf*2hh + 2kh + c][t]    the half spectrum as (re, im) rows, c = 0, 1,
// and the half-mode DFTs of the tile are two small real matrix products against one shared
// matrix Fr[jh][2kh + c] = (cos, -sin)(2 pi kh jh / nh):
//   forward  (R2C)   yt = Fr^T zt   per jf block (M = 2hh rows, K = nh);
//   inverse  (C2R)   zt = Fr  (w . yt) per jf block (M = nh rows, K = 2hh), where the weights
//                    w_kh = c_kh / (nf nh) (c = 1 at kh = 0 and nh/2, else 2) are applied when
//                    the spectrum is loaded.
// Blocks of zt are nh4 = nh rounded up to 4 rows, blocks of yt and the rows of Fr q4 = 2hh
// rounded up to 8 (Fr has nh4 rows), all padding zero, so the products run over K in steps
// of 4 with 128-bit loads: the forward reads Fr rows r..r+RM-1 of one k at once, the inverse
// 4 k of one row.  256 threads = 8 groups of 4 tubes x 32 groups of RM consecutive rows; a
// thread accumulates RM rows x 4 tubes with packed FP32x2 FMAs (two tubes per register pair).
// The full-mode DFT of the 4-way case (length nf <= 8) runs in registers per (kh, tube).
// The fused ADMM steps are those of the thread-per-tube form above, on the tile in shared
// memory.
constexpr int TT = 32;
constexpr int TILE_THREADS = 256;
constexpr int NF_MAX = 8;

// Barrier of the TILE_THREADS threads that run a tile (named barrier 1): a CTA with more
// threads runs tiles on its first TILE_THREADS threads while the others skip them.
__device__ __forceinline__ void tile_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(TILE_THREADS) : "memory");
}

struct TileSmem {
  float* fr;     // [nh][ldq]
  float* zt;     // [nf*nh][TT]
  float* yt;     // [nf*2hh][TT]
  float* nrm;    // [RS][TT] partial tube norms (RPCA tube mode)
  int ldq;
};

__host__ __device__ inline int tile_nh4(const TubeGeom& g) { return (g.nh + 3) & ~3; }
// q4 a multiple of 8: a row group r0 = RM rg < q4 (RM = 2, 4, 8) then ends inside the row
__host__ __device__ inline int tile_q4(const TubeGeom& g) { return (2 * g.hh + 7) & ~7; }
__host__ __device__ inline int tile_ldq(const TubeGeom& g) { return tile_q4(g); }

// Floats of the Fr matrix (a multiple of 16: the tiles after it stay 16-byte aligned).
__host__ __device__ inline size_t tile_fr_floats(const TubeGeom& g) {
  return (size_t)tile_nh4(g) * tile_q4(g);
}

__host__ __device__ inline size_t tile_smem_bytes(const TubeGeom& g) {
  return (tile_fr_floats(g) + (size_t)g.nf * tile_nh4(g) * TT + (size_t)g.nf * tile_q4(g) * TT +
          (size_t)(TILE_THREADS / TT) * TT) * sizeof(float);
}

__device__ __forceinline__ float2 ffma2s(float a, float2 b, float2 c) {
  return __ffma2_rn(make_float2(a, a), b, c);
}

// out[r][t] = sum_{k < K} A(r, k) B[k][t] for r < M and the 32 tubes of the tile; K is a
// multiple of 4 (B rows and A entries past the true extent are zero).  FWD: A(r, k) =
// fr[k * ldq + r]; otherwise A(r, k) = fr[r * ldq + k].  Rows past Fr's extent (rext: ldq for
// FWD, the row count otherwise) read a clamped, in-bounds position once and are not stored.
template <int RM, bool FWD>
__device__ __forceinline__ void tile_product(const float* __restrict__ fr, int ldq, int rext,
                                             const float* __restrict__ b, float* __restrict__ out,
                                             int M, int K) {
  const int tg = threadIdx.x & 7, rg = threadIdx.x >> 3;
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
  const int nf = g.nf, hh = g.hh, q4 = tile_q4(g);
  for (int idx = threadIdx.x; idx < hh * TT; idx += TILE_THREADS) {
    const int kh = idx / TT, t = idx % TT;
    float2 x[NF_MAX], y[NF_MAX];
    for (int f = 0; f < nf; ++f) {
      const size_t row = (size_t)f * q4 + 2 * kh;
      x[f] = make_float2(s.yt[row * TT + t], s.yt[(row + 1) * TT + t]);
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
      const size_t row = (size_t)f * q4 + 2 * kh;
      s.yt[row * TT + t] = y[f].x;
      s.yt[(row + 1) * TT + t] = y[f].y;
    }
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
  const int nh4 = tile_nh4(g), q4 = tile_q4(g);
  for (int f = 0; f < g.nf; ++f)
    tile_product<RM, false>(s.fr, s.ldq, nh4, s.yt + (size_t)f * q4 * TT,
                            s.zt + (size_t)f * nh4 * TT, g.nh, q4);
  tile_sync();
}

// Real tile -> spectrum tile.
template <int RM>
__device__ void tile_forward(const TileSmem& s, const TubeGeom& g, const float2* twf,
                             const float2* fm) {
  const int nh4 = tile_nh4(g), q4 = tile_q4(g);
  for (int f = 0; f < g.nf; ++f)
    tile_product<RM, true>(s.fr, s.ldq, s.ldq, s.zt + (size_t)f * nh4 * TT,
                           s.yt + (size_t)f * q4 * TT, 2 * g.hh, nh4);
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
  const int nf = g.nf, nh = g.nh, hh = g.hh, q4 = tile_q4(g);
  const float inv = 1.f / (float)(nf * nh);
  const int total = nf * hh * TT;
  constexpr int U = 4;   // loads a thread keeps in flight (see the element loops)
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
      const size_t row = (size_t)kf * q4 + 2 * kh;
      s.yt[row * TT + t] = v[u].x * w;
      s.yt[(row + 1) * TT + t] = v[u].y * w;
    }
  }
}

__device__ void tile_store_spectrum(const TileSmem& s, const TubeGeom& g, float2* __restrict__ spec,
                                    int64_t t0) {
  const int nf = g.nf, hh = g.hh, q4 = tile_q4(g);
  for (int idx = threadIdx.x; idx < nf * hh * TT; idx += TILE_THREADS) {
    const int q = idx / TT, t = idx % TT;
    if (t0 + t >= g.N12) continue;
    const int kf = q % nf, kh = q / nf;
    const size_t row = (size_t)kf * q4 + 2 * kh;
    spec[(size_t)q * g.N12 + t0 + t] = make_float2(s.yt[row * TT + t], s.yt[(row + 1) * TT + t]);
  }
}

// One tile of TT tubes starting at tube t0, run by threads 0 .. TILE_THREADS - 1 of the CTA
// (their barrier is tile_sync); smem_raw holds tile_smem_bytes(a.g) bytes.
template <int RM>
__device__ void tube_tile_body(const TubeArgs& a, int64_t t0, unsigned char* smem_raw) {
  const TubeGeom g = a.g;
  TileSmem s;
  s.ldq = tile_ldq(g);
  s.fr = reinterpret_cast<float*>(smem_raw);
  const int nh4 = tile_nh4(g), q4 = tile_q4(g);
  s.zt = s.fr + tile_fr_floats(g);
  s.yt = s.zt + (size_t)g.nf * nh4 * TT;
  s.nrm = s.yt + (size_t)g.nf * q4 * TT;
  const int tid = threadIdx.x;
  const int nh = g.nh, hh = g.hh, nreal = g.nf * g.nh;
  const int64_t N12 = g.N12;
  // Fr[jh][2kh + c] from the twiddle table (exact at the quarter points), one row per thread
  // with the index jh kh mod nh stepped by jh; zero past nh rows and 2hh columns
  for (int jh = tid; jh < nh4; jh += TILE_THREADS) {
    float2* row = reinterpret_cast<float2*>(s.fr + (size_t)jh * s.ldq);
    int m = 0;
    for (int kh = 0; kh < q4 / 2; ++kh) {
      float2 v = make_float2(0.f, 0.f);
      if (jh < nh && kh < hh) {
        const float2 w = a.twid_h[m];
        v = make_float2(w.x, -w.y);
      }
      row[kh] = v;
      m += jh;
      if (m >= nh) m -= nh;
    }
  }
  // zero the padding rows of the zt and yt blocks (never written below)
  for (int f = 0; f < g.nf; ++f) {
    for (int idx = tid; idx < (nh4 - nh) * TT; idx += TILE_THREADS)
      s.zt[((size_t)f * nh4 + nh) * TT + idx] = 0.f;
    for (int idx = tid; idx < (q4 - 2 * hh) * TT; idx += TILE_THREADS)
      s.yt[((size_t)f * q4 + 2 * hh) * TT + idx] = 0.f;
  }
  const bool need_inv = a.mode == TUBE_INV || a.mode == TUBE_RPCA ||
                        (a.mode == TUBE_COMPLETE && !a.first);
  if (need_inv) tile_load_spectrum(s, g, a.spec_in, t0, a.fpart);
  tile_sync();
  if (need_inv) tile_inverse<RM>(s, g, a.twid_f, a.fmat);

  // element (j, t) of the tile; t = tid % TT is fixed per thread (TILE_THREADS % TT == 0).
  // Tube offset j = jf + nf*jh of the tensor (mode 3 fastest) is tile row jf*nh4 + jh.
  const int t = tid % TT;
  const int nf = g.nf;
  auto zrow = [&](int j) -> size_t { return ((size_t)(j % nf) * nh4 + j / nf) * TT + t; };
  const bool live = t0 + t < N12;
  // rows j0, j0 + RS, ... of a thread are processed U at a time: the U rows' global loads are
  // issued together before any of their stores (restrict pointers), so each thread keeps U
  // loads in flight instead of one
  constexpr int RS = TILE_THREADS / TT;
  constexpr int U = 4;
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

// The tile form handles nf <= NF_MAX, 2 hh <= 256 (RM <= 8) and a tile that fits in shared
// memory.
inline int tile_rm(const TubeGeom& g) {
  const int m = 2 * g.hh > g.nh ? 2 * g.hh : g.nh;
  if (g.nf > NF_MAX || m > 256 || tile_smem_bytes(g) > 200 * 1024) return 0;
  return m <= 64 ? 2 : m <= 128 ? 4 : 8;
}

}  // namespace
}  // namespace tsvd
