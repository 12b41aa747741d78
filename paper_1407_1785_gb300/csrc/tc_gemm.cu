// tc_gemm.cu -- tensor-core engines of the batched complex slice products of the mixed form
// (sketch Y = Aw P, projection Bt = Aw^T conj(Q), rebuild Zw = Q Dt^T; see rsvt.cu).
//
// 3M complex product: with A = Ar + i Ai and B = Br + i Bi,
//     T1 = Ar Br,  T2 = Ai Bi,  T3 = (Ar + Ai)(Br + Bi),  C = (T1 - T2) + i (T3 - T1 - T2),
// three real products instead of four.  Each real product runs as tcgen05.mma with the
// operands in shared memory and the FP32 accumulators T1, T2, T3 in tensor memory:
//   TF32    operands rounded to TF32 (cvt.rna), kind::tf32, K = 8 per instruction;
//   3XTF32  x = hi + lo with hi = tf32(x), lo = tf32(x - hi); every real product is
//           hi*hi + hi*lo + lo*hi (the lo*lo term is below FP32 rounding), kind::tf32;
//   BF16    operands rounded to BF16, kind::f16 with BF16 inputs, K = 16 per instruction.
//
// Work split.  One CTA (256 threads) per 128 x 64 tile of C and per batch entry.  The K
// range is walked in chunks; for each chunk all threads load the complex operand tiles from
// global memory (any strides, optional conjugation), form the real planes (re, im, re+im; hi
// and lo for 3XTF32) and store them in the canonical no-swizzle K-major layout: 8-row x
// 16-byte core matrices, consecutive 8-row groups 128 bytes apart (stride-dimension offset),
// consecutive K core matrices one plane height apart (leading-dimension offset).  One
// thread then issues the chunk's MMAs and commits them to the chunk buffer's mbarrier; two
// chunk buffers alternate so loading chunk c+1 overlaps the MMAs of chunk c.  With 3XTF32
// each thread copies its share of the raw complex entries with cp.async into three private
// slots, two chunks ahead, and converts chunk c from its slot: the global latency overlaps
// two chunks of conversion and MMA issue instead of sitting in front of each chunk.  The epilogue
// reads T1..T3 with tcgen05.ld (warp w reads TMEM lanes 32 (w mod 4) .. +31, i.e. its rows of
// the tile, and half of the columns) and writes C.
//
// Every mbarrier wait is bounded; on expiry the kernel counts a timeout (read by the host
// through tc_gemm_take_timeouts), waits again (bounded) for its own MMAs, frees its tensor
// memory and returns.
#include "tsvd_internal.h"

#include <cuda_bf16.h>

namespace tsvd {

__device__ int g_tc_timeouts = 0;

namespace {

constexpr int BM = 128, BN = 64, NTHR = 256;
constexpr int TMEM_COLS = 256;     // >= 3 * BN fp32 accumulator columns, power of two
constexpr long long kWaitIters = 1ll << 24;
constexpr uint64_t kWaitNs = 2000000000ull;   // 2 s

template <int ENG>
struct Cfg;
template <>
struct Cfg<RSVT_GEMM_TF32> {
  static constexpr int EB = 4, EPC = 4, BK = 32, NSPLIT = 1, KMMA = 8, FMT = 2, F16 = 0;
};
template <>
struct Cfg<RSVT_GEMM_3XTF32> {
  static constexpr int EB = 4, EPC = 4, BK = 16, NSPLIT = 2, KMMA = 8, FMT = 2, F16 = 0;
};
template <>
struct Cfg<RSVT_GEMM_BF16> {
  static constexpr int EB = 2, EPC = 8, BK = 64, NSPLIT = 1, KMMA = 16, FMT = 1, F16 = 1;
};

template <int ENG>
struct Layout {
  using C = Cfg<ENG>;
  static constexpr int KG = C::BK / C::EPC;                  // core matrices along K
  static constexpr int PLANE_A = BM * C::BK * C::EB;         // bytes
  static constexpr int PLANE_B = BN * C::BK * C::EB;
  static constexpr int NPLANE = 3 * C::NSPLIT;
  static constexpr int STAGE = NPLANE * (PLANE_A + PLANE_B);
  // 3XTF32: raw complex operand chunks copied asynchronously (cp.async) into per-thread slots,
  // up to two chunks ahead of the one being converted; the other engines' planes leave no
  // room for them and load through registers
  static constexpr int RAW_STAGES = ENG == RSVT_GEMM_3XTF32 ? 3 : 0;
  static constexpr int RAW_A = BM * C::BK * 8;               // bytes of one raw A chunk
  static constexpr int RAW_B = BN * C::BK * 8;
  static constexpr int RAW = RAW_STAGES * (RAW_A + RAW_B);
  static constexpr int SMEM = 2 * STAGE + RAW + 64;          // + mbarriers and TMEM address
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// Shared-memory matrix descriptor: no swizzle, K-major core matrices.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of tcgen05
  return d;
}

template <int ENG>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t acc) {
  if (Cfg<ENG>::F16)
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  else
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
}

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Waits for the phase of parity `parity` of the mbarrier; false after kWaitNs or
// kWaitIters polls, whichever comes first.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = now_ns();
  for (long long it = 0; it < kWaitIters; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred P1;\nmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n"
        "selp.b32 %0, 1, 0, P1;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255) == 255 && now_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

// 8-byte asynchronous global -> shared copy; with pred false it writes zeros and reads nothing.
__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool pred) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src),
               "r"(pred ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// The real planes of EPC consecutive complex entries (one core-matrix row of each plane).
template <int ENG>
struct Row {
  uint32_t w[3 * Cfg<ENG>::NSPLIT][Cfg<ENG>::EPC * Cfg<ENG>::EB / 4];
};

template <int ENG>
__device__ __forceinline__ void make_planes(const float2 (&x)[Cfg<ENG>::EPC], Row<ENG>& row) {
  using C = Cfg<ENG>;
  if (C::F16) {
#pragma unroll
    for (int q = 0; q < C::EPC; q += 2) {
      const float r0 = x[q].x, i0 = x[q].y, r1 = x[q + 1].x, i1 = x[q + 1].y;
      const __nv_bfloat162 br = __floats2bfloat162_rn(r0, r1);
      const __nv_bfloat162 bi = __floats2bfloat162_rn(i0, i1);
      const __nv_bfloat162 bs = __floats2bfloat162_rn(r0 + i0, r1 + i1);
      row.w[0][q / 2] = *reinterpret_cast<const uint32_t*>(&br);
      row.w[1][q / 2] = *reinterpret_cast<const uint32_t*>(&bi);
      row.w[2][q / 2] = *reinterpret_cast<const uint32_t*>(&bs);
    }
  } else {
#pragma unroll
    for (int q = 0; q < C::EPC; ++q) {
      const float v[3] = {x[q].x, x[q].y, x[q].x + x[q].y};
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        const uint32_t hi = tf32_rna(v[p]);
        row.w[p * C::NSPLIT][q] = hi;
        if (C::NSPLIT == 2) row.w[p * C::NSPLIT + 1][q] = tf32_rna(v[p] - __uint_as_float(hi));
      }
    }
  }
}

// Loads and stores the planes of one operand tile (R rows x BK complex entries of chunk l0).
// Row r of the tile is operand row row0 + r; entry (row, l) sits at base[row * sr + l * sl].
template <int ENG, int R>
__device__ __forceinline__ void stage_operand(unsigned char* planes, int plane_bytes,
                                              const float2* base, int64_t sr, int64_t sl,
                                              int conj, int row0, int nrows, int l0, int K) {
  using C = Cfg<ENG>;
  constexpr int KG = Layout<ENG>::KG;
  constexpr int ITEMS = R * KG;
  constexpr int PER = ITEMS / NTHR;
  static_assert(ITEMS % NTHR == 0, "tile items must divide the thread count");
  float2 x[PER][C::EPC];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int item = threadIdx.x + NTHR * u;
    const int r = item % R, kg = item / R;
    const int row = row0 + r;
#pragma unroll
    for (int q = 0; q < C::EPC; ++q) {
      const int l = l0 + kg * C::EPC + q;
      float2 v = make_float2(0.f, 0.f);
      if (row < nrows && l < K) {
        v = base[(int64_t)row * sr + (int64_t)l * sl];
        if (conj) v.y = -v.y;
      }
      x[u][q] = v;
    }
  }
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int item = threadIdx.x + NTHR * u;
    const int r = item % R, kg = item / R;
    Row<ENG> row;
    make_planes<ENG>(x[u], row);
    const int off = (kg * (R / 8) + r / 8) * 128 + (r % 8) * 16;
#pragma unroll
    for (int pl = 0; pl < 3 * C::NSPLIT; ++pl) {
      uint4 val;
      val.x = row.w[pl][0];
      val.y = row.w[pl][1];
      val.z = row.w[pl][2];
      val.w = row.w[pl][3];
      *reinterpret_cast<uint4*>(planes + (size_t)pl * plane_bytes + off) = val;
    }
  }
}

// Asynchronous copy of a thread's share of one operand tile (chunk l0) into its raw slots
// raw[(u EPC + q) NTHR + tid]: the thread that converts an entry is the one that copied it,
// so the copies need no barrier, only the thread's own cp.async.wait_group.
template <int ENG, int R>
__device__ __forceinline__ void issue_operand(float2* raw, const float2* base, int64_t sr,
                                              int64_t sl, int row0, int nrows, int l0, int K) {
  using C = Cfg<ENG>;
  constexpr int PER = R * Layout<ENG>::KG / NTHR;
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int item = threadIdx.x + NTHR * u;
    const int r = item % R, kg = item / R;
    const int row = row0 + r;
#pragma unroll
    for (int q = 0; q < C::EPC; ++q) {
      const int l = l0 + kg * C::EPC + q;
      const bool ok = row < nrows && l < K;
      const float2* src = ok ? base + (int64_t)row * sr + (int64_t)l * sl : base;
      cp_async8(raw + (size_t)(u * C::EPC + q) * NTHR + threadIdx.x, src, ok);
    }
  }
}

// Converts a thread's raw share into the planes (conjugating on the way).
template <int ENG, int R>
__device__ __forceinline__ void convert_operand(const float2* raw, int conj, unsigned char* planes,
                                                int plane_bytes) {
  using C = Cfg<ENG>;
  constexpr int PER = R * Layout<ENG>::KG / NTHR;
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int item = threadIdx.x + NTHR * u;
    const int r = item % R, kg = item / R;
    float2 x[C::EPC];
#pragma unroll
    for (int q = 0; q < C::EPC; ++q) {
      x[q] = raw[(size_t)(u * C::EPC + q) * NTHR + threadIdx.x];
      if (conj) x[q].y = -x[q].y;
    }
    Row<ENG> row;
    make_planes<ENG>(x, row);
    const int off = (kg * (R / 8) + r / 8) * 128 + (r % 8) * 16;
#pragma unroll
    for (int pl = 0; pl < 3 * C::NSPLIT; ++pl) {
      uint4 val;
      val.x = row.w[pl][0];
      val.y = row.w[pl][1];
      val.z = row.w[pl][2];
      val.w = row.w[pl][3];
      *reinterpret_cast<uint4*>(planes + (size_t)pl * plane_bytes + off) = val;
    }
  }
}

template <int ENG>
__global__ void __launch_bounds__(NTHR, 1) cgemm_tc_kernel(CGemm g) {
  using C = Cfg<ENG>;
  using L = Layout<ENG>;
  extern __shared__ __align__(1024) unsigned char smem[];
  if (g.kdev) {
    const int kk = *g.kdev;
    if (g.dynM) g.M = kk;
    if (g.dynN) g.N = kk;
    if (g.dynK) g.K = kk;
  }
  // tiles past a device-chosen extent have nothing to do (before any barrier or allocation)
  if ((int)blockIdx.x * BM >= g.M || (int)blockIdx.y * BN >= g.N) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int bz = blockIdx.z;
  const float2* A = g.a.p + (int64_t)(g.a.idx ? g.a.idx[bz] : bz) * g.a.bs;
  const float2* B = g.b.p + (int64_t)(g.b.idx ? g.b.idx[bz] : bz) * g.b.bs;
  float2* Cp = const_cast<float2*>(g.c.p) + (int64_t)(g.c.idx ? g.c.idx[bz] : bz) * g.c.bs;
  const int i0 = blockIdx.x * BM, j0 = blockIdx.y * BN;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * L::STAGE + L::RAW);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 2 * L::STAGE + L::RAW + 32);
  float2* raw = reinterpret_cast<float2*>(smem + 2 * L::STAGE);   // RAW_STAGES x (A, B)
  auto raw_a = [&](int c) { return raw + (size_t)(c % 3) * ((L::RAW_A + L::RAW_B) / 8); };
  auto raw_b = [&](int c) { return raw_a(c) + L::RAW_A / 8; };
  const uint32_t bar0 = smem_u32(&bars[0]), bar1 = smem_u32(&bars[1]);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    mbar_init(bar0);
    mbar_init(bar1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  constexpr uint32_t idesc = (1u << 4) | ((uint32_t)C::FMT << 7) | ((uint32_t)C::FMT << 10) |
                             ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
  constexpr uint32_t LBO_A = (BM / 8) * 128, LBO_B = (BN / 8) * 128, SBO = 128;
  constexpr int KSTEPS = C::BK / C::KMMA;
  const int nk = (g.K + C::BK - 1) / C::BK;
  bool timed_out = false;
  if constexpr (L::RAW_STAGES > 0) {
    // chunks 0 and 1 in flight before the loop; one commit group per chunk (empty past nk)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (c < nk) {
        issue_operand<ENG, BM>(raw_a(c), A, g.a.s0, g.a.s1, i0, g.M, c * C::BK, g.K);
        issue_operand<ENG, BN>(raw_b(c), B, g.b.s1, g.b.s0, j0, g.N, c * C::BK, g.K);
      }
      cp_async_commit();
    }
  }
  int kc = 0;
  for (; kc < nk; ++kc) {
    const int buf = kc & 1;
    if constexpr (L::RAW_STAGES > 0) {
      // chunk kc + 2 into the slot chunk kc - 1 used (converted by this thread last time)
      if (kc + 2 < nk) {
        issue_operand<ENG, BM>(raw_a(kc + 2), A, g.a.s0, g.a.s1, i0, g.M, (kc + 2) * C::BK, g.K);
        issue_operand<ENG, BN>(raw_b(kc + 2), B, g.b.s1, g.b.s0, j0, g.N, (kc + 2) * C::BK, g.K);
      }
      cp_async_commit();
    }
    if (kc >= 2) {
      const bool ok = mbar_wait(buf ? bar1 : bar0, (uint32_t)(((kc >> 1) - 1) & 1));
      if (__syncthreads_or(!ok)) {
        timed_out = true;
        break;
      }
    }
    unsigned char* st = smem + (size_t)buf * L::STAGE;
    unsigned char* pa = st;
    unsigned char* pb = st + L::NPLANE * L::PLANE_A;
    if constexpr (L::RAW_STAGES > 0) {
      cp_async_wait<2>();   // this thread's copies of chunk kc have landed
      convert_operand<ENG, BM>(raw_a(kc), g.a.conj, pa, L::PLANE_A);
      convert_operand<ENG, BN>(raw_b(kc), g.b.conj, pb, L::PLANE_B);
    } else {
      const int l0 = kc * C::BK;
      stage_operand<ENG, BM>(pa, L::PLANE_A, A, g.a.s0, g.a.s1, g.a.conj, i0, g.M, l0, g.K);
      stage_operand<ENG, BN>(pb, L::PLANE_B, B, g.b.s1, g.b.s0, g.b.conj, j0, g.N, l0, g.K);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_base = smem_u32(pa), b_base = smem_u32(pb);
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        const uint32_t d = tmem + (uint32_t)(p * BN);
#pragma unroll
        for (int s = 0; s < KSTEPS; ++s) {
#pragma unroll
          for (int t = 0; t < (C::NSPLIT == 2 ? 3 : 1); ++t) {
            // 3XTF32 terms: (hi, hi), (hi, lo), (lo, hi)
            const int ha = t == 2 ? 1 : 0, hb = t == 1 ? 1 : 0;
            const uint32_t aa = a_base + (uint32_t)((p * C::NSPLIT + ha) * L::PLANE_A) +
                                (uint32_t)(s * 2) * LBO_A;
            const uint32_t bb = b_base + (uint32_t)((p * C::NSPLIT + hb) * L::PLANE_B) +
                                (uint32_t)(s * 2) * LBO_B;
            const uint32_t acc = (kc > 0 || s > 0 || t > 0) ? 1u : 0u;
            mma<ENG>(d, sdesc(aa, LBO_A, SBO), sdesc(bb, LBO_B, SBO), idesc, acc);
          }
        }
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              buf ? bar1 : bar0)
          : "memory");
    }
  }
  // no asynchronous copy may still be landing in shared memory when the CTA moves on or exits
  if constexpr (L::RAW_STAGES > 0) cp_async_wait<0>();
  // wait for the last committed chunk (its commit covers every earlier MMA)
  const int last = (timed_out ? kc : nk) - 1;
  bool ok = true;
  if (last >= 0) ok = mbar_wait((last & 1) ? bar1 : bar0, (uint32_t)((last >> 1) & 1));
  if (!ok || timed_out) {
    if (tid == 0) atomicAdd(&g_tc_timeouts, 1);
  }
  const bool good = !timed_out && !__syncthreads_or(!ok);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (good && nk > 0) {
    const int q = warp & 3, half = warp >> 2;
    const int i = i0 + 32 * q + lane;
#pragma unroll
    for (int cc = 0; cc < 32; cc += 16) {
      const uint32_t col = (uint32_t)(32 * half + cc);
      const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + col;
      float t1[16], t2[16], t3[16];
      tmem_ld16(ta, t1);
      tmem_ld16(ta + BN, t2);
      tmem_ld16(ta + 2 * BN, t3);
      if (i < g.M) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int j = j0 + (int)col + e;
          if (j < g.N)
            Cp[(int64_t)i * g.c.s0 + (int64_t)j * g.c.s1] =
                make_float2(t1[e] - t2[e], t3[e] - t1[e] - t2[e]);
        }
      }
    }
  } else if (nk == 0) {
    // empty contraction: C = 0
    for (int idx = tid; idx < BM * BN; idx += NTHR) {
      const int i = i0 + idx % BM, j = j0 + idx / BM;
      if (i < g.M && j < g.N) Cp[(int64_t)i * g.c.s0 + (int64_t)j * g.c.s1] = make_float2(0.f, 0.f);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS));
  }
}

template <int ENG>
cudaError_t launch_eng(const CGemm& g, cudaStream_t st) {
  static bool attr = false;
  const int smem = Layout<ENG>::SMEM;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(cgemm_tc_kernel<ENG>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((g.M + BM - 1) / BM, (g.N + BN - 1) / BN, g.batch);
  cgemm_tc_kernel<ENG><<<grid, NTHR, smem, st>>>(g);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_cgemm_tc(const CGemm& g, int engine, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.batch > 65535) return cudaErrorInvalidValue;
  switch (engine) {
    case RSVT_GEMM_TF32: return launch_eng<RSVT_GEMM_TF32>(g, st);
    case RSVT_GEMM_3XTF32: return launch_eng<RSVT_GEMM_3XTF32>(g, st);
    case RSVT_GEMM_BF16: return launch_eng<RSVT_GEMM_BF16>(g, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t tc_gemm_take_timeouts(int* count, cudaStream_t st) {
  int h = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(&h, g_tc_timeouts, sizeof h, 0,
                                            cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && h) {
    const int zero = 0;
    e = cudaMemcpyToSymbolAsync(g_tc_timeouts, &zero, sizeof zero, 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  *count = h;
  return e;
}

}  // namespace tsvd
