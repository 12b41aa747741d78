// tube_pass.cu -- the HBM-bound tube passes of the t-SVT ADMM loops.
//
// One thread owns one tube (pixel t = i + n1*j) and runs, entirely in shared memory, the
// DFT along the tube modes (Sec. 2.1: the t-product and the t-SVD are computed "by
// performing the FFT along the tube fibers"; Algorithm 1's fft(.,[],i) loop over modes
// 3..N), keeping only the conjugate-symmetric half of the last mode.  Warp lanes own
// adjacent tubes, so every global access of a warp is one contiguous 128 B (real) or
// 256 B (complex) run.
//
// The fused ADMM passes fold the elementwise steps of both methods into the transforms:
//   TUBE_COMPLETE (Sec. 4, eq. proj + dual ascent), per tube entry e, with V = X + Q:
//       Z = C2R(Zhat);  Q = (V - Z) * rho_k/rho_{k+1};  X = Omega ? Y : Z - Q;
//       V = X + Q;  Vhat = R2C(V)
//   TUBE_RPCA (Sec. 5, eq. sparse / eq. sparse2 + eq. dual), with scaled dual W:
//       L = C2R(Lhat);  D = M - W - L;  S = shrink(D, lambda/rho_k);
//       W = (S - D) * rho_k/rho_{k+1}   (= (W + L + S - M) rescaled);
//       V = M - S - W;  Vhat = R2C(V)
// so each ADMM iteration reads and writes every tensor once.
#include "tsvd_internal.h"
#include "tube_tile.cuh"

#include <algorithm>

namespace tsvd {
namespace {

struct Smem {
  float2* tw_h;  // nh
  float2* tw_f;  // nf
  float2* sp;    // [nf*hh][TB]
  float2* tmp;   // [nf][TB]
  float* re;     // [nf*nh][TB]
};

template <int TB>
__device__ __forceinline__ Smem carve(unsigned char* raw, const TubeGeom& g) {
  Smem s;
  s.tw_h = reinterpret_cast<float2*>(raw);
  s.tw_f = s.tw_h + g.nh;
  s.sp = s.tw_f + g.nf;
  s.tmp = s.sp + (size_t)g.nf * g.hh * TB;
  s.re = reinterpret_cast<float*>(s.tmp + (size_t)g.nf * TB);
  return s;
}

// Spectrum (this thread's column of sp) -> real tube (column of re).  Inverse DFT along the
// full mode, then complex-to-real along the half mode, scaled by 1/(nf*nh).
template <int TB>
__device__ void inverse_tube(const Smem& s, const TubeGeom& g, int tid,
                             const float2* __restrict__ fm) {
  const int nf = g.nf, nh = g.nh, hh = g.hh;
  float2* sp = s.sp + tid;
  float2* tmp = s.tmp + tid;
  if (nf > 1) {
    for (int kh = 0; kh < hh; ++kh) {
      for (int jf = 0; jf < nf; ++jf) {
        float ar = 0.f, ai = 0.f;
        int m = 0;
        for (int kf = 0; kf < nf; ++kf) {
          const float2 x = sp[(size_t)(kf + nf * kh) * TB];
          const float2 w = fm ? fm[(size_t)jf * nf + kf] : s.tw_f[m];
          ar += x.x * w.x - x.y * w.y;
          ai += x.x * w.y + x.y * w.x;
          m += jf;
          if (m >= nf) m -= nf;
        }
        tmp[(size_t)jf * TB] = make_float2(ar, ai);
      }
      for (int jf = 0; jf < nf; ++jf) sp[(size_t)(jf + nf * kh) * TB] = tmp[(size_t)jf * TB];
    }
  }
  const float scale = 1.f / (float)(nf * nh);
  const bool even = (nh & 1) == 0;
  float* re = s.re + tid;
  for (int jf = 0; jf < nf; ++jf) {
    for (int jh = 0; jh < nh; ++jh) {
      float acc = sp[(size_t)jf * TB].x;
      int m = jh;
      for (int kh = 1; kh < hh; ++kh) {
        const float2 x = sp[(size_t)(jf + nf * kh) * TB];
        const float2 w = s.tw_h[m];
        const float c = (even && 2 * kh == nh) ? 1.f : 2.f;
        acc += c * (x.x * w.x - x.y * w.y);
        m += jh;
        if (m >= nh) m -= nh;
      }
      re[(size_t)(jf + nf * jh) * TB] = acc * scale;
    }
  }
}

// Real tube (column of re) -> half spectrum (column of sp): real-to-complex DFT along the
// half mode, then the full complex DFT along the other mode.
template <int TB>
__device__ void forward_tube(const Smem& s, const TubeGeom& g, int tid,
                             const float2* __restrict__ fm) {
  const int nf = g.nf, nh = g.nh, hh = g.hh;
  const float* re = s.re + tid;
  float2* sp = s.sp + tid;
  for (int jf = 0; jf < nf; ++jf) {
    for (int kh = 0; kh < hh; ++kh) {
      float ar = 0.f, ai = 0.f;
      int m = 0;
      for (int jh = 0; jh < nh; ++jh) {
        const float x = re[(size_t)(jf + nf * jh) * TB];
        const float2 w = s.tw_h[m];
        ar += x * w.x;
        ai -= x * w.y;
        m += kh;
        if (m >= nh) m -= nh;
      }
      sp[(size_t)(jf + nf * kh) * TB] = make_float2(ar, ai);
    }
  }
  if (nf > 1) {
    float2* tmp = s.tmp + tid;
    for (int kh = 0; kh < hh; ++kh) {
      for (int kf = 0; kf < nf; ++kf) {
        float ar = 0.f, ai = 0.f;
        int m = 0;
        for (int jf = 0; jf < nf; ++jf) {
          const float2 x = sp[(size_t)(jf + nf * kh) * TB];
          const float2 w = fm ? fm[(size_t)kf * nf + jf] : s.tw_f[m];
          // x * e^{-i theta}
          ar += x.x * w.x + x.y * w.y;
          ai += x.y * w.x - x.x * w.y;
          m += kf;
          if (m >= nf) m -= nf;
        }
        tmp[(size_t)kf * TB] = make_float2(ar, ai);
      }
      for (int kf = 0; kf < nf; ++kf) sp[(size_t)(kf + nf * kh) * TB] = tmp[(size_t)kf * TB];
    }
  }
}

// Load the stored half spectrum of tube t.  For kh = 0 and kh = nh/2 the slices whose
// conjugate partner has the smaller full index (kf > nf/2 for one full mode: partner nf - kf;
// several full modes: the table fp) are the complex conjugates of that partner (the t-SVT only
// computes the distinct member of each pair), so they are taken from the partner.
template <int TB>
__device__ void load_spectrum(const Smem& s, const TubeGeom& g, const float2* __restrict__ spec,
                              int64_t t, int tid, const int* __restrict__ fp) {
  const int nf = g.nf, nh = g.nh, hh = g.hh;
  for (int kh = 0; kh < hh; ++kh) {
    const bool selfcol = (kh == 0) || (2 * kh == nh);
    for (int kf = 0; kf < nf; ++kf) {
      float2 v;
      const int pk = fp ? fp[kf] : (nf - kf) % nf;
      if (selfcol && pk < kf) {
        v = spec[(size_t)(pk + nf * kh) * g.N12 + t];
        v.y = -v.y;
      } else {
        v = spec[(size_t)(kf + nf * kh) * g.N12 + t];
      }
      s.sp[(size_t)(kf + nf * kh) * TB + tid] = v;
    }
  }
}

template <int TB>
__device__ void store_spectrum(const Smem& s, const TubeGeom& g, float2* __restrict__ spec,
                               int64_t t, int tid) {
  for (int q = 0; q < g.nstore; ++q) spec[(size_t)q * g.N12 + t] = s.sp[(size_t)q * TB + tid];
}

template <int TB>
__global__ void __launch_bounds__(TB) tube_pass_kernel(TubeArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const TubeGeom g = a.g;
  const Smem s = carve<TB>(smem_raw, g);
  const int tid = threadIdx.x;
  for (int m = tid; m < g.nh; m += TB) s.tw_h[m] = a.twid_h[m];
  for (int m = tid; m < g.nf; m += TB) s.tw_f[m] = a.twid_f[m];
  __syncthreads();
  const int64_t t = (int64_t)blockIdx.x * TB + tid;
  if (t >= g.N12) return;  // no block-wide barrier below this point
  const int nreal = g.nf * g.nh;
  float* re = s.re + tid;
  const int64_t N12 = g.N12;

  switch (a.mode) {
    case TUBE_FWD: {
      for (int j = 0; j < nreal; ++j) re[(size_t)j * TB] = a.in[t + N12 * j];
      forward_tube<TB>(s, g, tid, a.fmat);
      store_spectrum<TB>(s, g, a.spec_out, t, tid);
      break;
    }
    case TUBE_INV: {
      load_spectrum<TB>(s, g, a.spec_in, t, tid, a.fpart);
      inverse_tube<TB>(s, g, tid, a.fmat);
      for (int j = 0; j < nreal; ++j) a.out0[t + N12 * j] = re[(size_t)j * TB];
      break;
    }
    case TUBE_COMPLETE: {
      if (!a.first) {
        load_spectrum<TB>(s, g, a.spec_in, t, tid, a.fpart);
        inverse_tube<TB>(s, g, tid, a.fmat);
      }
      for (int j = 0; j < nreal; ++j) {
        const int64_t e = t + N12 * j;
        float z = 0.f, q = 0.f;
        if (!a.first) {
          z = re[(size_t)j * TB];
          q = (a.state[e] - z) * a.ratio;
        }
        const float y = a.in[e];
        const float x = (y != y) ? z - q : y;   // NaN marks an unobserved entry
        const float v = x + q;
        a.state[e] = v;
        re[(size_t)j * TB] = v;
        if (a.write_out) a.out0[e] = x;
      }
      forward_tube<TB>(s, g, tid, a.fmat);
      store_spectrum<TB>(s, g, a.spec_out, t, tid);
      break;
    }
    case TUBE_RPCA: {
      load_spectrum<TB>(s, g, a.spec_in, t, tid, a.fpart);
      inverse_tube<TB>(s, g, tid, a.fmat);
      const float kappa = a.kappa;
      float f = 0.f;
      if (a.tube_sparse) {
        // eq. sparse2: one shrink factor for the whole tube
        float nrm2 = 0.f;
        for (int j = 0; j < nreal; ++j) {
          const int64_t e = t + N12 * j;
          const float l = re[(size_t)j * TB];
          if (a.last) a.out0[e] = l;
          const float w = a.first ? 0.f : a.state[e];
          const float d = a.in[e] - w - l;
          re[(size_t)j * TB] = d;
          nrm2 += d * d;
        }
        const float nrm = sqrtf(nrm2);
        f = nrm > 0.f ? fmaxf(1.f - kappa / nrm, 0.f) : 0.f;
      }
      for (int j = 0; j < nreal; ++j) {
        const int64_t e = t + N12 * j;
        const float m = a.in[e];
        float d;
        if (a.tube_sparse) {
          d = re[(size_t)j * TB];
        } else {
          const float l = re[(size_t)j * TB];
          if (a.last) a.out0[e] = l;
          const float w = a.first ? 0.f : a.state[e];
          d = m - w - l;
        }
        float sv;
        if (a.tube_sparse) {
          sv = f * d;
        } else {
          const float r = fabsf(d) - kappa;
          sv = r > 0.f ? (d > 0.f ? r : -r) : 0.f;
        }
        if (a.last) {
          a.out1[e] = sv;
        } else {
          const float wn = (sv - d) * a.ratio;
          a.state[e] = wn;
          re[(size_t)j * TB] = m - sv - wn;
        }
      }
      if (!a.last) {
        forward_tube<TB>(s, g, tid, a.fmat);
        store_spectrum<TB>(s, g, a.spec_out, t, tid);
      }
      break;
    }
    default:
      break;
  }
}

// Persistent over tiles: a CTA builds the tables once and takes tiles blockIdx.x, + gridDim.x, ...
template <int RM>
__global__ void __launch_bounds__(TILE_THREADS) tube_tile_kernel(TubeArgs a, int64_t ntiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
    tube_tile_body<RM>(a, tile * TT, smem_raw, tile == (int64_t)blockIdx.x);
}

template <int RM>
cudaError_t launch_tile(const TubeArgs& a, cudaStream_t st) {
  const size_t smem = tile_smem_bytes(a.g);
  cudaError_t e = cudaFuncSetAttribute(tube_tile_kernel<RM>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (a.g.N12 + TT - 1) / TT;
  // a persistent grid: the CTAs that fit on the device at once (or fewer tiles)
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tube_tile_kernel<RM>, TILE_THREADS,
                                                    smem);
  if (e != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  const int64_t grid = std::min<int64_t>(ntiles, (int64_t)per_sm * device_sm_count());
  tube_tile_kernel<RM><<<(unsigned)grid, TILE_THREADS, smem, st>>>(a, ntiles);
  return cudaGetLastError();
}

size_t tube_smem_bytes(const TubeGeom& g, int tb) {
  return (size_t)(g.nh + g.nf) * sizeof(float2) + (size_t)g.nf * g.hh * tb * sizeof(float2) +
         (size_t)g.nf * tb * sizeof(float2) + (size_t)g.nf * g.nh * tb * sizeof(float);
}

template <int TB>
cudaError_t launch_tb(const TubeArgs& a, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(tube_pass_kernel<TB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t grid = (a.g.N12 + TB - 1) / TB;
  if (grid > 0x7fffffff) return cudaErrorInvalidValue;
  tube_pass_kernel<TB><<<(unsigned)grid, TB, smem, st>>>(a);
  return cudaGetLastError();
}

__global__ void encode_observed_kernel(const float* __restrict__ M, const uint8_t* __restrict__ om,
                                       float* __restrict__ Yn, int64_t N, int* bad) {
  int local = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (om[e]) {
      const float m = M[e];
      if (!isfinite(m)) ++local;
      Yn[e] = m;
    } else {
      Yn[e] = __int_as_float(0x7fc00000);
    }
  }
  if (local) atomicAdd(bad, local);
}

__global__ void count_nonfinite_kernel(const float* __restrict__ x, int64_t N, int* bad) {
  int local = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N;
       e += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(x[e])) ++local;
  if (local) atomicAdd(bad, local);
}

__global__ void project_observed_kernel(const float* __restrict__ M, const uint8_t* __restrict__ om,
                                        float* __restrict__ X, int64_t N) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N;
       e += (int64_t)gridDim.x * blockDim.x)
    X[e] = om[e] ? M[e] : 0.f;
}

// out = (a x + b y + c z + d w) * scale, absent inputs (nullptr) counting as zero.
__global__ void combine4_kernel(float* __restrict__ out, const float* __restrict__ x, float a,
                                const float* __restrict__ y, float b, const float* __restrict__ z,
                                float c, const float* __restrict__ w, float d, float scale,
                                int64_t N) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N;
       e += (int64_t)gridDim.x * blockDim.x) {
    float v = 0.f;
    if (x) v = fmaf(a, x[e], v);
    if (y) v = fmaf(b, y[e], v);
    if (z) v = fmaf(c, z[e], v);
    if (w) v = fmaf(d, w[e], v);
    out[e] = v * scale;
  }
}

unsigned elementwise_grid(int64_t N) {
  int64_t b = (N + 255) / 256;
  const int64_t cap = (int64_t)device_sm_count() * 16;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (unsigned)b;
}

}  // namespace

int device_sm_count() {
  static int cached[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 1;
  }
  if (cached[dev] <= 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      return 1;
    }
    cached[dev] = n;
  }
  return cached[dev];
}

bool tube_pass_supported(const TubeGeom& g) {
  return tile_rm(g) > 0 || tube_smem_bytes(g, 32) <= 220 * 1024;
}

cudaError_t launch_tube_pass(const TubeArgs& a, cudaStream_t st) {
  if (a.g.N12 <= 0) return cudaSuccess;
  const int rm = tile_rm(a.g);
  if (rm == 2) return launch_tile<2>(a, st);
  if (rm == 4) return launch_tile<4>(a, st);
  if (rm == 8) return launch_tile<8>(a, st);
  size_t smem = tube_smem_bytes(a.g, 128);
  if (smem <= 110 * 1024) return launch_tb<128>(a, smem, st);
  smem = tube_smem_bytes(a.g, 64);
  if (smem <= 220 * 1024) return launch_tb<64>(a, smem, st);
  smem = tube_smem_bytes(a.g, 32);
  if (smem <= 220 * 1024) return launch_tb<32>(a, smem, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_encode_observed(const float* M, const uint8_t* omega, float* Yn, int64_t N,
                                   int* bad, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  encode_observed_kernel<<<elementwise_grid(N), 256, 0, st>>>(M, omega, Yn, N, bad);
  return cudaGetLastError();
}

cudaError_t launch_count_nonfinite(const float* x, int64_t N, int* bad, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  count_nonfinite_kernel<<<elementwise_grid(N), 256, 0, st>>>(x, N, bad);
  return cudaGetLastError();
}

cudaError_t launch_combine4(float* out, const float* x, float a, const float* y, float b,
                           const float* z, float c, const float* w, float d, float scale,
                           int64_t N, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  combine4_kernel<<<elementwise_grid(N), 256, 0, st>>>(out, x, a, y, b, z, c, w, d, scale, N);
  return cudaGetLastError();
}

cudaError_t launch_project_observed(const float* M, const uint8_t* omega, float* X, int64_t N,
                                    cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  project_observed_kernel<<<elementwise_grid(N), 256, 0, st>>>(M, omega, X, N);
  return cudaGetLastError();
}

}  // namespace tsvd
