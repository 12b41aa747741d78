// tsvd_noalloc.cu -- tsvt_static(): the t-SVT of tsvt() for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: a process that hands the whole device memory budget
// to its own pool allocator at start-up (a later cudaMalloc outside the pool fails or
// fragments it), or a latency-critical loop that must not pay the implicit device-wide
// synchronisation of cudaMalloc / cudaFree.  tsvt() allocates a workspace on its first call
// (and grows it), so it is closed to them.  tsvt_static() runs the same kernels with all of
// its scratch -- the two half spectra, the twiddle tables and the list of distinct Fourier
// slices -- carved from one file-scope __device__ array of kStaticScratchBytes (64 MiB).
// The caller still passes the input and output tensors (device memory).
//
// Facts a caller must know:
//  * The array is part of this library's device code: every GPU that loads the library holds
//    the 64 MiB until the process exits, whether or not tsvt_static() is called.
//  * In host code the array's name is only a host-side handle, not a device address.  The
//    first tsvt_static() call on a device (with that device current) looks the address up
//    once with cudaGetSymbolAddress and caches it per device; make that first call before
//    any stream capture.  The cached address belongs to the device's primary context, so
//    resetting the device (cudaDeviceReset) while the library is loaded is not supported.
//  * Every call on a device shares the one array and it keeps the last call's contents.
//    Nothing in it needs to start at zero: each call's first kernel writes the twiddle table
//    and the list of distinct Fourier slices from its launch arguments (no host buffer is
//    read), the forward pass writes every stored slice of the input spectrum and the SVT
//    kernel writes every slice that the inverse pass reads.  Calls that overlap on the GPU
//    (different streams, or different host threads without ordering) race on the array and
//    corrupt each other.
//  * No cudaMalloc, cudaFree or allocating library routine is called.
#include "tsvd.h"
#include "tsvd_internal.h"

#include <cmath>
#include <mutex>

using namespace tsvd;

namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;
constexpr size_t kAlign = 256;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_tsvt_scratch[kStaticScratchBytes];

void* g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Device address of g_tsvt_scratch on the current device (looked up once per device).
tsvd_status scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return TSVD_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return TSVD_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_tsvt_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return TSVD_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return TSVD_OK;
}

bool on_device(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// The tables a call needs, written by the device from the launch arguments: the twiddles
// (cos, sin)(2 pi m / n) of the half mode (n = nh) and of the full mode (n = nf, order 4), and
// the distinct stored slices in increasing order, by the same rules as tsvt() (twiddle_value,
// slice_is_distinct).
__global__ void static_tables_kernel(TubeGeom g, float2* __restrict__ twid, int* __restrict__ slices) {
  for (int m = threadIdx.x; m < g.nh + g.nf; m += blockDim.x)
    twid[m] = m < g.nh ? twiddle_value(m, g.nh) : twiddle_value(m - g.nh, g.nf);
  if (threadIdx.x == 0) {
    int n = 0;
    for (int kh = 0; kh < g.hh; ++kh)
      for (int kf = 0; kf < g.nf; ++kf)
        if (slice_is_distinct(g, kf, kh)) slices[n++] = kf + g.nf * kh;
  }
}

tsvd_status from_launch(cudaError_t e) {
  if (e == cudaSuccess) return TSVD_OK;
  if (e == cudaErrorInvalidValue) return TSVD_EUNSUPPORTED;
  return TSVD_ECUDA;
}

}  // namespace

extern "C" tsvd_status tsvt_static(const float* Y, float* Z, int order, const int64_t* dims,
                                   float tau, void* cuda_stream) {
  if (!Y || !Z || !dims || (order != 3 && order != 4)) return TSVD_EINVAL;
  if (!(tau >= 0.f) || !std::isfinite(tau)) return TSVD_EINVAL;
  for (int d = 0; d < order; ++d)
    if (dims[d] < 1) return TSVD_EINVAL;
  if (dims[0] > (1 << 30) || dims[1] > (1 << 30) || dims[2] > (1 << 20) ||
      (order == 4 && dims[3] > (1 << 20)))
    return TSVD_EUNSUPPORTED;

  TubeGeom g{};
  g.N12 = dims[0] * dims[1];
  g.nf = order == 4 ? (int)dims[2] : 1;
  g.nh = order == 4 ? (int)dims[3] : (int)dims[2];
  g.hh = g.nh / 2 + 1;
  g.nstore = g.nf * g.hh;
  if (order == 4) {   // one full-DFT mode (mode 3), as tsvt() sets it up
    g.nfm = 1;
    g.fdim[0] = g.nf;
  }
  if (!tube_pass_supported(g) || !jacobi_svt_supported((int)dims[0], (int)dims[1]))
    return TSVD_EUNSUPPORTED;

  // scratch layout: spectrum A | spectrum B | twiddles (nh + nf) | distinct slice list |
  // slice-SVT exchange buffers (multi-CTA slices)
  int ndistinct = 0;
  for (int kh = 0; kh < g.hh; ++kh)
    for (int kf = 0; kf < g.nf; ++kf)
      if (slice_is_distinct(g, kf, kh)) ++ndistinct;
  const size_t spec = align_up((size_t)g.nstore * (size_t)g.N12 * sizeof(float2));
  const size_t tw = align_up((size_t)(g.nh + g.nf) * sizeof(float2));
  const size_t lst = align_up((size_t)g.nstore * sizeof(int));
  const SliceKnobs knobs = {0, 0, 0, 0};
  const size_t jsc = align_up(jacobi_svt_scratch_bytes((int)dims[0], (int)dims[1], ndistinct, knobs));
  if (2 * spec + tw + lst + jsc > kStaticScratchBytes) return TSVD_ENOMEM;

  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return TSVD_ECUDA;
  }
  if (!on_device(Y, dev) || !on_device(Z, dev)) return TSVD_EINVAL;
  void* base = nullptr;
  tsvd_status st = scratch_address(&base);
  if (st != TSVD_OK) return st;
  char* b = static_cast<char*>(base);
  float2* spec_a = reinterpret_cast<float2*>(b);
  float2* spec_b = reinterpret_cast<float2*>(b + spec);
  float2* twid = reinterpret_cast<float2*>(b + 2 * spec);
  int* slices = reinterpret_cast<int*>(b + 2 * spec + tw);
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);

  static_tables_kernel<<<1, 256, 0, stream>>>(g, twid, slices);
  if ((st = from_launch(cudaGetLastError())) != TSVD_OK) return st;

  TubeArgs f{};
  f.g = g;
  f.mode = TUBE_FWD;
  f.twid_h = twid;
  f.twid_f = twid + g.nh;
  f.in = Y;
  f.spec_out = spec_a;
  f.ratio = 1.f;
  if ((st = from_launch(launch_tube_pass(f, stream))) != TSVD_OK) return st;

  SliceArgs s{};
  s.ahat = spec_a;
  s.zhat = spec_b;
  s.slices = slices;
  s.nslices = ndistinct;
  s.n1 = (int)dims[0];
  s.n2 = (int)dims[1];
  s.N12 = g.N12;
  s.tau = tau;
  tsvd_opts o;
  tsvd_default_opts(&o);
  s.tol = o.jacobi_tol;
  s.max_sweeps = o.max_sweeps;
  s.abs_stop = o.jacobi_stop == TSVD_STOP_SVT ? 1 : 0;
  s.stat = nullptr;
  s.acc = nullptr;
  s.scratch = jsc ? b + 2 * spec + tw + lst : nullptr;
  s.scratch_bytes = jsc;
  s.knobs = knobs;
  if ((st = from_launch(launch_jacobi_svt(s, stream))) != TSVD_OK) return st;

  TubeArgs inv{};
  inv.g = g;
  inv.mode = TUBE_INV;
  inv.twid_h = twid;
  inv.twid_f = twid + g.nh;
  inv.spec_in = spec_b;
  inv.out0 = Z;
  inv.ratio = 1.f;
  return from_launch(launch_tube_pass(inv, stream));
}
